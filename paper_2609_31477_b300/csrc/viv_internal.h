// Internal structures shared by the host runtime and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/viv.h"

namespace viv {

// ----- error handling --------------------------------------------------------
void set_error(const std::string& msg);
struct Error {
  vivStatus status;
  std::string msg;
};
#define VIV_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw ::viv::Error{VIV_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
#define VIV_CHECK(cond, code, msg)                 \
  do {                                             \
    if (!(cond)) throw ::viv::Error{code, (msg)};  \
  } while (0)

// ----- device memory ---------------------------------------------------------
struct DeviceArena {
  vivAllocator alloc{};
  bool custom = false;
  std::vector<void*> blocks;
  size_t bytes = 0;
  void* get(size_t n);
  template <class T>
  T* make(size_t count) { return static_cast<T*>(get(count * sizeof(T))); }
  template <class T>
  T* upload(const std::vector<T>& v, cudaStream_t s) {
    T* d = make<T>(v.size() ? v.size() : 1);
    if (!v.empty()) {
      VIV_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    return d;
  }
  void release();
  ~DeviceArena() { release(); }
};

// per node field slots of node_dof (the z slots stay -1 on 2-D meshes)
enum { S_UX = 0, S_UY = 1, S_UZ = 2, S_XX = 3, S_XY = 4, S_XZ = 5, S_P = 6, S_LX = 7, S_LY = 8, S_LZ = 9,
       NSLOT = 10 };

// local pairs of the element matrix scattered through e2nz (structural nonzeros)
constexpr int VOL_PAIRS = 1188;    // u rows x (u,x,p) + p rows x (u,x) + x rows x x
constexpr int FACE_PAIRS = 120;    // u x lambda, lambda x (u, delta), delta x lambda
// 3-D (27-node hexahedra, 8 pressure vertices, 9-node Gamma faces): element
// columns cs = 6 a + f (f < 3: u_f, else x_{f-3}) and 162 + c (pressure)
constexpr int VOL_PAIRS3 = 81 * 170 + 8 * 162 + 81 * 81;   // 21,627
constexpr int FACE_PAIRS3 = 243 + 243 + 18 + 18;            // u x lambda, lambda x u, lambda x delta, delta x lambda
__host__ __device__ inline int pairA3(int a, int i, int cs) { return (3 * a + i) * 170 + cs; }
__host__ __device__ inline int pairB3(int c, int cs) { return 13770 + c * 162 + cs; }
__host__ __device__ inline int pairC3(int a, int i, int b, int k) { return 15066 + (3 * a + i) * 81 + 3 * b + k; }
// P2-P1 triangles with a P1 position: columns u (2 a + i, a < 6), x of the
// vertices (12 + 2 v + k), pressure (18 + c); rows u (12), p (3), x (6)
constexpr int TRI_PAIRS = 12 * 21 + 3 * 18 + 6 * 6;   // 342
__host__ __device__ inline int tpairA(int a, int i, int cs) { return (2 * a + i) * 21 + cs; }
__host__ __device__ inline int tpairB(int c, int cs) { return 252 + c * 18 + cs; }
__host__ __device__ inline int tpairC(int v, int i, int w, int k) { return 306 + (2 * v + i) * 6 + 2 * w + k; }
__host__ __device__ inline int fpairD3(int b, int i, int bp) { return (3 * b + i) * 9 + bp; }
__host__ __device__ inline int fpairE3(int b, int i, int bp) { return 243 + (3 * b + i) * 9 + bp; }
__host__ __device__ inline int fpairG3(int b, int i) { return 486 + 2 * b + i; }
__host__ __device__ inline int fpairF3(int i, int bp) { return 504 + 9 * i + bp; }

// ----- blocked factorisation schedule ---------------------------------------
enum LaunchKind {
  L_ASSEMBLE = 0, L_PANEL = 1, L_TRSM = 2, L_GEMM = 3, L_PANEL_CL = 4, L_LASWP = 5, L_PANEL_1 = 6, L_TC_GEMM = 7,
  L_DIAG = 8,      // windowed pivoting: one warp factors the 32 x 32 diagonal block
  L_WINDOW = 9,    // windowed pivoting: L21 rows and permuted / solved columns
  L_TC_SPLIT = 10, // tensor-core operands: hi/lo TF32 images of the outer block's L21 and U12 chunks
  L_BLOCK_LU = 11, // windowed FP32: one CTA factors a large front's 128-column block, writes its inverse images
  L_BLOCK_PERM = 12  // windowed FP32: the block rows' permutation on the front's other columns
};
constexpr int WORK_STRIDE = 8;   // ints per work item
// work items:  ASSEMBLE (f, c0)           PANEL* (f)              LASWP (f, c0)
//              TRSM (f, c0, c_end, k)      GEMM (f, rb, cb, r_end, c_end, k_begin, k_len)
//              TC_SPLIT (f, start, kind, k0, klen, block, limit)  [one 128 x 32 operand chunk]
//              TC_GEMM (f, rb, cb, r_end, c_end, a_block, b_block, nchunks)  [128 x 128 tiles, tensor cores]
//              DIAG (f)   WINDOW (0, f, r0) rows of L21 | (1, f, c0, c_end) permuted / solved columns
//              BLOCK_LU (f, k2, a_inv_block, b_inv_block, nchunks)   BLOCK_PERM (f, k2, c0)
constexpr int WINDOW_THREADS = 256;   // rows or columns per WINDOW item
// solves: the bandwidth-bound products with the off-diagonal factor blocks run
// as items of SOLVE_ROWS rows x SOLVE_SLICE columns (one partial sum per slice)
constexpr int SOLVE_ROWS = 256;
constexpr int SOLVE_SLICE = 256;
// levels of small fronts form those products inside their chain CTAs instead
// (one thread per row, a loop over the columns), decided per tree level so a
// level runs one launch: forward when every front has at most SOLVE_FUSE_F
// pivots and 2 SOLVE_SLICE non-pivot rows, backward when every front has at
// most SOLVE_FUSE_B non-pivot columns and SOLVE_SLICE pivots (measured at
// 38,800 quads: longer loops lose to the multi-CTA slice products)
constexpr int SOLVE_FUSE_F = 64;
constexpr int SOLVE_FUSE_B = 200;
constexpr int PERM_SMEM_MAX = 200 * 1024;   // composed permutation of one front (2 ints per pivot)
constexpr int BIG_FRONT = 96;    // default: fronts at least this large use 128-column outer blocks
constexpr int OUTER_NB = 128;    // outer block width (K of the outer Schur update)
constexpr int MULTI_CHAIN_P = 512;   // block-LU fronts with this many pivots solve their chains on many CTAs
// operand images of the tensor-core updates: 32 KB per 128 x 32 chunk (hi + lo);
// the launches of one outer-block step are cut into groups of at most this
// many chunks, which bounds each mixed case's image buffer (256 MB)
constexpr int64_t TC_IMG_CHUNK_BYTES = 32 * 1024;
constexpr int64_t TC_IMG_MAX_CHUNKS = 8192;
struct Launch {
  int kind;
  int level;
  int k;          // panel start (pivot index) for PANEL/LASWP
  int64_t item0;  // first work item
  int64_t count;  // work items
  int aux = 0;    // PANEL_CL: rows per CTA (shared-memory sizing); ASSEMBLE: threads per item
};

constexpr int PANEL_NB = 32;    // pivot block
constexpr int GEMM_TILE = 64;   // Schur update tile
constexpr int TRSM_COLS = 64;   // columns per TRSM item
constexpr int ASM_COLS = 32;    // parent columns per assembly item
constexpr int PANEL_CLUSTER = 8;          // CTAs per panel cluster
constexpr int PANEL_SMEM_BYTES = 200 * 1024;   // panel rows held per CTA in shared memory
constexpr int LASWP_COLS = 256;           // columns per row-interchange item

struct FrontTables {              // device copies
  int32_t n_fronts = 0;
  int64_t* off = nullptr;         // front storage offset (entries)
  int32_t* m = nullptr;           // order
  int32_t* p = nullptr;           // pivots
  int32_t* first = nullptr;       // first own dof
  int64_t* idx_off = nullptr;     // index list offset
  int32_t* idx = nullptr;         // global dof of each front row/col
  int64_t* nz_off = nullptr;      // original-entry list, sorted by local column
  int32_t* nz_csr = nullptr;
  int32_t* nz_pos = nullptr;      // local position row + col*m
  int32_t* child_off = nullptr;   // children list
  int32_t* child = nullptr;
  int64_t* ea_off = nullptr;      // per front: positions of its CB in the parent
  int32_t* ea = nullptr;
  int32_t* parent = nullptr;
  int64_t* vec_off = nullptr;     // solve workspace offset (entries)
  int32_t* piv_off = nullptr;     // pivot list offset
  int32_t* col_nz = nullptr;      // per front, per ASM_COLS chunk: first nz of the chunk (relative)
  int64_t* col_nz_off = nullptr;
  int32_t* work = nullptr;        // all work items (3 ints each)
};

struct Mesh {
  // host copies
  int64_t n_nodes = 0, n_elems = 0, n_faces = 0;
  int dim = 2;                     // 2: Q2 quads; 3: Q2 hexahedra
  bool tri = false;                // P2-P1 triangles with a P1 position (2-D)
  std::vector<int32_t> mid_parent; // triangles: per node the end vertices of its edge (-1: a vertex)
  int npe = 9, nvert = 4, fpe = 3; // nodes per element, pressure vertices, nodes per Gamma face
  int vol_pairs = VOL_PAIRS, face_pairs = FACE_PAIRS;
  double span = 0;                 // 3-D: period in z (0: not periodic)
  std::vector<double> X;           // n x dim
  std::vector<int32_t> conn;       // E x npe
  std::vector<int32_t> wrap;       // 3-D: per element, bit a: local node a at X + span e_z
  std::vector<int32_t> tags;
  std::vector<int32_t> faces;      // F x fpe node ids (along the edge / in face order)
  std::vector<int32_t> face_wrap;  // 3-D: per face, bit b: face node b at X + span e_z
  std::vector<int32_t> face_elem;
  std::vector<int32_t> node_dof;   // n x NSLOT
  std::vector<int32_t> delta_dof;  // 2 (or -1)
  int64_t n_dofs = 0;
  int64_t n_front_dofs = 0;        // unknowns the fronts hold: all but delta (numbered last)
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col;
  std::vector<int32_t> e2nz;       // E x VOL_PAIRS
  std::vector<int32_t> f2nz;       // F x FACE_PAIRS
  int32_t dd_nz[2] = {-1, -1};     // CSR slots of (delta_i, delta_i)
  // border of the Jacobian, J = [A B; C D] with the two delta unknowns last:
  // C = delta rows in front columns (bc_col / bc_q, rows split at bc_off),
  // B = delta columns in front rows (bb_row / bb_q, columns split at bb_off),
  // D slots bd_q[2 i + j] (-1 where structurally zero)
  std::vector<int32_t> bc_off, bc_col, bc_q, bb_off, bb_row, bb_q;
  int32_t bd_q[4] = {-1, -1, -1, -1};
  std::vector<int32_t> color_off;  // element colours: elements sorted by colour
  std::vector<int32_t> color_elems;
  std::vector<int32_t> fcolor_off;
  std::vector<int32_t> fcolor_faces;
  std::vector<int64_t> dof_node;
  std::vector<int32_t> dof_field;
  // fronts (host)
  int n_fronts = 0, n_levels = 0, max_front = 0;
  std::vector<int64_t> f_off, f_idx_off, f_nz_off, f_ea_off, f_vec_off, f_col_nz_off;
  std::vector<int32_t> f_m, f_p, f_first, f_idx, f_nz_csr, f_nz_pos, f_child_off, f_child, f_ea,
      f_parent, f_piv_off, f_col_nz, f_level;
  std::vector<int32_t> work;
  std::vector<Launch> sched[4];    // numeric factorisation launches in order: [FP64 + 2 * windowed pivoting]
  std::vector<int32_t> level_off;  // fronts sorted by level
  std::vector<int32_t> level_fronts;
  std::vector<int32_t> level_maxm;   // largest front order per level
  std::vector<int32_t> level_threads;  // solve threads per front at each level
  std::vector<int32_t> level_maxp;     // largest pivot count per level
  int max_p = 0;                       // largest pivot count of any front
  std::vector<int32_t> inv_items;      // (front, first row) of every 32 x 32 diagonal block
  std::vector<uint8_t> solve_fused;    // per front: 1 forward, 2 backward slice products in the chain CTA
  // windowed FP32 schedule: fronts whose 128-column blocks the block LU
  // factors (it stores each block's diagonal part inverted: the solves step
  // 128 rows at a time there), and the 32 x 32 inversions left for the others
  std::vector<uint8_t> blk_front;      // 1: block-LU front, 2: and its solve chains span many CTAs
  std::vector<int8_t> level_block;     // per tree level: the block LU allowed (empty: every level; autotuner)
  std::vector<int32_t> inv_items_blk;
  // multi-CTA solve chains (block-LU fronts of order >= MULTI_CHAIN_P): per
  // level, tasks (front, block, first flag) in dependency order (forward:
  // blocks top down, backward: bottom up; fronts interleaved), and one flag
  // per block (per case: chain_flag_bound covers any large-front threshold)
  std::vector<int32_t> mc_fwd, mc_bwd, mc_off;
  int32_t mc_flags = 0, chain_flag_bound = 0;
  std::vector<int32_t> fg_items, fg_off;   // forward slice items (f, r0, slice, 0) by level
  std::vector<int32_t> bg_items, bg_off;   // backward slice items by level
  int64_t front_entries = 0, vec_entries = 0, piv_entries = 0;
  double factor_flops = 0;
  int big_front = 0;          // large-front threshold of the current schedules
  size_t work_cap = 0;        // device capacity of the work-item array
  int sched_version = 0;      // bumped whenever the schedules are rebuilt
  double gemm_flops = 0, panel_flops = 0, trsm_flops = 0;   // per numeric factorisation
  double outer_flops = 0;   // part of gemm_flops done by the K = 128 outer updates (tensor cores)
  int64_t tc_img_chunks = 0;   // image chunks a mixed case holds: the largest group of any schedule
  int64_t tc_split_chunks = 0, tc_tiles = 0;   // per numeric factorisation: chunks split, tiles updated
  bool block_lu = true;        // FP32 windowed schedule: 128-column blocks of large fronts by block_lu_kernel
  double window_tc_flops = 0;  // per factorisation of that schedule: tensor-core flops,
  double window_lu_flops = 0;  //   pivot-block LU flops (block inverses included),
  double window_gemm_flops = 0;//   SIMT Schur-update flops
  // device copies
  cudaStream_t stream = nullptr;
  bool on_device = false;
  DeviceArena arena;
  double* d_X = nullptr;
  int32_t* d_conn = nullptr;
  int32_t* d_wrap = nullptr;
  int32_t* d_mid_parent = nullptr;
  int32_t* d_face_wrap = nullptr;
  double* d_hex_tab = nullptr;         // 3-D: shape-function tables at the Gauss points (FP64, FP32)
  float* d_hex_tab_f = nullptr;
  int32_t* d_tags = nullptr;
  int32_t* d_faces = nullptr;
  int32_t* d_node_dof = nullptr;
  int32_t* d_delta_dof = nullptr;
  int64_t* d_row_ptr = nullptr;
  int32_t* d_col = nullptr;
  int32_t* d_e2nz = nullptr;
  int32_t* d_f2nz = nullptr;
  int32_t* d_color_elems = nullptr;
  int32_t* d_fcolor_faces = nullptr;
  int32_t* d_level_fronts = nullptr;
  int32_t* d_inv_items = nullptr;
  uint8_t* d_solve_fused = nullptr;
  uint8_t* d_blk_front = nullptr;      // (device copies, sized once: n_fronts / inv_items)
  int32_t* d_inv_items_blk = nullptr;
  int32_t* d_mc_fwd = nullptr;         // (device copies, sized for the largest task list)
  int32_t* d_mc_bwd = nullptr;
  size_t mc_cap = 0;
  int32_t* d_fg_items = nullptr;
  int32_t* d_bg_items = nullptr;
  int32_t *d_bc_col = nullptr, *d_bc_q = nullptr, *d_bb_row = nullptr, *d_bb_q = nullptr;
  FrontTables ft;
};

// device state of one case
struct CaseState {
  double *u, *p, *x, *lam, *delta;      // current iterate
  double *u_n, *x_n, *u_nm1, *x_nm1;    // history
  double *hu, *hx;                      // BDF history part of the nodal rates
  double* lame;                         // per element lambda_s (= mu_s)
  double* R;                            // residual (n_dofs)
  double* dU;                           // Newton correction
  double* r;                            // refinement residual
  double* d;                            // one refinement correction
  double* mR;                           // right-hand side of the refined solve
  double* y2;                           // solution of viv_solve_rhs
  double* J64;                          // CSR values (FP64 path and refinement)
  float* J32;                           // CSR values (mixed path)
  void* fronts;                         // front pool (double or float)
  void* vec;                            // solve workspace (double or float)
  void* yv;                             // forward-solve vector (n_dofs)
  int32_t* piv;                         // row pivots of all fronts
  int32_t* perm;                        // composed row permutation of each front (solves)
  int32_t* stats;                       // [0] perturbed, [1] threshold misses, [2] a bounded device wait expired
  int32_t* chain;                       // multi-CTA solve chains: task counter + one flag per block
  unsigned char* tc_img;                // operand images of the tensor-core updates (mixed path)
  double* Y;                            // border: A^{-1} B (2 columns of n_dofs; rows < n_front_dofs used)
  double* Sb;                           // border: S_b = D - C Y (4) and its inverse (4), FP64
  double* btmp;                         // border: delta of the current solve (2) and scratch
  double* Bcol;                         // border: the two columns of B as dense vectors (2 x n_dofs)
  void* vec2;                           // border: solve workspaces of the two columns (2 x vec_entries, T)
  void* yv2;                            // border: forward-solve vectors of the two columns (2 x n_dofs, T)
  double* partial;                      // norm partial sums
  double* scal;                         // host-visible scalars (device side)
  double* step;                         // {time of the step being solved, BDF rate coefficient c0}
};

}  // namespace viv

// ----- launch accounting and per-kind event timing ----------------------------
namespace viv {
enum KernelKind {
  K_RES = 0, K_JAC, K_FACE, K_FRONT_ASM, K_PANEL, K_TRSM, K_GEMM, K_FWD, K_BWD, K_SPMV, K_VEC, K_TCGEMM, K_TCSPLIT,
  K_NKINDS
};
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind, level;
  size_t used = 0;
  int cur_level = -1;                 // tree level of the factorisation launches being issued (-1: none)
  std::vector<double> level_ms;       // [level][kind] factorisation time of the last read
  void start(int k, cudaStream_t s);
  void stop(cudaStream_t s);
  void read(double* ms, int64_t* count);   // synchronises on the recorded events
  ~Profiler();
};
// tag the factorisation launches that follow with their tree level (profiling only)
void prof_level(int l);
extern thread_local Profiler* g_prof;
void count_launch();
void count_launches(int64_t n);
int64_t launches();
struct Launched {           // wraps one kernel launch: counts it and, when profiling, times it
  cudaStream_t s;
  bool timed;
  Launched(int k, cudaStream_t st) : s(st), timed(g_prof && g_prof->on) {
    count_launch();
    if (timed) g_prof->start(k, s);
  }
  ~Launched() {
    if (timed) g_prof->stop(s);
  }
};
}  // namespace viv

struct vivMesh {
  viv::Mesh m;
};

struct vivCase {
  vivMesh* mesh = nullptr;
  vivParams prm{};
  cudaStream_t stream = nullptr;
  viv::DeviceArena arena;
  viv::CaseState s{};
  double t = 0.0;
  int nstep = 0;
  bool have_prev2 = false;     // BDF2 available for the next step
  bool step_open = false;      // begin_step called
  double c0 = 0.0;             // rate coefficient of the current step
  double dt_prev = 0.0;        // size of the previous step (variable-step BDF2)
  bool factored = false;
  bool have_dU = false;
  double* h_pinned = nullptr;  // pinned scalars
  viv::Profiler prof;
  // CUDA graphs of the per-iteration phases (captured on first use; re-captured
  // when the mesh schedule changes; not used while profiling or on stream 0)
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;   // kernel launches captured in the graph (added to the counter per replay)
  };
  bool graphs = true;
  int graph_version = -1;
  Graph g_res, g_upd_res, g_jac, g_fac, g_sinit, g_sweep;
};

// kernels (defined in .cu files), all launched on the case stream
namespace viv {
void launch_element_areas(const Mesh& m, double* lame, double scale, bool constant, double* scratch,
                          cudaStream_t s);
void launch_quasi_init(const Mesh& m, const CaseState& st, const vivParams& prm, cudaStream_t s);
// P2-P1 triangle element kernels and the midside positions (assembly_tri.cu)
template <class T, bool JAC>
void run_assembly_tri(const Mesh& m, const CaseState& st, const vivParams& prm, double* R, T* vals, cudaStream_t s);
void launch_triangle_areas(const Mesh& m, double* area, cudaStream_t s);
void launch_midside_positions(const Mesh& m, double* x, cudaStream_t s);
// 3-D (hexahedral) element, face and border kernels (assembly3d.cu)
void upload_hex_tables(Mesh& m, cudaStream_t s);
void prepare_hex_kernels();
void launch_element_volumes(const Mesh& m, double* vol, cudaStream_t s);
template <class T, bool JAC>
void run_assembly3(const Mesh& m, const CaseState& st, const vivParams& prm, double* R, T* vals, cudaStream_t s,
                   int parts);
void launch_residual(const Mesh& m, const CaseState& st, const vivParams& prm, cudaStream_t s);
template <class T>
void launch_jacobian(const Mesh& m, const CaseState& st, const vivParams& prm, T* vals, cudaStream_t s);
void launch_norm2(const double* v, int64_t n, double* partial, double* out, cudaStream_t s);
void launch_step_constants(const CaseState& st, double t_new, double c0, cudaStream_t s);
void launch_mms_dirichlet(const Mesh& m, const CaseState& st, const vivParams& prm, cudaStream_t s);
void launch_bdf_history(const Mesh& m, CaseState& st, double a_n, double a_nm1, bool shift, cudaStream_t s);
void launch_extrapolate(const Mesh& m, CaseState& st, double w, cudaStream_t s);
double launch_cfl(const Mesh& m, const CaseState& st, double dt, double* partial, double* out, double* host,
                  cudaStream_t s);
void launch_update(const Mesh& m, CaseState& st, const double* dU, cudaStream_t s);
void launch_spmv_residual(const Mesh& m, const double* J, const double* x, const double* b, double* r,
                          cudaStream_t s);
void launch_axpy(double* y, const double* x, double a, int64_t n, cudaStream_t s);
void launch_scale_copy(double* y, const double* x, double a, int64_t n, cudaStream_t s);
void launch_f64_to_f32(float* y, const double* x, int64_t n, cudaStream_t s);
void launch_f32_to_f64(double* y, const float* x, int64_t n, cudaStream_t s);
void launch_jacobian_split(const Mesh& m, const CaseState& st, const vivParams& prm, float* J32, double* J64,
                           cudaStream_t s);
// border of the Jacobian (the two delta unknowns, eliminated after the fronts)
void launch_border_column(const Mesh& m, const double* J, int j, double* dst, cudaStream_t s);
void launch_border_schur(const Mesh& m, const double* J, const double* Y, double* Sb, int32_t* flag,
                         cudaStream_t s);
void launch_border_solve(const Mesh& m, const double* J, const double* b, double* x, const double* Y,
                         const double* Sb, double* dtmp, cudaStream_t s);
template <class T>
void prepare_kernels();
template <class T>
void factor_numeric(const Mesh& m, const double* J64, const float* J32, T* fronts, int32_t* piv, int32_t* perm,
                    int32_t* stats, double threshold, bool window, unsigned char* tc_img, cudaStream_t s);
// the case's factors come from the block LU (mixed precision, windowed pivoting)
bool block_factors(const vivCase* c);
int device_sm_count();   // streaming multiprocessors of the current device
// blk: the factors come from the block LU of the windowed FP32 schedule
// (diagonal 128-blocks of the flagged fronts stored inverted)
// (chain: the case's multi-CTA chain flags, err: its expired-wait flag;
// both used with blk)
template <class T>
void solve_fronts(const Mesh& m, const T* fronts, const int32_t* perm, const double* b, double* x,
                  T* vec, T* yv, bool blk, int32_t* chain, int32_t* err, cudaStream_t s);
template <class T>
void solve_fronts2(const Mesh& m, const T* fronts, const int32_t* perm, const double* b, double* x, T* vec, T* yv,
                   bool blk, int32_t* chain, int32_t* err, cudaStream_t s);
}  // namespace viv

// ----- canonical order of the element matrix pairs scattered through e2nz ----
// element column slots: 4*b + f (node b, f = u_x, u_y, x_x, x_y), 36 + c (pressure vertex c)
namespace viv {
__host__ __device__ inline int pairA(int a, int i, int cs) { return (2 * a + i) * 40 + cs; }     // u row x any
__host__ __device__ inline int pairB(int c, int cs) { return 720 + c * 36 + cs; }               // p row x (u,x)
__host__ __device__ inline int pairC(int a, int i, int b, int k) { return 864 + (2 * a + i) * 18 + 2 * b + k; }
// face slots along the edge: b = 0..2
__host__ __device__ inline int fpairD(int b, int i, int bp, int k) { return (2 * b + i) * 6 + 2 * bp + k; }   // u x lambda
__host__ __device__ inline int fpairE(int b, int i, int cs12) { return 36 + (2 * b + i) * 12 + cs12; }     // lambda x (u | x->delta)
__host__ __device__ inline int fpairF(int i, int bp, int k) { return 108 + i * 6 + 2 * bp + k; }             // delta x lambda
}  // namespace viv

