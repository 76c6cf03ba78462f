// C ABI entry points: argument checks, the case state machine, the Newton /
// BDF driver (Eq. NR_iteration; BDF1 first step then BDF2) and the
// refinement loop of the linear solve.  All device work of a case is ordered
// on its stream; the host only reads back scalars (norms) to steer Newton.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>

#include "viv_internal.h"

namespace viv {
void tc_gemm_update(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int M, int N, int K,
                    int* err, cudaStream_t s);
void lu_solve_noalloc(vivCase* c, const double* b, double* x);
void noalloc_prepare();
void build_mesh(Mesh& m, const vivMeshDesc* d);
void upload_mesh(Mesh& m, cudaStream_t s);
void build_schedule(Mesh& m, int big_front);
void upload_work(Mesh& m, cudaStream_t s);

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
// the factors come from the block LU (mixed precision, windowed pivoting)
bool block_factors(const vivCase* c) {
  return c->prm.precision == VIV_MIXED && c->prm.pivoting == VIV_PIVOT_WINDOW && c->mesh->m.block_lu;
}

}  // namespace viv

using namespace viv;

#define API_BEGIN try {
#define API_END                              \
  }                                          \
  catch (const viv::Error& e) {              \
    set_error(e.msg);                        \
    return e.status;                         \
  }                                          \
  catch (const std::bad_alloc&) {            \
    set_error("host allocation failed");     \
    return VIV_ERR_OOM;                      \
  }                                          \
  catch (const std::exception& e) {          \
    set_error(e.what());                     \
    return VIV_ERR_ARG;                      \
  }                                          \
  return VIV_OK;

namespace {

// binds the case's profiler to this thread for the duration of an API call
struct ProfBind {
  Profiler* prev;
  explicit ProfBind(vivCase* c) : prev(g_prof) { g_prof = c ? &c->prof : nullptr; }
  ~ProfBind() { g_prof = prev; }
};

bool mixed(const vivCase* c) { return c->prm.precision == VIV_MIXED; }

std::string fmt_e(double v) {
  char b[32];
  std::snprintf(b, sizeof b, "%.3e", v);
  return b;
}

double read_scalar(vivCase* c, const double* dptr) {
  VIV_CUDA(cudaMemcpyAsync(c->h_pinned, dptr, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  VIV_CUDA(cudaStreamSynchronize(c->stream));
  return c->h_pinned[0];
}

double norm2(vivCase* c, const double* v, int64_t n) {
  launch_norm2(v, n, c->s.partial, c->s.scal, c->stream);
  return read_scalar(c, c->s.scal);
}

void drop_graphs(vivCase* c) {
  for (vivCase::Graph* g : {&c->g_res, &c->g_upd_res, &c->g_jac, &c->g_fac, &c->g_sinit, &c->g_sweep})
    if (g->exec) {
      cudaGraphExecDestroy(g->exec);
      g->exec = nullptr;
      g->kernels = 0;
    }
}

// Run `body` (a fixed sequence of launches on the case stream) through a CUDA
// graph captured on first use; plain launches while profiling, on the legacy
// default stream, or with graphs switched off.
template <class F>
void run_graph(vivCase* c, vivCase::Graph& g, F&& body) {
  if (!c->graphs || c->stream == nullptr || c->prof.on) {
    body();
    return;
  }
  // kernel arguments are captured by value: the schedule version keys the
  // graphs (the step's time and BDF coefficient reach the kernels through
  // device memory, so the same graphs serve every step size)
  if (c->graph_version != c->mesh->m.sched_version) {
    drop_graphs(c);
    c->graph_version = c->mesh->m.sched_version;
  }
  if (!g.exec) {
    cudaGraph_t graph = nullptr;
    const int64_t before = launches();
    VIV_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    try {
      body();
    } catch (...) {
      cudaStreamEndCapture(c->stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    VIV_CUDA(cudaStreamEndCapture(c->stream, &graph));
    g.kernels = launches() - before;
    count_launches(-g.kernels);   // counted when the graph runs, not when it is captured
    cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    VIV_CUDA(e);
  }
  VIV_CUDA(cudaGraphLaunch(g.exec, c->stream));
  count_launches(g.kernels);
}

void copy_in(vivCase* c, double* dst, const double* src, size_t count) {
  if (src) VIV_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, c->stream));
}
void copy_out(vivCase* c, double* dst, const double* src, size_t count) {
  if (dst) VIV_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, c->stream));
}

void begin_step(vivCase* c) {
  const Mesh& m = c->mesh->m;
  CaseState& s = c->s;
  const bool bdf2 = c->nstep > 0 || c->have_prev2;
  if (bdf2) {
    std::swap(s.u_nm1, s.u_n);
    std::swap(s.x_nm1, s.x_n);
  }
  const size_t n2 = m.dim * m.n_nodes * sizeof(double);
  VIV_CUDA(cudaMemcpyAsync(s.u_n, s.u, n2, cudaMemcpyDeviceToDevice, c->stream));
  VIV_CUDA(cudaMemcpyAsync(s.x_n, s.x, n2, cudaMemcpyDeviceToDevice, c->stream));
  const double dt = c->prm.dt;
  if (bdf2) {
    // BDF2 with step ratio w = dt / dt_prev: the derivative at t^{n+1} of the
    // quadratic through the last three levels
    const double w = dt / c->dt_prev;
    c->c0 = (1 + 2 * w) / ((1 + w) * dt);
    launch_bdf_history(m, s, -(1 + w) / dt, w * w / ((1 + w) * dt), false, c->stream);
    if (c->prm.predictor == 1) launch_extrapolate(m, s, w, c->stream);
  } else {
    c->c0 = 1.0 / dt;
    launch_bdf_history(m, s, -1.0 / dt, 0.0, false, c->stream);
  }
  launch_step_constants(s, c->t + dt, c->c0, c->stream);
  // time-dependent manufactured solution: the Dirichlet data of the new time
  // level (the history keeps the previous level's)
  if (c->prm.source == 2) launch_mms_dirichlet(m, s, c->prm, c->stream);
  c->step_open = true;
  c->factored = false;
  c->have_dU = false;
}

// Jacobian values: FP64 element arithmetic (rounded to FP32 for the mixed
// fronts), or, with jacobian_fp32 on the mixed path, FP32 arithmetic for the
// volume elements and FP64 for the Gamma faces and border rows (widened to
// FP64 for the refinement products)
void jacobian(vivCase* c) {
  const Mesh& m = c->mesh->m;
  const int64_t nnz = m.row_ptr[m.n_dofs];
  if (mixed(c) && c->prm.jacobian_fp32) {
    launch_jacobian_split(m, c->s, c->prm, c->s.J32, c->s.J64, c->stream);
  } else {
    launch_jacobian<double>(m, c->s, c->prm, c->s.J64, c->stream);
    if (mixed(c)) launch_f64_to_f32(c->s.J32, c->s.J64, nnz, c->stream);
  }
}

double assemble(vivCase* c, int what, bool want_norm) {
  const Mesh& m = c->mesh->m;
  VIV_CHECK(c->step_open, VIV_ERR_STATE, "viv_assemble before viv_begin_step");
  double nr = 0;
  if (what & VIV_RES) {
    launch_residual(m, c->s, c->prm, c->stream);
    if (want_norm) nr = norm2(c, c->s.R, m.n_dofs);
  }
  if (what & VIV_JAC) {
    jacobian(c);
    c->factored = false;
  }
  return nr;
}

bool has_border(const Mesh& m) { return m.n_front_dofs < m.n_dofs; }


// x[0 : n_front_dofs] = A^{-1} b[0 : n_front_dofs] with the fronts' factors
void front_solve(vivCase* c, const double* b, double* x) {
  const Mesh& m = c->mesh->m;
  if (mixed(c))
    solve_fronts<float>(m, (const float*)c->s.fronts, c->s.perm, b, x, (float*)c->s.vec, (float*)c->s.yv,
                        block_factors(c), c->s.chain, c->s.stats + 2, c->stream);
  else
    solve_fronts<double>(m, (const double*)c->s.fronts, c->s.perm, b, x, (double*)c->s.vec,
                         (double*)c->s.yv, false, nullptr, nullptr, c->stream);
}

// Numeric factorisation of A (the Jacobian without the delta rows and
// columns) in the fronts, then the border: Y = A^{-1} B with those factors
// and the 2 x 2 Schur block S_b = D - C Y formed and inverted in FP64
// (Eq. coupling_constraint: the force-position rows eliminated last).
void factor(vivCase* c) {
  const Mesh& m = c->mesh->m;
  double thr = c->prm.pivot_threshold > 0 ? c->prm.pivot_threshold : 0.01;
  const bool win = c->prm.pivoting == VIV_PIVOT_WINDOW;
  if (mixed(c))
    factor_numeric<float>(m, nullptr, c->s.J32, (float*)c->s.fronts, c->s.piv, c->s.perm, c->s.stats, thr, win,
                          c->s.tc_img, c->stream);
  else
    factor_numeric<double>(m, c->s.J64, nullptr, (double*)c->s.fronts, c->s.piv, c->s.perm, c->s.stats, thr, win,
                           nullptr, c->stream);
  if (has_border(m)) {
    // both columns of B through the fronts in one pass
    for (int j = 0; j < 2; ++j) launch_border_column(m, c->s.J64, j, c->s.Bcol + (int64_t)j * m.n_dofs, c->stream);
    if (mixed(c))
      solve_fronts2<float>(m, (const float*)c->s.fronts, c->s.perm, c->s.Bcol, c->s.Y, (float*)c->s.vec2,
                           (float*)c->s.yv2, block_factors(c), c->s.chain, c->s.stats + 2, c->stream);
    else
      solve_fronts2<double>(m, (const double*)c->s.fronts, c->s.perm, c->s.Bcol, c->s.Y, (double*)c->s.vec2,
                            (double*)c->s.yv2, false, nullptr, nullptr, c->stream);
    launch_border_schur(m, c->s.J64, c->s.Y, c->s.Sb, c->s.stats + 3, c->stream);
  }
  c->factored = true;
}

// x = J^{-1} b for the factored J = [A B; C D]: z = A^{-1} b_A from the
// fronts, delta = S_b^{-1} (b_delta - C z), x_A = z - Y delta
void lu_solve(vivCase* c, const double* b, double* x) {
  const Mesh& m = c->mesh->m;
  front_solve(c, b, x);
  if (has_border(m)) launch_border_solve(m, c->s.J64, b, x, c->s.Y, c->s.Sb, c->s.btmp, c->stream);
}

// y = J^{-1} b with refinement against the FP64 Jacobian; b, y device
int refined_solve(vivCase* c, const double* b, double* y) {
  const Mesh& m = c->mesh->m;
  CaseState& s = c->s;
  const int64_t n = m.n_dofs;
  VIV_CHECK(c->factored, VIV_ERR_STATE, "solve before factor");
  const int max_sweeps = 1 + (c->prm.refine_max > 0 ? c->prm.refine_max : (mixed(c) ? 10 : 1));
  const double tol = c->prm.refine_tol > 0 ? c->prm.refine_tol : 1e-13;
  double nb = norm2(c, b, n);
  VIV_CUDA(cudaMemsetAsync(y, 0, n * sizeof(double), c->stream));
  VIV_CUDA(cudaMemcpyAsync(s.r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  int sweeps = 0;
  for (;;) {
    lu_solve(c, s.r, s.d);
    launch_axpy(y, s.d, 1.0, n, c->stream);
    ++sweeps;
    if (sweeps >= max_sweeps || nb == 0) break;
    launch_spmv_residual(m, s.J64, y, b, s.r, c->stream);
    double nr = norm2(c, s.r, n);
    VIV_CHECK(std::isfinite(nr), VIV_ERR_NONFINITE, "refinement residual is not finite");
    if (nr <= tol * nb) break;
  }
  return sweeps;
}

}  // namespace

extern "C" {

const char* viv_last_error(void) { return g_err.c_str(); }
const char* viv_version(void) { return "viv-b300 0.1 (sm_103a)"; }

int64_t viv_kernel_launches(void) { return launches(); }

vivStatus viv_profile(vivCase* c, int on) {
  API_BEGIN
  VIV_CHECK(c, VIV_ERR_ARG, "NULL case");
  c->prof.on = on != 0;
  c->prof.used = 0;
  API_END
}

vivStatus viv_profile_read(vivCase* c, double* ms, int64_t* count) {
  API_BEGIN
  VIV_CHECK(c && ms && count, VIV_ERR_ARG, "NULL argument");
  c->prof.read(ms, count);
  API_END
}

vivStatus viv_profile_levels(const vivCase* c, double* ms, int32_t max_levels, int32_t* n_levels) {
  API_BEGIN
  VIV_CHECK(c && n_levels && (max_levels <= 0 || ms), VIV_ERR_ARG, "NULL argument");
  const std::vector<double>& lv = c->prof.level_ms;
  const int32_t nl = (int32_t)(lv.size() / K_NKINDS);
  *n_levels = nl;
  for (int32_t l = 0; l < max_levels && l < nl; ++l)
    for (int k = 0; k < K_NKINDS; ++k) ms[(int64_t)l * K_NKINDS + k] = lv[(int64_t)l * K_NKINDS + k];
  API_END
}

vivStatus viv_mesh_create(const vivMeshDesc* desc, const vivAllocator* alloc, void* stream, vivMesh** out) {
  API_BEGIN
  VIV_CHECK(out, VIV_ERR_ARG, "out is NULL");
  *out = nullptr;
  vivMesh* h = new vivMesh();
  try {
    if (alloc && alloc->alloc && alloc->free) {
      h->m.arena.alloc = *alloc;
      h->m.arena.custom = true;
    }
    h->m.stream = (cudaStream_t)stream;
    build_mesh(h->m, desc);
    upload_mesh(h->m, (cudaStream_t)stream);
    h->m.on_device = true;
  } catch (...) {
    delete h;
    throw;
  }
  *out = h;
  API_END
}

vivStatus viv_mesh_analyze(const vivMeshDesc* desc, vivMesh** out) {
  API_BEGIN
  VIV_CHECK(out, VIV_ERR_ARG, "out is NULL");
  *out = nullptr;
  vivMesh* h = new vivMesh();
  try {
    build_mesh(h->m, desc);
  } catch (...) {
    delete h;
    throw;
  }
  *out = h;
  API_END
}

vivStatus viv_mesh_info(const vivMesh* mesh, vivMeshInfo* info) {
  API_BEGIN
  VIV_CHECK(mesh && info, VIV_ERR_ARG, "NULL argument");
  const Mesh& m = mesh->m;
  info->n_dofs = m.n_dofs;
  info->nnz = m.row_ptr[m.n_dofs];
  info->n_fronts = m.n_fronts;
  info->max_front = m.max_front;
  info->n_levels = m.n_levels;
  info->factor_flops = m.factor_flops;
  info->front_entries = (size_t)m.front_entries;
  size_t nodes = (size_t)m.n_nodes, nnz = (size_t)info->nnz, nd = (size_t)m.n_dofs;
  // nodal vectors: u, x, lambda, two history levels of u and x, the BDF sums (D each), p
  size_t state = 8 * ((9 * (size_t)m.dim + 1) * nodes + (size_t)m.n_elems + 3 * nd + 2 * 296 + 64) +
                 8 * (size_t)m.piv_entries +
                 4 * (1 + (size_t)std::max(1, m.chain_flag_bound));   // (+ the solve chains' flags)
  if (m.n_front_dofs < m.n_dofs) state += 8 * 4 * nd;   // border: Y and the columns of B
  const size_t nv = m.n_front_dofs < m.n_dofs ? 3 : 1;   // solve workspaces: one, plus two for the border columns
  info->device_bytes_fp64 = state + 8 * (nnz + (size_t)m.front_entries + nv * ((size_t)m.vec_entries + nd));
  info->device_bytes_mixed = state + 8 * nnz + 4 * (nnz + (size_t)m.front_entries + nv * ((size_t)m.vec_entries + nd)) +
                             (size_t)m.tc_img_chunks * TC_IMG_CHUNK_BYTES;
  info->n_colors = (int32_t)m.color_off.size() - 1;
  info->gemm_flops = m.gemm_flops;
  info->panel_flops = m.panel_flops;
  info->trsm_flops = m.trsm_flops;
  info->outer_flops = m.outer_flops;
  info->tc_split_chunks = m.tc_split_chunks;
  info->tc_tiles = m.tc_tiles;
  info->window_tc_flops = m.window_tc_flops;
  info->window_lu_flops = m.window_lu_flops;
  info->window_gemm_flops = m.window_gemm_flops;
  info->block_level_mask = 0;
  for (int l = 0; l < m.n_levels && l < 64; ++l)
    if (m.level_block.empty() || m.level_block[l]) info->block_level_mask |= (int64_t)1 << l;
  info->tc_image_bytes = (size_t)m.tc_img_chunks * TC_IMG_CHUNK_BYTES;
  info->dim = m.dim;
  info->elem_type = m.tri ? VIV_ELEM_TRI_P2P1 : VIV_ELEM_Q2;
  API_END
}

vivStatus viv_mesh_dof_labels(const vivMesh* mesh, int64_t* node, int32_t* field) {
  API_BEGIN
  VIV_CHECK(mesh, VIV_ERR_ARG, "NULL mesh");
  const Mesh& m = mesh->m;
  if (node) std::memcpy(node, m.dof_node.data(), m.n_dofs * sizeof(int64_t));
  if (field) std::memcpy(field, m.dof_field.data(), m.n_dofs * sizeof(int32_t));
  API_END
}

vivStatus viv_mesh_pattern(const vivMesh* mesh, int64_t* row_ptr, int32_t* col) {
  API_BEGIN
  VIV_CHECK(mesh, VIV_ERR_ARG, "NULL mesh");
  const Mesh& m = mesh->m;
  if (row_ptr) std::memcpy(row_ptr, m.row_ptr.data(), (m.n_dofs + 1) * sizeof(int64_t));
  if (col) std::memcpy(col, m.col.data(), m.col.size() * sizeof(int32_t));
  API_END
}

vivStatus viv_mesh_fronts(const vivMesh* mesh, int32_t* m_, int32_t* p_, int32_t* level, int32_t* parent) {
  API_BEGIN
  VIV_CHECK(mesh, VIV_ERR_ARG, "NULL mesh");
  const Mesh& m = mesh->m;
  const size_t nb = (size_t)m.n_fronts * sizeof(int32_t);
  if (m_) std::memcpy(m_, m.f_m.data(), nb);
  if (p_) std::memcpy(p_, m.f_p.data(), nb);
  if (level) std::memcpy(level, m.f_level.data(), nb);
  if (parent) std::memcpy(parent, m.f_parent.data(), nb);
  API_END
}

vivStatus viv_mesh_element_slots(const vivMesh* mesh, int32_t* elem_slots, int32_t* face_slots, int32_t* n_elem,
                                 int32_t* n_face) {
  API_BEGIN
  VIV_CHECK(mesh, VIV_ERR_ARG, "NULL mesh");
  const Mesh& m = mesh->m;
  if (n_elem) *n_elem = m.vol_pairs;
  if (n_face) *n_face = m.face_pairs;
  if (elem_slots) std::memcpy(elem_slots, m.e2nz.data(), m.e2nz.size() * sizeof(int32_t));
  if (face_slots) std::memcpy(face_slots, m.f2nz.data(), m.f2nz.size() * sizeof(int32_t));
  API_END
}

vivStatus viv_mesh_destroy(vivMesh* mesh) {
  API_BEGIN
  delete mesh;
  API_END
}

static vivStatus case_create_impl(vivMesh* mesh, const vivParams* prm, const double* u0, void* stream, vivCase** out,
                                  bool default_alloc);

// cases of the serving loop allocate with cudaMalloc (library-internal symbol)
__attribute__((visibility("hidden"))) vivStatus viv_internal_case_create(vivMesh* mesh, const vivParams* prm,
                                                                         const double* u0, void* s, vivCase** out) {
  return case_create_impl(mesh, prm, u0, s, out, true);
}

vivStatus viv_case_create(vivMesh* mesh, const vivParams* prm, const double* u0, void* stream, vivCase** out) {
  return case_create_impl(mesh, prm, u0, stream, out, false);
}

// Dimensionless inputs to the dimensional parameters the solver uses:
// Re = rho U_inf D / mu, and the reduced velocity of a massless cylinder
// U_r = pi U_inf sqrt(pi rho L / k) (Section 1) solved for k.
// The force-carrying length L defaults to the span of a periodic 3-D mesh, else 1.
static vivParams resolve_params(const vivParams& in, const Mesh& m) {
  vivParams p = in;
  const double L0 = m.dim == 3 && m.span > 0 ? m.span : 1.0;
  const double U = p.U_inf > 0 ? p.U_inf : 1.0, D = p.D > 0 ? p.D : 1.0, L = p.span_L > 0 ? p.span_L : L0;
  if (p.mu <= 0 && p.Re > 0) p.mu = p.rho * U * D / p.Re;
  if (p.k <= 0 && p.Ustar > 0) {
    const double pi = 3.14159265358979323846;
    p.k = pi * pi * pi * p.rho * L * U * U / (p.Ustar * p.Ustar);
  }
  return p;
}

static vivStatus case_create_impl(vivMesh* mesh, const vivParams* prm_in, const double* u0, void* stream,
                                  vivCase** out, bool default_alloc) {
  API_BEGIN
  VIV_CHECK(mesh && prm_in && u0 && out, VIV_ERR_ARG, "NULL argument");
  const vivParams resolved = resolve_params(*prm_in, mesh->m);
  const vivParams* prm = &resolved;
  VIV_CHECK(prm->dt > 0 && prm->rho > 0 && prm->mu > 0, VIV_ERR_ARG, "rho, mu (or Re) and dt must be positive");
  VIV_CHECK(prm->k >= 0, VIV_ERR_ARG, "spring stiffness k must not be negative");
  VIV_CHECK(prm->precision == VIV_FP64 || prm->precision == VIV_MIXED, VIV_ERR_ARG, "unknown precision");
  VIV_CHECK(prm->pivoting == VIV_PIVOT_THRESHOLD || prm->pivoting == VIV_PIVOT_WINDOW, VIV_ERR_ARG,
            "unknown pivoting");
  VIV_CHECK(prm->jacobian_fp32 == 0 || prm->jacobian_fp32 == 1, VIV_ERR_ARG, "jacobian_fp32 must be 0 or 1");
  VIV_CHECK(prm->predictor == 0 || prm->predictor == 1, VIV_ERR_ARG, "predictor must be 0 or 1");
  VIV_CHECK(prm->source >= 0 && prm->source <= 3, VIV_ERR_ARG, "source must be 0 .. 3");
  VIV_CHECK(prm->cfl_target >= 0 && prm->dt_max >= 0, VIV_ERR_ARG, "cfl_target and dt_max must not be negative");
  VIV_CHECK(mesh->m.on_device, VIV_ERR_STATE, "mesh was analysed on the host only");
  VIV_CHECK((mesh->m.dim == 2 && !mesh->m.tri) || (prm->source == 0 && prm->cfl_target == 0), VIV_ERR_ARG,
            "3-D and triangle meshes take no manufactured source and a constant step");
  *out = nullptr;
  vivCase* c = new vivCase();
  try {
    c->mesh = mesh;
    c->prm = *prm;
    if (c->prm.lame_scale == 0) c->prm.lame_scale = 1.0;
    if (c->prm.newton_tol <= 0) c->prm.newton_tol = 1e-10;
    if (c->prm.max_newton <= 0) c->prm.max_newton = 25;
    c->stream = (cudaStream_t)stream;
    c->dt_prev = c->prm.dt;
    c->arena.alloc = mesh->m.arena.alloc;
    c->arena.custom = mesh->m.arena.custom && !default_alloc;
    const Mesh& m = mesh->m;
    const int64_t n = m.n_nodes, nd = m.n_dofs, nnz = m.row_ptr[m.n_dofs], D = m.dim;
    DeviceArena& A = c->arena;
    CaseState& s = c->s;
    s.u = A.make<double>(D * n);
    s.p = A.make<double>(n);
    s.x = A.make<double>(D * n);
    s.lam = A.make<double>(D * n);
    s.delta = A.make<double>(2);
    s.u_n = A.make<double>(D * n);
    s.x_n = A.make<double>(D * n);
    s.u_nm1 = A.make<double>(D * n);
    s.x_nm1 = A.make<double>(D * n);
    s.hu = A.make<double>(D * n);
    s.hx = A.make<double>(D * n);
    s.lame = A.make<double>(m.n_elems);
    s.R = A.make<double>(nd);
    s.dU = A.make<double>(nd);
    s.r = A.make<double>(nd);
    s.d = A.make<double>(nd);
    s.mR = A.make<double>(nd);
    s.y2 = A.make<double>(nd);
    s.J64 = A.make<double>(nnz);
    s.J32 = mixed(c) ? A.make<float>(nnz) : nullptr;
    const size_t tsz = mixed(c) ? sizeof(float) : sizeof(double);
    s.fronts = A.get(tsz * (size_t)m.front_entries);
    s.vec = A.get(tsz * (size_t)m.vec_entries);
    s.yv = A.get(tsz * (size_t)nd);
    s.piv = A.make<int32_t>(m.piv_entries);
    s.perm = A.make<int32_t>(m.piv_entries);
    s.stats = A.make<int32_t>(4);
    s.chain = A.make<int32_t>(1 + (size_t)std::max(1, m.chain_flag_bound));
    if (has_border(m)) {
      s.Y = A.make<double>(2 * (size_t)nd);
      s.Bcol = A.make<double>(2 * (size_t)nd);
      const size_t tsz2 = mixed(c) ? sizeof(float) : sizeof(double);
      s.vec2 = A.get(2 * tsz2 * (size_t)m.vec_entries);
      s.yv2 = A.get(2 * tsz2 * (size_t)nd);
      s.Sb = A.make<double>(8);
      s.btmp = A.make<double>(4);
    }
    s.tc_img = mixed(c) && m.tc_img_chunks > 0
                   ? static_cast<unsigned char*>(A.get((size_t)m.tc_img_chunks * TC_IMG_CHUNK_BYTES))
                   : nullptr;
    s.partial = A.make<double>(296);
    s.scal = A.make<double>(8);
    s.step = A.make<double>(2);
    VIV_CUDA(cudaMallocHost(&c->h_pinned, 8 * sizeof(double)));
    cudaStream_t st = c->stream;
    VIV_CUDA(cudaMemcpyAsync(s.u, u0, D * n * sizeof(double), cudaMemcpyDefault, st));
    VIV_CUDA(cudaMemcpyAsync(s.x, m.d_X, D * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    VIV_CUDA(cudaMemsetAsync(s.p, 0, n * sizeof(double), st));
    VIV_CUDA(cudaMemsetAsync(s.lam, 0, D * n * sizeof(double), st));
    VIV_CUDA(cudaMemsetAsync(s.delta, 0, 2 * sizeof(double), st));
    VIV_CUDA(cudaMemsetAsync(s.u_nm1, 0, D * n * sizeof(double), st));
    VIV_CUDA(cudaMemsetAsync(s.x_nm1, 0, D * n * sizeof(double), st));
    VIV_CUDA(cudaMemsetAsync(s.stats, 0, 4 * sizeof(int32_t), st));
    if (mixed(c))
      prepare_kernels<float>();
    else
      prepare_kernels<double>();
    if (m.dim == 3) prepare_hex_kernels();
    noalloc_prepare();   // the allocation-free solve's fixed array is committed here, not on its first call
    launch_element_areas(m, s.lame, c->prm.lame_scale, c->prm.lame_constant != 0, s.scal + 1, st);
    if (c->prm.source == 3) launch_quasi_init(m, s, c->prm, st);   // the exact state at t = 0
    VIV_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    delete c;
    throw;
  }
  *out = c;
  API_END
}

vivStatus viv_case_destroy(vivCase* c) {
  API_BEGIN
  if (c) {
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    delete c;
  }
  API_END
}

vivStatus viv_set_state(vivCase* c, int, const double* u, const double* p, const double* x, const double* lam,
                        const double* delta, double t) {
  API_BEGIN
  VIV_CHECK(c, VIV_ERR_ARG, "NULL case");
  const int64_t n = c->mesh->m.n_nodes, D = c->mesh->m.dim;
  copy_in(c, c->s.u, u, D * n);
  copy_in(c, c->s.p, p, n);
  copy_in(c, c->s.x, x, D * n);
  if (x && c->mesh->m.tri) launch_midside_positions(c->mesh->m, c->s.x, c->stream);   // (P1 position)
  copy_in(c, c->s.lam, lam, D * n);
  copy_in(c, c->s.delta, delta, 2);
  c->t = t;
  VIV_CUDA(cudaStreamSynchronize(c->stream));
  API_END
}

vivStatus viv_set_history(vivCase* c, int, const double* u_prev, const double* x_prev) {
  API_BEGIN
  VIV_CHECK(c && u_prev && x_prev, VIV_ERR_ARG, "NULL argument");
  const int64_t n = c->mesh->m.n_nodes, D = c->mesh->m.dim;
  // begin_step moves u_n into u_nm1 when BDF2 is on
  copy_in(c, c->s.u_n, u_prev, D * n);
  copy_in(c, c->s.x_n, x_prev, D * n);
  if (c->mesh->m.tri) launch_midside_positions(c->mesh->m, c->s.x_n, c->stream);
  c->have_prev2 = true;
  VIV_CUDA(cudaStreamSynchronize(c->stream));
  API_END
}

vivStatus viv_get_state(const vivCase* cc, int, double* u, double* p, double* x, double* lam, double* delta,
                        double* t) {
  API_BEGIN
  VIV_CHECK(cc, VIV_ERR_ARG, "NULL case");
  vivCase* c = const_cast<vivCase*>(cc);
  const int64_t n = c->mesh->m.n_nodes, D = c->mesh->m.dim;
  copy_out(c, u, c->s.u, D * n);
  copy_out(c, p, c->s.p, n);
  copy_out(c, x, c->s.x, D * n);
  copy_out(c, lam, c->s.lam, D * n);
  copy_out(c, delta, c->s.delta, 2);
  if (t) *t = c->t;
  VIV_CUDA(cudaStreamSynchronize(c->stream));
  API_END
}

vivStatus viv_begin_step(vivCase* c) {
  API_BEGIN
  ProfBind pb_(c);
  VIV_CHECK(c, VIV_ERR_ARG, "NULL case");
  begin_step(c);
  API_END
}

vivStatus viv_assemble(vivCase* c, int what, double* res_norm) {
  API_BEGIN
  ProfBind pb_(c);
  VIV_CHECK(c && (what & (VIV_RES | VIV_JAC)), VIV_ERR_ARG, "bad arguments");
  double nr = assemble(c, what, res_norm != nullptr);
  if (res_norm) *res_norm = nr;
  API_END
}

vivStatus viv_get_residual(const vivCase* cc, double* r) {
  API_BEGIN
  VIV_CHECK(cc && r, VIV_ERR_ARG, "NULL argument");
  vivCase* c = const_cast<vivCase*>(cc);
  copy_out(c, r, c->s.R, c->mesh->m.n_dofs);
  VIV_CUDA(cudaStreamSynchronize(c->stream));
  API_END
}

vivStatus viv_get_jacobian(const vivCase* cc, double* vals) {
  API_BEGIN
  VIV_CHECK(cc && vals, VIV_ERR_ARG, "NULL argument");
  vivCase* c = const_cast<vivCase*>(cc);
  copy_out(c, vals, c->s.J64, c->mesh->m.row_ptr[c->mesh->m.n_dofs]);
  VIV_CUDA(cudaStreamSynchronize(c->stream));
  API_END
}

vivStatus viv_factor(vivCase* c) {
  API_BEGIN
  ProfBind pb_(c);
  VIV_CHECK(c, VIV_ERR_ARG, "NULL case");
  factor(c);
  API_END
}

vivStatus viv_border_block(const vivCase* cc, double* S) {
  API_BEGIN
  VIV_CHECK(cc && S, VIV_ERR_ARG, "NULL argument");
  vivCase* c = const_cast<vivCase*>(cc);
  VIV_CHECK(c->factored && has_border(c->mesh->m), VIV_ERR_STATE, "no factored border block");
  VIV_CUDA(cudaMemcpyAsync(S, c->s.Sb, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  VIV_CUDA(cudaStreamSynchronize(c->stream));
  API_END
}

vivStatus viv_solve(vivCase* c, int* sweeps) {
  API_BEGIN
  ProfBind pb_(c);
  VIV_CHECK(c, VIV_ERR_ARG, "NULL case");
  const int64_t n = c->mesh->m.n_dofs;
  launch_scale_copy(c->s.mR, c->s.R, -1.0, n, c->stream);
  int sw = refined_solve(c, c->s.mR, c->s.dU);
  c->have_dU = true;
  if (sweeps) *sweeps = sw;
  API_END
}

vivStatus viv_solve_rhs(vivCase* c, int, const double* b, double* y, int* sweeps) {
  API_BEGIN
  ProfBind pb_(c);
  VIV_CHECK(c && b && y, VIV_ERR_ARG, "NULL argument");
  const int64_t n = c->mesh->m.n_dofs;
  VIV_CUDA(cudaMemcpyAsync(c->s.mR, b, n * sizeof(double), cudaMemcpyDefault, c->stream));
  int sw = refined_solve(c, c->s.mR, c->s.y2);
  VIV_CUDA(cudaMemcpyAsync(y, c->s.y2, n * sizeof(double), cudaMemcpyDefault, c->stream));
  VIV_CUDA(cudaStreamSynchronize(c->stream));
  if (sweeps) *sweeps = sw;
  API_END
}

vivStatus viv_case_graphs(vivCase* c, int on) {
  API_BEGIN
  VIV_CHECK(c, VIV_ERR_ARG, "NULL case");
  c->graphs = on != 0;
  if (!c->graphs) drop_graphs(c);
  API_END
}

vivStatus viv_autotune(vivCase* c, int32_t* best_big_front, double* best_ms) {
  API_BEGIN
  ProfBind pb_(c);
  VIV_CHECK(c, VIV_ERR_ARG, "NULL case");
  Mesh& m = c->mesh->m;
  if (!c->step_open) begin_step(c);
  assemble(c, VIV_JAC, false);
  const int cands[] = {48, 64, 80, 96, 128, 192, 256, 384, 512, 768, 1024, 1 << 30};
  cudaEvent_t e0, e1;
  VIV_CUDA(cudaEventCreate(&e0));
  VIV_CUDA(cudaEventCreate(&e1));
  int best = m.big_front;
  double best_t = 1e300;
  for (int bf : cands) {
    build_schedule(m, bf);
    upload_work(m, c->stream);
    factor(c);   // warm-up
    VIV_CUDA(cudaEventRecord(e0, c->stream));
    for (int r = 0; r < 2; ++r) factor(c);
    VIV_CUDA(cudaEventRecord(e1, c->stream));
    VIV_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    VIV_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms / 2 < best_t) {
      best_t = ms / 2;
      best = bf;
    }
  }
  // per tree level (a front-size bucket) on the windowed FP32 schedule: the
  // block LU or the per-panel kernels for the level's large fronts, whichever
  // factors the level and runs its part of one solve faster (per-level CUDA
  // event timing; levels run one after the other, so their times add up)
  if (mixed(c) && c->prm.pivoting == VIV_PIVOT_WINDOW) {
    const bool prof_was_on = c->prof.on;
    auto level_times = [&](std::vector<double>& t) {
      build_schedule(m, best);
      upload_work(m, c->stream);
      factor(c);   // warm-up
      lu_solve(c, c->s.R, c->s.d);
      c->prof.used = 0;
      c->prof.on = true;
      factor(c);
      lu_solve(c, c->s.R, c->s.d);
      double ms[K_NKINDS];
      int64_t cnt[K_NKINDS];
      c->prof.read(ms, cnt);
      c->prof.on = false;
      t.assign(m.n_levels, 0.0);
      for (int l = 0; l < m.n_levels && (size_t)(l + 1) * K_NKINDS <= c->prof.level_ms.size(); ++l)
        for (int k = 0; k < K_NKINDS; ++k) t[l] += c->prof.level_ms[(size_t)l * K_NKINDS + k];
    };
    std::vector<double> t_on, t_off;
    m.level_block.assign(m.n_levels, 1);
    level_times(t_on);
    m.level_block.assign(m.n_levels, 0);
    level_times(t_off);
    for (int l = 0; l < m.n_levels; ++l) m.level_block[l] = t_on[l] <= t_off[l] ? 1 : 0;
    c->prof.on = prof_was_on;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  build_schedule(m, best);
  upload_work(m, c->stream);
  c->factored = false;
  if (best_big_front) *best_big_front = best;
  if (best_ms) *best_ms = best_t;
  API_END
}

vivStatus viv_set_big_front(vivCase* c, int32_t big_front) {
  API_BEGIN
  VIV_CHECK(c && big_front > 0, VIV_ERR_ARG, "viv_set_big_front: bad arguments");
  Mesh& m = c->mesh->m;
  if (m.big_front != big_front) {
    build_schedule(m, big_front);
    upload_work(m, c->stream);
    c->factored = false;
  }
  API_END
}

vivStatus viv_set_block_levels(vivCase* c, int64_t mask) {
  API_BEGIN
  VIV_CHECK(c, VIV_ERR_ARG, "viv_set_block_levels: NULL case");
  Mesh& m = c->mesh->m;
  std::vector<int8_t> want(m.n_levels);
  for (int l = 0; l < m.n_levels; ++l) want[l] = (l >= 64 ? mask < 0 : ((mask >> l) & 1)) ? 1 : 0;
  if (m.level_block != want) {
    m.level_block = want;
    build_schedule(m, m.big_front);
    upload_work(m, c->stream);
    c->factored = false;
  }
  API_END
}

vivStatus viv_lu_solve_noalloc(vivCase* c, const double* b, double* x) {
  API_BEGIN
  VIV_CHECK(c && b && x, VIV_ERR_ARG, "NULL argument");
  VIV_CHECK(c->factored, VIV_ERR_STATE, "viv_lu_solve_noalloc before viv_factor");
  lu_solve_noalloc(c, b, x);
  API_END
}

vivStatus viv_tc_schur_update(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int M, int N,
                              int K, int* err, void* stream) {
  API_BEGIN
  VIV_CHECK(A && B && C && err, VIV_ERR_ARG, "NULL argument");
  VIV_CHECK(M >= 0 && N >= 0 && K >= 0 && lda >= M && ldb >= K && ldc >= M, VIV_ERR_ARG, "bad GEMM shape");
  tc_gemm_update(A, lda, B, ldb, C, ldc, M, N, K, err, (cudaStream_t)stream);
  API_END
}

vivStatus viv_update(vivCase* c) {
  API_BEGIN
  ProfBind pb_(c);
  VIV_CHECK(c && c->have_dU, VIV_ERR_STATE, "update without a correction");
  launch_update(c->mesh->m, c->s, c->s.dU, c->stream);
  c->have_dU = false;
  API_END
}

// one Newton linear solve J dU = -R with FP64 refinement, through graphs:
// init (dU = 0, r = -R, ||R||) then sweeps (LU solve, dU += d, r = -R - J dU, ||r||).
// final = true: the closing correction of a converged mixed-path step: at
// least two sweeps, then until the linear residual is below 1e-6 of its
// right-hand side or stops falling (see step_impl)
// stale: the factors belong to an earlier Newton iterate (factor_reuse); the
// loop then also stops when a sweep contracts the residual by less than 1/2,
// and *converged says whether the tolerance was reached
static int refined_solve_graphs(vivCase* c, bool final = false, bool stale = false, bool* converged = nullptr) {
  const Mesh& m = c->mesh->m;
  CaseState& s = c->s;
  const int64_t n = m.n_dofs;
  const int max_sweeps =
      final ? 20 : 1 + (c->prm.refine_max > 0 ? c->prm.refine_max : (mixed(c) ? 10 : 1));
  // Newton needs the correction only as accurately as the step can use it: stop
  // when the linear residual is below refine_tol relative (default 1e-8), or
  // below a tenth of the Newton tolerance in absolute terms, whichever is looser
  const double tol = final ? 1e-6 : (c->prm.refine_tol > 0 ? c->prm.refine_tol : 1e-8);
  const double abs_tol = final ? 0.0 : 0.1 * c->prm.newton_tol;
  run_graph(c, c->g_sinit, [&] {
    launch_scale_copy(s.mR, s.R, -1.0, n, c->stream);
    VIV_CUDA(cudaMemsetAsync(s.dU, 0, n * sizeof(double), c->stream));
    VIV_CUDA(cudaMemcpyAsync(s.r, s.mR, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    launch_norm2(s.mR, n, s.partial, s.scal + 2, c->stream);
  });
  const double nb = read_scalar(c, s.scal + 2);
  int sweeps = 0;
  double prev = nb;
  for (;;) {
    run_graph(c, c->g_sweep, [&] {
      lu_solve(c, s.r, s.d);
      launch_axpy(s.dU, s.d, 1.0, n, c->stream);
      launch_spmv_residual(m, s.J64, s.dU, s.mR, s.r, c->stream);
      launch_norm2(s.r, n, s.partial, s.scal + 3, c->stream);
    });
    ++sweeps;
    const double nr = read_scalar(c, s.scal + 3);
    if (stale && !std::isfinite(nr)) {   // a stale preconditioner diverged: refactor
      if (converged) *converged = false;
      return sweeps;
    }
    VIV_CHECK(std::isfinite(nr), VIV_ERR_NONFINITE, "refinement residual is not finite");
    const bool done = nb == 0 || nr <= std::max(tol * nb, abs_tol);
    if (converged) *converged = done || final;
    if (sweeps >= max_sweeps || nb == 0) break;
    if (final && sweeps < 2) continue;   // (see step_impl)
    if (done) break;
    if (final && nr > 0.5 * prev) break;   // at the FP64 floor: further sweeps only add rounding
    if (stale && nr > 0.5 * prev) break;   // the stale factors no longer precondition well
    prev = nr;
  }
  return sweeps;
}

static void step_impl(vivCase* c, vivStepInfo* info) {
  const Mesh& m = c->mesh->m;
  begin_step(c);
  const double tol = c->prm.newton_tol;
  int iters = 0, sweeps = 0, reused = 0;
  double n0 = 0, nr = 0;
  int32_t st_acc[2] = {0, 0};
  bool polished = false;
  for (int it = 0;; ++it) {
    {
      auto res = [&] {
        launch_residual(m, c->s, c->prm, c->stream);
        launch_norm2(c->s.R, m.n_dofs, c->s.partial, c->s.scal, c->stream);
      };
      if (it == 0)
        run_graph(c, c->g_res, res);
      else
        run_graph(c, c->g_upd_res, [&] {
          launch_update(m, c->s, c->s.dU, c->stream);
          res();
        });
      nr = read_scalar(c, c->s.scal);
    }
    if (it == 0) n0 = nr;
    VIV_CHECK(std::isfinite(nr), VIV_ERR_NONFINITE, "residual norm is not finite");
    if (nr <= tol) {
      // Closing correction, with the factors at hand (no new Jacobian), on
      // both paths: a state that only just passed the test can be ~1e-8 off
      // the discrete solution in the pressure (all-Dirichlet problems), and the
      // correction takes it to round-off.  With FP32 volume Jacobians Newton converges linearly
      // (contraction ~1e-4 here) and stops just under the tolerance; and on
      // every mixed path the FP32 factors leave errors in directions the
      // residual barely sees - at 38,800 quads a near-constant pressure offset
      // of ~6e-12 (1.8e-9 of the pressure field) that moves ||NL|| by less than
      // its FP64 floor (~4e-14).  Refinement sweeps shrink that error even
      // after the linear residual is at the floor: measured there, one sweep
      // leaves the 1.8e-9, two bring the pressure to 3e-11..9e-11 of the FP64
      // path's, and more sweeps change nothing beyond that noise.  Hence at
      // least two sweeps, then to 1e-6 of the right-hand side.
      if (it > 0 && !polished) {
        polished = true;
        sweeps += refined_solve_graphs(c, true);
        continue;   // the next pass applies the correction and re-evaluates ||NL||
      }
      break;
    }
    VIV_CHECK(it < c->prm.max_newton, VIV_ERR_NEWTON,
              "Newton did not converge in " + std::to_string(c->prm.max_newton) + " iterations (|R| = " +
                  fmt_e(nr) + ", tolerance " + fmt_e(tol) + ")");
    run_graph(c, c->g_jac, [&] { jacobian(c); });
    bool solved = false;
    if (c->prm.factor_reuse && mixed(c) && it > 0 && c->factored) {
      // the factors of this step's first iterate precondition the refined solve
      // with the current Jacobian; refactor if refinement stalls
      sweeps += refined_solve_graphs(c, false, true, &solved);
      reused += solved ? 1 : 0;
    }
    if (!solved) {
      run_graph(c, c->g_fac, [&] { factor(c); });
      c->factored = true;
      sweeps += refined_solve_graphs(c);
      ++iters;
    }
    int32_t stv[4];
    VIV_CUDA(cudaMemcpyAsync(stv, c->s.stats, sizeof(stv), cudaMemcpyDeviceToHost, c->stream));
    VIV_CUDA(cudaStreamSynchronize(c->stream));
    VIV_CHECK(stv[2] == 0, VIV_ERR_TIMEOUT, "a bounded device wait expired (tensor-core pipeline or solve chain)");
    VIV_CHECK(stv[3] == 0, VIV_ERR_PIVOT, "the border Schur block of the cylinder position is singular");
    st_acc[0] += stv[0];
    st_acc[1] += stv[1];
  }
  // the loop ends on a converged residual of the updated state
  const double dt_used = c->prm.dt;
  c->t += dt_used;
  c->nstep += 1;
  c->step_open = false;
  c->dt_prev = dt_used;
  double cfl = 0;
  if (c->prm.cfl_target > 0) {
    // Section 6: the next step size from the Courant number of the new state
    // (target CFL as a convection error estimator), within a factor 1/2 .. 1.2
    // of the last (step ratio below 1 + sqrt 2: zero-stable BDF2) and dt_max
    cfl = launch_cfl(m, c->s, dt_used, c->s.partial, c->s.scal + 5, c->h_pinned + 5, c->stream);
    const double r = cfl > 0 ? c->prm.cfl_target / cfl : 1.2;
    double next = dt_used * std::min(1.2, std::max(0.5, r));
    if (c->prm.dt_max > 0) next = std::min(next, c->prm.dt_max);
    c->prm.dt = next;
  }
  if (info) {
    info->dt = dt_used;
    info->cfl = cfl;
    info->newton_iters = iters;
    info->reused_factor_solves = reused;
    info->refine_sweeps = sweeps;
    info->perturbed_pivots = st_acc[0];
    info->threshold_misses = st_acc[1];
    info->res_norm0 = n0;
    info->res_norm = nr;
    info->t = c->t;
    double d[2] = {0, 0}, rd[2] = {0, 0};
    VIV_CUDA(cudaMemcpyAsync(d, c->s.delta, sizeof(d), cudaMemcpyDeviceToHost, c->stream));
    if (m.delta_dof[0] >= 0)
      VIV_CUDA(cudaMemcpyAsync(rd, c->s.R + m.delta_dof[0], sizeof(rd), cudaMemcpyDeviceToHost, c->stream));
    VIV_CUDA(cudaStreamSynchronize(c->stream));
    info->delta[0] = d[0];
    info->delta[1] = d[1];
    // R[delta] = k delta + int lambda, so F_fluid = -int lambda = k delta - R[delta]
    info->force[0] = c->prm.k * d[0] - rd[0];
    info->force[1] = c->prm.k * d[1] - rd[1];
  }
}

vivStatus viv_step(vivCase* c, vivStepInfo* info) {
  API_BEGIN
  ProfBind pb_(c);
  VIV_CHECK(c, VIV_ERR_ARG, "NULL case");
  step_impl(c, info);
  API_END
}

vivStatus viv_case_params(const vivCase* c, vivParams* out) {
  API_BEGIN
  VIV_CHECK(c && out, VIV_ERR_ARG, "NULL argument");
  *out = c->prm;
  API_END
}

// Checkpoint layout (host bytes, native endianness):
//   char magic[8] = "VIVCKPT2"; int64 n_nodes, n_dofs; int32 precision, bdf2_ready;
//   double t, dt, dt_prev; int64 nstep;
//   double u[2n], p[n], x[2n], lam[2n], delta[2], u_n[2n], x_n[2n]
// u..delta is the current state (the last converged step), u_n and x_n the
// previous time level, which the next BDF2 step needs.
namespace {
constexpr char CKPT_MAGIC[8] = {'V', 'I', 'V', 'C', 'K', 'P', 'T', '2'};
constexpr size_t CKPT_HEADER = 8 + 2 * 8 + 2 * 4 + 3 * 8 + 8;
// u, x, lam, u_n, x_n (D n each), p (n), delta (2)
size_t ckpt_bytes(int64_t n, int64_t D) { return CKPT_HEADER + sizeof(double) * (size_t)(5 * D * n + n + 2); }
}  // namespace

vivStatus viv_case_save(const vivCase* cc, void* buf, size_t* bytes) {
  API_BEGIN
  VIV_CHECK(cc && bytes, VIV_ERR_ARG, "NULL argument");
  VIV_CHECK(!cc->step_open, VIV_ERR_STATE, "viv_case_save inside an open time step");
  vivCase* c = const_cast<vivCase*>(cc);
  const int64_t n = c->mesh->m.n_nodes, D = c->mesh->m.dim;
  const size_t need = ckpt_bytes(n, D);
  if (!buf) {
    *bytes = need;
    return VIV_OK;
  }
  VIV_CHECK(*bytes >= need, VIV_ERR_ARG, "checkpoint buffer too small: need " + std::to_string(need) + " bytes");
  unsigned char* b = static_cast<unsigned char*>(buf);
  auto put = [&](const void* v, size_t k) {
    std::memcpy(b, v, k);
    b += k;
  };
  const int64_t nd = c->mesh->m.n_dofs, ns = c->nstep;
  const int32_t prec = c->prm.precision, ready = (c->nstep > 0 || c->have_prev2) ? 1 : 0;
  put(CKPT_MAGIC, 8);
  put(&n, 8);
  put(&nd, 8);
  put(&prec, 4);
  put(&ready, 4);
  put(&c->t, 8);
  put(&c->prm.dt, 8);
  put(&c->dt_prev, 8);
  put(&ns, 8);
  double* d = reinterpret_cast<double*>(b);   // copies go through unified addressing (any alignment)
  const CaseState& s = c->s;
  copy_out(c, d, s.u, D * n);
  copy_out(c, d + D * n, s.p, n);
  copy_out(c, d + D * n + n, s.x, D * n);
  copy_out(c, d + 2 * D * n + n, s.lam, D * n);
  copy_out(c, d + 3 * D * n + n, s.delta, 2);
  copy_out(c, d + 3 * D * n + n + 2, s.u_n, D * n);
  copy_out(c, d + 4 * D * n + n + 2, s.x_n, D * n);
  VIV_CUDA(cudaStreamSynchronize(c->stream));
  *bytes = need;
  API_END
}

vivStatus viv_case_load(vivCase* c, const void* buf, size_t bytes) {
  API_BEGIN
  VIV_CHECK(c && buf, VIV_ERR_ARG, "NULL argument");
  const int64_t n = c->mesh->m.n_nodes, D = c->mesh->m.dim;
  VIV_CHECK(bytes >= CKPT_HEADER && std::memcmp(buf, CKPT_MAGIC, 8) == 0, VIV_ERR_ARG, "not a case checkpoint");
  const unsigned char* b = static_cast<const unsigned char*>(buf) + 8;
  auto get = [&](void* v, size_t k) {
    std::memcpy(v, b, k);
    b += k;
  };
  int64_t n_s = 0, nd_s = 0, ns = 0;
  int32_t prec = 0, ready = 0;
  double t = 0, dt = 0, dt_prev = 0;
  get(&n_s, 8);
  get(&nd_s, 8);
  get(&prec, 4);
  get(&ready, 4);
  get(&t, 8);
  get(&dt, 8);
  get(&dt_prev, 8);
  get(&ns, 8);
  VIV_CHECK(n_s == n && nd_s == c->mesh->m.n_dofs && bytes >= ckpt_bytes(n, D), VIV_ERR_ARG,
            "checkpoint was written for another mesh");
  // a constant-step case must resume with its own dt; an adaptive one resumes
  // with the saved step sizes
  VIV_CHECK(c->prm.cfl_target > 0 || dt == c->prm.dt, VIV_ERR_ARG, "checkpoint time step differs from the case's dt");
  const double* d = reinterpret_cast<const double*>(b);
  CaseState& s = c->s;
  copy_in(c, s.u, d, D * n);
  copy_in(c, s.p, d + D * n, n);
  copy_in(c, s.x, d + D * n + n, D * n);
  copy_in(c, s.lam, d + 2 * D * n + n, D * n);
  copy_in(c, s.delta, d + 3 * D * n + n, 2);
  copy_in(c, s.u_n, d + 3 * D * n + n + 2, D * n);
  copy_in(c, s.x_n, d + 4 * D * n + n + 2, D * n);
  VIV_CUDA(cudaStreamSynchronize(c->stream));
  c->t = t;
  c->prm.dt = dt;
  c->dt_prev = dt_prev;
  c->nstep = (int)ns;
  c->have_prev2 = ready != 0;
  c->step_open = false;
  c->factored = false;
  c->have_dU = false;
  API_END
}

int64_t viv_state_size(const vivMesh* mesh) {
  if (!mesh) return -1;
  const int64_t n = mesh->m.n_nodes, D = mesh->m.dim;
  return 5 * D * n + n + 2 + 2;
}

// packed host state: u(Dn) p(n) x(Dn) lam(Dn) delta(2) u_prev(Dn) x_prev(Dn) [t, have_prev]
vivStatus viv_step_host(vivCase* c, const double* in, double* out, vivStepInfo* info) {
  API_BEGIN
  ProfBind pb_(c);
  VIV_CHECK(c && in && out, VIV_ERR_ARG, "NULL argument");
  const int64_t n = c->mesh->m.n_nodes, D = c->mesh->m.dim;
  const double* q = in;
  copy_in(c, c->s.u, q, D * n);
  q += D * n;
  copy_in(c, c->s.p, q, n);
  q += n;
  copy_in(c, c->s.x, q, D * n);
  if (c->mesh->m.tri) launch_midside_positions(c->mesh->m, c->s.x, c->stream);
  q += D * n;
  copy_in(c, c->s.lam, q, D * n);
  q += D * n;
  copy_in(c, c->s.delta, q, 2);
  q += 2;
  const double* up = q;
  q += D * n;
  const double* xp = q;
  q += D * n;
  c->t = q[0];
  const bool have_prev = q[1] != 0.0;
  c->nstep = 0;
  c->have_prev2 = have_prev;
  if (have_prev) {
    copy_in(c, c->s.u_n, up, D * n);
    copy_in(c, c->s.x_n, xp, D * n);
    if (c->mesh->m.tri) launch_midside_positions(c->mesh->m, c->s.x_n, c->stream);
  }
  step_impl(c, info);
  double* o = out;
  copy_out(c, o, c->s.u, D * n);
  o += D * n;
  copy_out(c, o, c->s.p, n);
  o += n;
  copy_out(c, o, c->s.x, D * n);
  o += D * n;
  copy_out(c, o, c->s.lam, D * n);
  o += D * n;
  copy_out(c, o, c->s.delta, 2);
  o += 2;
  copy_out(c, o, c->s.u_n, D * n);
  o += D * n;
  copy_out(c, o, c->s.x_n, D * n);
  o += D * n;
  VIV_CUDA(cudaStreamSynchronize(c->stream));
  o[0] = c->t;
  o[1] = 1.0;
  API_END
}

}  // extern "C"
