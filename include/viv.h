/*
 * viv.h - C ABI of the B300 monolithic ALE solver for a massless,
 * spring-mounted cylinder (vortex-induced vibrations at zero mass ratio).
 *
 * One implicit system per Newton step holds the fluid velocity u and
 * pressure p on the moving mesh, the mesh position x (linear-elastic
 * pseudo-solid on the reference mesh), the Lagrange multiplier lambda on the
 * cylinder boundary Gamma, and the cylinder displacement delta
 * (Section 2, Eq. system; Section 3.1, Eq. weak_system; Eq. lambda_coupling).
 * Discretisation: Q2 velocity / Q1 pressure / Q2 position on 9-node quads,
 * Q2 multiplier traces on Gamma, BDF2 in time with a BDF1 first step.
 *
 * Conventions
 *  - Every function returns vivStatus and never aborts; on failure
 *    viv_last_error() returns a thread-local message.
 *  - Host pointers are read during the call only; the library copies what it
 *    keeps.  Output host buffers are caller-allocated.
 *  - Handles are owned by the caller and released by the matching *_destroy.
 *  - `stream` arguments are cudaStream_t values passed as void*; NULL means the
 *    legacy default stream.  All device work of a case is ordered on its
 *    stream.  A case is not thread-safe; distinct cases may run concurrently.
 *  - Device memory comes from the allocator given at mesh creation (or
 *    cudaMalloc when NULL); a failed allocation returns VIV_ERR_OOM.
 *  - No device code waits on a flag; there is no unbounded device wait.
 */
#ifndef VIV_H
#define VIV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VIV_OK = 0,
  VIV_ERR_ARG = 1,             /* bad argument or inconsistent mesh */
  VIV_ERR_OOM = 2,             /* device allocation failed */
  VIV_ERR_CUDA = 3,            /* a CUDA runtime call failed */
  VIV_ERR_PIVOT = 4,           /* a front met an exactly zero pivot column */
  VIV_ERR_NEWTON = 5,          /* Newton did not reach the tolerance in max_newton */
  VIV_ERR_NONFINITE = 6,       /* a residual or correction norm is NaN/Inf */
  VIV_ERR_TIMEOUT = 7,         /* a bounded device wait expired (tensor-core mbarrier, or a
                                  multi-CTA solve chain's release flag) */
  VIV_ERR_ADMISSION = 8,       /* server: request exceeds the memory budget */
  VIV_ERR_STATE = 9            /* call out of order (e.g. solve before factor) */
} vivStatus;

/* node tag bits (per mesh node): which nodal values a Dirichlet condition holds */
enum {
  VIV_TAG_U_FIX_X = 1, VIV_TAG_U_FIX_Y = 2,   /* velocity component held (Eq. flowBC) */
  VIV_TAG_X_FIX_X = 4, VIV_TAG_X_FIX_Y = 8,   /* position component held (Eq. psBC) */
  VIV_TAG_CYL = 16,                            /* node on Gamma: x = X + delta, lambda lives here */
  VIV_TAG_OUTLET = 32,                         /* informational */
  VIV_TAG_P_FIX = 64,                          /* pressure held (all-Dirichlet problems) */
  VIV_TAG_U_FIX_Z = 128,                       /* 3-D: velocity z-component held */
  VIV_TAG_X_FIX_Z = 256                        /* 3-D: position z-component held */
};

/* precision of the factors (and of the Jacobian; see jacobian_fp32); residual,
 * refinement, state: FP64 always */
enum { VIV_FP64 = 0, VIV_MIXED = 1 };
/* what viv_assemble builds */
enum { VIV_RES = 1, VIV_JAC = 2 };
/* field codes of viv_mesh_dof_labels */
enum { VIV_F_UX = 0, VIV_F_UY = 1, VIV_F_XX = 2, VIV_F_XY = 3, VIV_F_P = 4,
       VIV_F_LX = 5, VIV_F_LY = 6, VIV_F_DX = 7, VIV_F_DY = 8,
       VIV_F_UZ = 9, VIV_F_XZ = 10, VIV_F_LZ = 11 };   /* z codes: 3-D meshes only */

typedef struct {
  void* (*alloc)(size_t bytes, void* ctx);   /* returns device memory or NULL */
  void (*free)(void* ptr, void* ctx);
  void* ctx;
} vivAllocator;

typedef struct vivMesh vivMesh;
typedef struct vivCase vivCase;

/* Mesh description.  dim 0 or 2: two dimensions; 3: three.
 * 2-D: X: n_nodes x 2 reference coordinates (row-major).  conn: n_elems x 9
 * node ids of each Q2 quad, lexicographic (node 3*b + a, a along xi),
 * positively oriented.  gamma_faces: n_gamma_faces x 2 (element, local edge)
 * pairs of Gamma, edges 0: xi=0 (nodes 0,3,6), 1: xi=1 (2,5,8), 2: eta=0
 * (0,1,2), 3: eta=1 (6,7,8).
 * 3-D: X: n_nodes x 3.  conn: n_elems x 27 node ids of each Q2 hexahedron
 * (node 9*c + 3*b + a, c along zeta), positively oriented; gamma_faces:
 * (element, local face) with faces 0/1: xi = 0/1, 2/3: eta = 0/1,
 * 4/5: zeta = 0/1.  span > 0 makes the mesh periodic in z with that period:
 * bit a of wrap[e] (n_elems entries, or NULL for none) says that local node a
 * of element e sits at its stored coordinates + span e_z (the element crosses
 * the seam); the periodicity is on the displacement x - X.  Gamma nodes move
 * by (delta_x, delta_y, 0): their z position must be held (VIV_TAG_X_FIX_Z);
 * the multiplier has three components there.
 * elem_type VIV_ELEM_TRI_P2P1 (2-D only): the paper's own spaces (Section 3.3),
 * P2 velocity on 6-node triangles, P1 pressure and P1 mesh position on the
 * vertices, P2 multiplier traces: conn n_elems x 6 (vertices 0, 1, 2
 * counter-clockwise, then the midpoints of edges 0-1, 1-2, 2-0), gamma_faces
 * (element, local edge e = (v_e, midpoint, v_{e+1})); every midside node must
 * sit at the midpoint of its edge (straight edges; VIV_ERR_ARG otherwise).  A
 * midside node carries no position unknown: its position is the mean of the
 * edge's end vertices, which the library keeps in the nodal x array (and
 * restores from the vertices in positions the caller passes in, off Gamma).
 * Every element must be positively oriented (its corner edge vectors at local
 * node 0 span a positive area or volume; VIV_ERR_ARG otherwise).
 * tags: n_nodes VIV_TAG_* bit sets.  leaf_elems: nested-dissection leaf size
 * in elements (0: default, 4 in 2-D, 2 in 3-D, 8 for triangles). */
enum { VIV_ELEM_Q2 = 0, VIV_ELEM_TRI_P2P1 = 1 };
typedef struct {
  int64_t n_nodes, n_elems, n_gamma_faces;
  const double* X;
  const int64_t* conn;
  const int32_t* tags;
  const int64_t* gamma_faces;
  int32_t leaf_elems;
  int32_t dim;
  double span;
  const int64_t* wrap;
  int32_t elem_type;
} vivMeshDesc;

typedef struct {
  int64_t n_dofs;          /* unknowns: free u, p, x, lambda, and delta (2) */
  int64_t nnz;             /* structural nonzeros of the Jacobian (CSR) */
  int64_t n_fronts;        /* supernodes of the nested-dissection tree */
  int64_t max_front;       /* largest front order */
  int64_t n_levels;        /* tree height + 1 */
  double factor_flops;     /* flops of one numeric factorisation */
  size_t front_entries;    /* sum of front order^2 (factor storage in entries) */
  size_t device_bytes_fp64;   /* predicted device bytes of one FP64 case */
  size_t device_bytes_mixed;  /* predicted device bytes of one mixed case */
  int32_t n_colors;        /* element colours of the deterministic scatter */
  double gemm_flops;       /* Schur-update (GEMM) flops of one factorisation */
  double panel_flops;      /* in-panel LU flops of one factorisation */
  double trsm_flops;       /* panel TRSM flops of one factorisation */
  double outer_flops;      /* part of gemm_flops in K = 128 outer updates (tensor cores, mixed path) */
  int64_t tc_split_chunks; /* mixed path, per factorisation: 128 x 32 operand chunks split into hi/lo
                              TF32 images (16 KB read, 32 KB written each) */
  int64_t tc_tiles;        /* mixed path, per factorisation: 128 x 128 tiles of the outer updates */
  size_t tc_image_bytes;   /* the operand-image buffer a mixed case holds (in device_bytes_mixed) */
  /* mixed path with windowed pivoting, per factorisation (the counters above
   * describe the threshold-pivoting schedule): */
  double window_tc_flops;  /* tensor-core flops: L21, U12 and Schur updates of the 128-column blocks */
  double window_lu_flops;  /* LU flops of the pivot blocks (windows and block LU incl. the block inverses) */
  double window_gemm_flops;/* SIMT Schur-update flops (fronts below the large-front order) */
  int64_t block_level_mask;/* tree levels (bit l) whose large fronts may use the block LU */
  int32_t dim;             /* 2 or 3: components of u, x and lambda per node */
  int32_t elem_type;       /* VIV_ELEM_Q2 or VIV_ELEM_TRI_P2P1 */
} vivMeshInfo;

/* Physical and solver parameters.  rho, mu: fluid density and viscosity;
 * k: spring stiffness of Eq. solid_balance (mu and k may instead come from Re
 * and Ustar, see the last fields); dt: constant time step;
 * lame_scale: lambda_s = mu_s = lame_scale * min|K_0| / |K_0| per element
 *   (reference areas; 0 means 1);
 * newton_tol: absolute ||NL||_2 stop; refine_tol: relative residual at which
 * the refinement of a Newton correction stops (0: 1e-8; it also stops once the
 * residual is below newton_tol / 10); refine_max: refinement sweeps (0: 10 on
 * the mixed path, 1 on the FP64 path).  viv_solve_rhs refines to 1e-13. */
typedef struct {
  double rho, mu, k, dt;
  double lame_scale;
  double newton_tol;
  int32_t max_newton;
  int32_t precision;       /* VIV_FP64 or VIV_MIXED */
  double refine_tol;
  int32_t refine_max;
  double pivot_threshold;  /* threshold u of partial pivoting in fronts (0.01) */
  int32_t source;          /* 0: none (the physical problem); 1: steady manufactured
                              solution of Section 5.1 on a mesh deformed by
                              X + source_amp sin(pi X) sin(pi Y) (1, 1); 2: Section 5.1's
                              time-dependent solution (u = t^3 (sin pi x cos pi y,
                              sin pi x sin pi y), p = t^2 cos pi x cos pi y) on a mesh moved by
                              X + source_amp sin(pi t) sin(pi X) sin(pi Y) (1, 1), whose
                              Dirichlet data the library sets at each step's time; 3: the
                              coupled quasi-manufactured solution of Section 5.2 on the
                              unit square around a cylinder of radius 0.15 at (1/2, 1/2)
                              (kernel radius 0.45, total displacement source_amp (0.8, 0.6),
                              f(t) = sin 2 pi t, pressure -k f psi (e.d) / (0.15 pi)), for
                              which viv_case_create sets the exact initial velocity and
                              which needs no Dirichlet update (source_amp <= 0.05); sources
                              of 1 .. 3 assume lambda_s = mu_s = 1 (lame_constant = 1);
                              for verification */
  double source_amp;
  int32_t pivoting;        /* VIV_PIVOT_THRESHOLD (0): threshold partial pivoting over all
                              fully summed rows of a front; VIV_PIVOT_WINDOW (1): partial
                              pivoting inside each 32 x 32 diagonal block only (faster
                              panels; the refinement recovers the accuracy) */
  int32_t jacobian_fp32;   /* mixed path only: 1 evaluates the volume element Jacobians in
                              FP32 arithmetic (Gamma-face and border rows, the residual, the
                              Newton test and the refinement products stay FP64); 0 (default)
                              evaluates every Jacobian entry in FP64 */
  int32_t predictor;       /* Newton starting point of a BDF2 step: 0 (default) the previous
                              time level U^n; 1 the linear extrapolation 2 U^n - U^{n-1} of
                              velocity and position (and so of delta); p and lambda start
                              from U^n either way.  The converged state does not depend on it
                              beyond the Newton tolerance. */
  /* Dimensionless inputs, converted by viv_case_create (and by the server at
   * admission) when the corresponding dimensional value is not given:
   *   mu <= 0 and Re > 0:    mu = rho U_inf D / Re;
   *   k <= 0 and Ustar > 0:  k = pi^3 rho L U_inf^2 / Ustar^2, the stiffness at
   *                          which the reduced velocity of a massless cylinder,
   *                          U_r = pi U_inf sqrt(pi rho L / k) (Section 1), equals
   *                          Ustar; L = span_L, the length that carries the force
   *                          (1 for a 2-D section).
   * U_inf and D default to 1 when 0; span_L defaults to the span of a periodic
   * 3-D mesh, else 1.  k = 0 with Ustar = 0 is a problem
   * without a cylinder (no border unknowns). */
  double Re, Ustar, U_inf, D, span_L;
  /* Adaptive time stepping (Section 6: a target Courant number as a simple
   * convection error estimator).  cfl_target > 0: after every step the library
   * computes CFL = dt max_e (max_a |u_a| / h_e) (largest nodal velocity of an
   * element over its shortest corner-to-corner edge, current configuration)
   * and sets the next step to dt cfl_target / CFL, kept within [dt / 2, 1.2 dt]
   * (a step ratio below 1 + sqrt 2 keeps variable-step BDF2 zero-stable) and
   * at most dt_max (when > 0).  BDF2 then uses the step ratio w = dt / dt_prev:
   * rates [(1 + 2w)/(1 + w) v^{n+1} - (1 + w) v^n + w^2/(1 + w) v^{n-1}] / dt.
   * cfl_target = 0 (default): constant dt. */
  double cfl_target, dt_max;
  int32_t lame_constant;   /* 1: lambda_s = mu_s = lame_scale on every element (the
                              manufactured solutions); 0 (default): lame_scale min|K_0|/|K_0| */
  int32_t factor_reuse;    /* mixed path: 0 (default, as in Section 6) factors the Jacobian at
                              every Newton iteration; 1 factors it at a step's first iteration
                              only: later iterations assemble their Jacobian and solve with it by
                              FP64 iterative refinement preconditioned with the factors at hand,
                              refactoring when refinement stalls (contraction worse than 1/2, or
                              not converged within the sweep limit).  The Newton correction is the
                              same to the refinement tolerance; fewer factorisations, more sweeps. */
} vivParams;
enum { VIV_PIVOT_THRESHOLD = 0, VIV_PIVOT_WINDOW = 1 };

typedef struct {
  int32_t newton_iters;    /* Jacobian factorisations this step */
  int32_t refine_sweeps;   /* refinement sweeps summed over the step */
  int32_t perturbed_pivots;/* pivots replaced by a static perturbation */
  int32_t threshold_misses;/* pivots taken below the threshold */
  double res_norm0, res_norm; /* ||NL|| at the predictor and at convergence */
  double t;                /* time reached */
  double delta[2];         /* cylinder displacement x_c - X_c */
  double force[2];         /* F_fluid = -int_Gamma lambda */
  double dt;               /* size of this step */
  double cfl;              /* Courant number of the new state (0 unless cfl_target > 0) */
  int32_t reused_factor_solves; /* Newton iterations solved with reused factors (factor_reuse) */
} vivStepInfo;

/* ---- mesh: numbering, sparsity, nested dissection, symbolic factorisation
 * (Section 6: the pattern is fixed because ALE moves nodes, not
 * connectivity, so analysis runs once per mesh) --------------------------- */
vivStatus viv_mesh_create(const vivMeshDesc* desc, const vivAllocator* alloc, void* stream,
                          vivMesh** out);
/* Host-only analysis of the same mesh (no device memory, no CUDA call):
 * numbering, pattern and symbolic factorisation.  The handle answers
 * viv_mesh_info, viv_mesh_dof_labels and viv_mesh_pattern; viv_case_create
 * on it returns VIV_ERR_STATE. */
vivStatus viv_mesh_analyze(const vivMeshDesc* desc, vivMesh** out);
vivStatus viv_mesh_info(const vivMesh* mesh, vivMeshInfo* info);
/* per unknown: owning node (n_nodes for delta) and VIV_F_* field code */
vivStatus viv_mesh_dof_labels(const vivMesh* mesh, int64_t* node, int32_t* field);
/* CSR pattern of the Jacobian: row_ptr (n_dofs+1), col (nnz), host buffers */
vivStatus viv_mesh_pattern(const vivMesh* mesh, int64_t* row_ptr, int32_t* col);
/* per front (supernode, in elimination order): order m, pivots p, tree level
 * (0 = leaves) and parent (-1 for the root); host buffers of n_fronts */
vivStatus viv_mesh_fronts(const vivMesh* mesh, int32_t* m, int32_t* p, int32_t* level, int32_t* parent);
/* The element-to-nonzero maps the element kernels scatter through, for callers
 * that add element contributions of their own to the Jacobian's CSR values:
 * per element, the CSR value index (or -1: the row or column is not an
 * unknown) of every structural pair of its local matrix, in the family's
 * fixed pair order (momentum rows against every column, continuity rows
 * against the velocity and position columns, pseudo-solid rows against the
 * position columns; Gamma position columns are the delta columns); per Gamma
 * edge or face, the same for its multiplier and border couplings.  *n_elem and
 * *n_face receive the entries per element and per face; the arrays (host,
 * n_elems x *n_elem and n_gamma_faces x *n_face int32) are filled when not
 * NULL. */
vivStatus viv_mesh_element_slots(const vivMesh* mesh, int32_t* elem_slots, int32_t* face_slots, int32_t* n_elem,
                                 int32_t* n_face);
vivStatus viv_mesh_destroy(vivMesh* mesh);

/* ---- case: state on the device ------------------------------------------ */
/* u0: n_nodes x dim host initial velocity (its prescribed components are the
 * Dirichlet values); x starts at X, p, lambda and delta at 0. */
vivStatus viv_case_create(vivMesh* mesh, const vivParams* params, const double* u0,
                          void* stream, vivCase** out);
vivStatus viv_case_destroy(vivCase* c);

/* The parameters the case runs with, after the Re / Ustar conversions of
 * viv_case_create (mu and k as used by the residual and the border rows). */
vivStatus viv_case_params(const vivCase* c, vivParams* out);

/* Checkpoint / resume of a case between time steps.  viv_case_save writes
 * the current state (u, p, x, lambda, delta), the previous time level that
 * the next BDF2 step needs, the time, the step count and dt into a host
 * buffer of *bytes bytes (caller-owned); with buf == NULL it only stores the
 * required size in *bytes.  viv_case_load restores such a buffer into a case
 * created on the same mesh with the same dt (VIV_ERR_ARG otherwise); the
 * next viv_step then computes exactly what the saved case would have
 * computed (same kernels, same inputs, deterministic reductions).  Saving
 * inside an open step (after viv_begin_step) returns VIV_ERR_STATE.  Factors
 * are not saved: the next step assembles and factors anew.  A constant-step
 * case (cfl_target = 0) must have the checkpoint's dt; an adaptive case
 * resumes with the saved step sizes.  The format is native-endian and tied to
 * the mesh's node count. */
vivStatus viv_case_save(const vivCase* c, void* buf, size_t* bytes);
vivStatus viv_case_load(vivCase* c, const void* buf, size_t bytes);

/* Overwrite the state.  Each pointer may be NULL (left unchanged); pointers
 * may be host or device memory (the `device` flag documents which; copies use
 * unified addressing).  u, x, lam: n_nodes x dim; p: n_nodes (vertex values);
 * delta: 2.  Inside a step (after viv_begin_step) this changes the Newton
 * iterate only; the BDF history was fixed by viv_begin_step. */
vivStatus viv_set_state(vivCase* c, int device, const double* u, const double* p, const double* x,
                        const double* lam, const double* delta, double t);
/* Give the previous time level (u, x at t - dt, n_nodes x dim each); the next
 * step then uses BDF2 instead of the BDF1 start. */
vivStatus viv_set_history(vivCase* c, int device, const double* u_prev, const double* x_prev);
vivStatus viv_get_state(const vivCase* c, int device, double* u, double* p, double* x, double* lam,
                        double* delta, double* t);

/* Begin a time step: shift the BDF history and form the nodal rate
 * coefficients (BDF1 on the first step, BDF2 after).  With predictor = 1 a
 * BDF2 step's Newton iterate starts from 2 U^n - U^{n-1} (u, x, delta). */
vivStatus viv_begin_step(vivCase* c);

/* Residual NL(U) (Eq. nonlinear_functional_discrete) and/or Jacobian
 * (Section 3.2, with shape derivatives) of the current state into device
 * storage.  res_norm (nullable): ||NL||_2 on the host. */
vivStatus viv_assemble(vivCase* c, int what, double* res_norm);
/* copies of the assembled residual (n_dofs) / Jacobian values (nnz, FP64
 * path: FP64; mixed path: the FP32 values widened) to host buffers */
vivStatus viv_get_residual(const vivCase* c, double* r);
vivStatus viv_get_jacobian(const vivCase* c, double* vals);

/* Numeric factorisation of the Jacobian J = [A B; C D], delta last.  A (every
 * unknown but delta) is factored by the multifrontal LU with threshold partial
 * pivoting inside fronts, or windowed pivoting (vivParams.pivoting), in the
 * case's precision.  The force-position border (Eq. coupling_constraint) is
 * then eliminated as a dense FP64 Schur block: Y = A^{-1} B (two solves with
 * the factors), S_b = D - C Y, and S_b^{-1}, all in FP64; every solve then
 * takes delta = S_b^{-1} (b_delta - C A^{-1} b_A).  A singular S_b returns
 * VIV_ERR_PIVOT from viv_step.  The factors keep each 32 x 32 diagonal block's
 * L and U inverted (for the solves); on the mixed path with windowed pivoting
 * the fronts of order >= the large-front threshold with more than 32 pivots
 * are factored in 128-column blocks and keep each 128 x 128 diagonal block's
 * L and U inverted instead.  The factors are read only by this library's
 * solves. */
vivStatus viv_factor(vivCase* c);
/* The FP64 border Schur block S_b = D - C A^{-1} B of the last factorisation,
 * row major (4 doubles, host).  VIV_ERR_STATE before viv_factor or on a mesh
 * without a cylinder. */
vivStatus viv_border_block(const vivCase* c, double* S);
/* Solve J dU = -NL for the Newton correction with iterative refinement
 * against the FP64 Jacobian values (with jacobian_fp32: the widened FP32
 * volume entries); sweeps (nullable) receives the sweep count. */
vivStatus viv_solve(vivCase* c, int* sweeps);
/* Solve J y = b for a host or device right-hand side b (n_dofs, FP64). */
vivStatus viv_solve_rhs(vivCase* c, int device, const double* b, double* y, int* sweeps);
/* Allocation-free solve (the paper has no counterpart; this serves callers).
 * Some callers cannot allocate device memory while they run - a host
 * framework whose memory pool is already committed and may not grow during a
 * time step, or a latency-bound loop that cannot take the device-wide
 * synchronisation of cudaMalloc/cudaFree.  This entry point performs one
 * forward + backward multifrontal solve J x = b with the case's current
 * factors (no refinement) and allocates nothing: its workspace is a fixed
 * 8 MiB device array inside the library.  A GPU holds the array from the
 * first viv_case_create on it until the process exits: case creation looks
 * up the array's device address (cudaGetSymbolAddress), which loads the
 * library module that holds it, and caches the address per device; so the
 * allocation-free call itself never triggers that load.  b and x are device
 * pointers to n_dofs doubles (caller-owned); work is ordered on the case's
 * stream.
 *  - A mesh whose workspace (every front's solve vector with its slice
 *    partial sums, plus n_dofs; 4 bytes per entry on the mixed path, 8 on the
 *    FP64 path; plus 256 bytes for the cylinder position) exceeds 8 MiB is
 *    rejected with VIV_ERR_ARG.
 *  - The cylinder position is solved through the FP64 border block of the
 *    last factorisation, as in every other solve.
 *  - All calls share the array and it keeps the last call's contents; the
 *    solve writes every workspace entry before reading it, so no clearing is
 *    needed.  Calls whose GPU work overlaps (other streams or threads) race on
 *    the array and must be ordered by the caller.
 *  - Returns VIV_ERR_STATE if the case has not been factored. */
vivStatus viv_lu_solve_noalloc(vivCase* c, const double* b, double* x);

/* Front Schur-complement update C -= A * B (the multifrontal GEMM of the
 * mixed path) on the tcgen05 tensor cores with 3xTF32 compensation (FP32
 * accuracy from TF32 products).  A: M x K, B: K x N, C: M x N, column-major
 * FP32 device arrays with leading dimensions lda >= M, ldb >= K, ldc >= M.
 * err: device int set to 1 if a bounded wait for the tensor cores expired.
 * Enqueued on `stream`. */
vivStatus viv_tc_schur_update(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int M, int N,
                              int K, int* err, void* stream);

/* U += dU (the last correction); Gamma nodes follow x = X + delta. */
vivStatus viv_update(vivCase* c);

/* One BDF step: begin_step, then Newton (Eq. NR_iteration) until
 * ||NL||_2 <= newton_tol.  Once ||NL|| passes the test (after at least one
 * Newton iteration), one closing correction is applied with the factors at
 * hand (no new Jacobian), with at least two refinement sweeps and then to a
 * linear residual of 1e-6 of its right-hand side (counted in refine_sweeps),
 * and ||NL|| is evaluated again.  It takes a state that only just passed the
 * test to round-off, and on the mixed path removes the error the FP32 factors
 * leave in directions the residual norm barely sees (a near-constant pressure
 * offset), so both paths land on the same discrete solution.  info nullable. */
vivStatus viv_step(vivCase* c, vivStepInfo* info);
/* Same step with host buffers: uploads the state and history, steps, and
 * downloads the new state (the end-to-end form of one step).  Packed state
 * (doubles, D = the mesh's dim, n = n_nodes): u (n x D), p (n), x (n x D),
 * lambda (n x D), delta (2), u and x of the previous level (n x D each),
 * then the time and a flag (nonzero: the previous level is valid, so the
 * step is BDF2).  state_out receives the new state with the stepped-from
 * level as the previous one, the new time and flag 1.  Host buffers of
 * viv_state_size doubles; VIV_ERR_ARG on NULL. */
vivStatus viv_step_host(vivCase* c, const double* state_in, double* state_out, vivStepInfo* info);
/* size in doubles of the packed host state used by viv_step_host: 5 D n + n + 4 */
int64_t viv_state_size(const vivMesh* mesh);

/* ---- force history analysis (host only, no device work) ------------------ */
typedef struct {
  double cd_mean, cd_amp;  /* drag coefficient C_D = F_x / (rho U^2 D / 2): time mean, half range */
  double cl_mean, cl_amp;  /* lift coefficient C_L = F_y / (rho U^2 D / 2): time mean, half range */
  double cl_rms;           /* root mean square of C_L - mean */
  double frequency;        /* dominant frequency of the lift */
  double strouhal;         /* St = frequency D / U */
  int64_t samples;         /* samples analysed */
} vivForceStats;
/* Force coefficients and the vortex-shedding frequency of a force history
 * (F = vivStepInfo.force, the fluid force -int_Gamma lambda of Section 5.3, at
 * the step times t; n samples, increasing times; host arrays read during the
 * call).  Only samples with t >= t_start are analysed (the start-up is
 * excluded).  Means and the RMS are trapezoidal time averages (the times may
 * be uneven, as with adaptive steps).  The frequency is the peak of the
 * spectrum of the lift minus its mean, resampled linearly on as many uniform
 * times, Hann-windowed and zero-padded eightfold, with the peak refined by a
 * parabola through the log-magnitudes of its bin and the two neighbours.
 * VIV_ERR_ARG with fewer than 8 samples after t_start. */
vivStatus viv_force_analysis(const double* t, const double* Fx, const double* Fy, int64_t n, double rho, double U,
                             double D, double t_start, vivForceStats* out);

/* ---- launch batching and tuning ------------------------------------------ */
/* Switch the per-case CUDA graphs on (default) or off.  With graphs on, the
 * residual, Jacobian, factorisation and each refinement sweep of viv_step are
 * captured once per case on its stream (which must not be the legacy default
 * stream) and replayed as single graph launches; they are re-captured when the
 * mesh schedule changes.  Profiling (viv_profile) bypasses the graphs. */
vivStatus viv_case_graphs(vivCase* c, int on);
/* Project autotuner: times the numeric factorisation of the case's current
 * Jacobian for several large-front thresholds (fronts at least this large use
 * 128-column outer blocks whose Schur updates run on the tensor cores) and
 * keeps the fastest.  On the mixed path with windowed pivoting it then chooses
 * per tree level (a front-size bucket) between the block LU and the per-panel
 * kernels for the level's large fronts, by the level's factorisation and solve
 * time (vivMeshInfo.block_level_mask reports the choice).  The choice belongs
 * to the mesh, never to a mix of cases: it affects every case of the mesh, so
 * call it while no other case of the mesh is running. */
vivStatus viv_autotune(vivCase* c, int32_t* best_big_front, double* best_ms);
/* Set the large-front threshold by hand (a front of order >= big_front uses
 * 128-column outer blocks); rebuilds the mesh's schedules when it changes.
 * Same scope rules as viv_autotune.  VIV_ERR_ARG if big_front <= 0. */
vivStatus viv_set_big_front(vivCase* c, int32_t big_front);
/* Set by hand the tree levels whose large fronts may use the block LU (bit l
 * for level l; -1: every level), as viv_autotune chooses them: a tuned
 * schedule can be restored without re-tuning.  Rebuilds the mesh's schedules
 * when the set changes; same scope rules as viv_autotune. */
vivStatus viv_set_block_levels(vivCase* c, int64_t mask);

/* ---- serving: parameter sweeps with continuous admission ------------------ */
typedef struct vivServer vivServer;
typedef struct {
  vivMesh* mesh;           /* device mesh (viv_mesh_create); may be shared by requests */
  vivParams params;
  const double* u0;        /* n_nodes x dim host initial velocity; copied at submit */
  int32_t n_steps;         /* BDF steps to run */
  double arrival_time;     /* seconds after server creation when the request arrives */
} vivRequest;
typedef struct {
  int64_t id;
  vivStatus status;        /* VIV_ERR_ADMISSION if it can never fit the budget */
  int32_t steps_done, newton_total;
  double t, delta[2], force[2];
  double submit_s, admit_s, finish_s;   /* server clock, seconds */
  double step_ms_mean, step_ms_max;
  char message[160];       /* error text when status != VIV_OK */
} vivResult;
typedef struct {
  double step_ms_p50, step_ms_p99;      /* over every completed step of every case */
  int64_t steps, cases_done;
  double elapsed_s;
  int32_t peak_active, active, pending;
  size_t peak_bytes;                    /* peak of the admitted predicted device bytes */
  double steady_ms_p50, steady_ms_p99;  /* the same without each case's first two steps, which
                                           capture the case's CUDA graphs (BDF1, then BDF2) */
} vivServerStats;
/* A serving loop: requests arrive over time, are admitted FIFO while the
 * predicted device bytes of the admitted cases (viv_mesh_info) stay within
 * mem_budget and fewer than max_active cases run; each admitted case runs on
 * its own stream and worker thread, so cases overlap on the GPU, and its
 * memory is returned when it finishes.  A failed case reports its status and
 * does not affect the others.  Cases allocate with cudaMalloc. */
vivStatus viv_server_create(size_t mem_budget, int32_t max_active, vivServer** out);
vivStatus viv_server_submit(vivServer* s, const vivRequest* req, int64_t* id);
/* finished results not yet polled (up to max); waits up to wait_ms for one */
vivStatus viv_server_poll(vivServer* s, vivResult* out, int32_t max, int32_t* n, int32_t wait_ms);
/* final state of a finished case: u, x, lam (n_nodes x dim), p (n_nodes), delta (2) */
vivStatus viv_server_state(vivServer* s, int64_t id, double* u, double* p, double* x, double* lam,
                           double* delta);
vivStatus viv_server_stats(vivServer* s, vivServerStats* out);
/* runs every submitted request to completion, then frees the server */
vivStatus viv_server_destroy(vivServer* s);

/* ---- instrumentation ----------------------------------------------------- */
/* kernel launches issued by this library in this process so far */
int64_t viv_kernel_launches(void);
/* per-case CUDA-event timing of every kernel launch, by kind:
 * 0 residual elements, 1 Jacobian elements, 2 Gamma faces and border rows,
 * 3 front assembly, 4 panel LU, 5 TRSM, 6 Schur GEMM, 7 forward solve,
 * 8 backward solve, 9 refinement SpMV, 10 vector kernels, 11 tensor-core
 * (tcgen05) Schur updates, 12 their operand split (hi/lo TF32 images).
 * viv_profile_read(ms[13], count[13]) synchronises and resets. */
enum { VIV_NKINDS = 13 };
vivStatus viv_profile(vivCase* c, int on);
vivStatus viv_profile_read(vivCase* c, double* ms, int64_t* count);
/* Factorisation kernel time of the last viv_profile_read split by elimination
 * tree level (0 = leaves) and kind: ms[l * VIV_NKINDS + k] for
 * l < min(max_levels, *n_levels); *n_levels receives the number of levels
 * recorded.  Host buffer of max_levels * VIV_NKINDS doubles. */
vivStatus viv_profile_levels(const vivCase* c, double* ms, int32_t max_levels, int32_t* n_levels);

const char* viv_last_error(void);
const char* viv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VIV_H */
