// Vector kernels of the Newton driver: deterministic norms, BDF history,
// the Newton update, the FP64 refinement residual r = b - J x (CSR SpMV).
#include <cuda_runtime.h>

#include "viv_internal.h"

namespace viv {
namespace {

constexpr int NORM_BLOCKS = 296;   // 2 x 148 SMs
constexpr int NORM_THREADS = 256;

// sum of squares per block, in a fixed order for a fixed grid (deterministic)
__global__ void __launch_bounds__(NORM_THREADS) sumsq_partial(const double* v, int64_t n, double* partial) {
  __shared__ double red[NORM_THREADS];
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)NORM_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * NORM_THREADS) {
    double a = v[i];
    s += a * a;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = NORM_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(NORM_THREADS) sumsq_final(const double* partial, int n, double* out) {
  __shared__ double red[NORM_THREADS];
  double s = 0;
  for (int i = threadIdx.x; i < n; i += NORM_THREADS) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = NORM_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(red[0]);
}

__global__ void bdf_kernel(int64_t n2, const double* u_n, const double* u_nm1, const double* x_n,
                           const double* x_nm1, double a_n, double a_nm1, double* hu, double* hx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n2) return;
  double su = a_n * u_n[i], sx = a_n * x_n[i];
  if (a_nm1 != 0.0) {
    su += a_nm1 * u_nm1[i];
    sx += a_nm1 * x_nm1[i];
  }
  hu[i] = su;
  hx[i] = sx;
}

// Newton starting point U^n + w (U^n - U^{n-1}) for u and x (all nodal
// entries): the linear extrapolation with step ratio w = dt / dt_prev
__global__ void extrapolate_kernel(int64_t n2, const double* u_n, const double* u_nm1, const double* x_n,
                                   const double* x_nm1, double w, double* u, double* x) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n2) return;
  u[i] = (1.0 + w) * u_n[i] - w * u_nm1[i];
  x[i] = (1.0 + w) * x_n[i] - w * x_nm1[i];
}

// Courant number: per element the largest nodal |u| over the shortest edge
// between corner nodes (current configuration); block maxima, then the max
__global__ void __launch_bounds__(NORM_THREADS) cfl_partial_kernel(int64_t E, const int32_t* conn, const double* x,
                                                                   const double* u, double* partial) {
  __shared__ double red[NORM_THREADS];
  double mx = 0;
  for (int64_t e = blockIdx.x * (int64_t)NORM_THREADS + threadIdx.x; e < E; e += (int64_t)gridDim.x * NORM_THREADS) {
    const int32_t* c = conn + 9 * e;
    const int corner[4] = {0, 2, 8, 6};
    double h2 = 1e300, um2 = 0;
    for (int k = 0; k < 4; ++k) {
      const int a = c[corner[k]], b = c[corner[(k + 1) & 3]];
      const double dx = x[2 * a] - x[2 * b], dy = x[2 * a + 1] - x[2 * b + 1];
      h2 = fmin(h2, dx * dx + dy * dy);
    }
    for (int k = 0; k < 9; ++k) {
      const int a = c[k];
      um2 = fmax(um2, u[2 * a] * u[2 * a] + u[2 * a + 1] * u[2 * a + 1]);
    }
    mx = fmax(mx, sqrt(um2) / sqrt(h2));
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = NORM_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(NORM_THREADS) cfl_final_kernel(const double* partial, int n, double dt, double* out) {
  __shared__ double red[NORM_THREADS];
  double mx = 0;
  for (int i = threadIdx.x; i < n; i += NORM_THREADS) mx = fmax(mx, partial[i]);
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = NORM_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = dt * red[0];
}

// delta read back from a Gamma node's position (x = X + (delta, 0) on Gamma)
__global__ void delta_from_x_kernel(int64_t a, int D, const double* X, const double* x, double* delta) {
  if (threadIdx.x < 2) delta[threadIdx.x] = x[D * a + threadIdx.x] - X[D * a + threadIdx.x];
}

// U += dU for every nodal field (D components of u, x, lambda); Gamma nodes
// follow x = X + (delta_new, 0) (their z position is held)
__global__ void update_kernel(int64_t n, int D, const int32_t* node_dof, const int32_t* tags, const double* X,
                              const int32_t* delta_dof, const double* delta, const double* dU, double* u,
                              double* p, double* x, double* lam) {
  int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n) return;
  const int32_t* d = node_dof + a * NSLOT;
  for (int i = 0; i < D; ++i)
    if (d[S_UX + i] >= 0) u[D * a + i] += dU[d[S_UX + i]];
  if (d[S_P] >= 0) p[a] += dU[d[S_P]];
  if (tags[a] & VIV_TAG_CYL) {
    for (int i = 0; i < D; ++i) lam[D * a + i] += dU[d[S_LX + i]];
    for (int i = 0; i < 2; ++i) x[D * a + i] = X[D * a + i] + (delta[i] + dU[delta_dof[i]]);
  } else {
    for (int i = 0; i < D; ++i)
      if (d[S_XX + i] >= 0) x[D * a + i] += dU[d[S_XX + i]];
  }
}

__global__ void delta_update_kernel(const int32_t* delta_dof, const double* dU, double* delta) {
  if (threadIdx.x < 2 && delta_dof[0] >= 0) delta[threadIdx.x] += dU[delta_dof[threadIdx.x]];
}

// r = b - J x, one warp per row (rows hold ~20-90 entries)
__global__ void spmv_residual_kernel(int64_t nrows, const int64_t* rp, const int32_t* col, const double* J,
                                     const double* x, const double* b, double* r) {
  int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= nrows) return;
  double s = 0;
  for (int64_t q = rp[row] + lane; q < rp[row + 1]; q += 32) s += J[q] * x[col[q]];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) r[row] = b[row] - s;
}

__global__ void axpy_kernel(double* y, const double* x, double a, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

__global__ void scale_copy_kernel(double* y, const double* x, double a, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i];
}

__global__ void f64_to_f32_kernel(float* y, const double* x, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

__global__ void f32_to_f64_kernel(double* y, const float* x, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (double)x[i];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---- border: the two delta unknowns eliminated after the fronts -------------
// (J = [A B; C D]; Y = A^{-1} B from the factors, S_b = D - C Y in FP64)

// column j of B as a dense front-row vector (dst zeroed beforehand)
__global__ void border_scatter_kernel(int n, const int32_t* __restrict__ row, const int32_t* __restrict__ q,
                                      const double* __restrict__ J, double* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[row[i]] = J[q[i]];
}

constexpr int BORDER_THREADS = 256;

// deterministic block sum of one value per thread
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = BORDER_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// S_b = D - C Y and its inverse: Sb[0..3] = S (row major), Sb[4..7] = S^{-1};
// a singular S_b sets *flag
__global__ void __launch_bounds__(BORDER_THREADS) border_schur_kernel(int c0_end, int c1_end, const int32_t* col,
                                                                      const int32_t* q, int4 dq, const double* J,
                                                                      const double* Y, int64_t ldy, double* Sb,
                                                                      int32_t* flag) {
  __shared__ double red[BORDER_THREADS];
  double S[4];
  for (int i = 0; i < 2; ++i) {
    const int b0 = i == 0 ? 0 : c0_end, b1 = i == 0 ? c0_end : c1_end;
    double a0 = 0, a1 = 0;
    for (int k = b0 + threadIdx.x; k < b1; k += BORDER_THREADS) {
      const double c = J[q[k]];
      a0 += c * Y[col[k]];
      a1 += c * Y[ldy + col[k]];
    }
    const int d0 = i == 0 ? dq.x : dq.z, d1 = i == 0 ? dq.y : dq.w;
    S[2 * i] = (d0 >= 0 ? J[d0] : 0.0) - block_sum(a0, red);
    S[2 * i + 1] = (d1 >= 0 ? J[d1] : 0.0) - block_sum(a1, red);
  }
  if (threadIdx.x == 0) {
    const double det = S[0] * S[3] - S[1] * S[2];
    const double scale = fabs(S[0] * S[3]) + fabs(S[1] * S[2]);
    for (int k = 0; k < 4; ++k) Sb[k] = S[k];
    if (!(fabs(det) > 1e-300 && fabs(det) > 1e-14 * scale)) {
      atomicExch(flag, 1);
      for (int k = 4; k < 8; ++k) Sb[k] = 0.0;
    } else {
      Sb[4] = S[3] / det;
      Sb[5] = -S[1] / det;
      Sb[6] = -S[2] / det;
      Sb[7] = S[0] / det;
    }
  }
}

// delta = S_b^{-1} (b_delta - C z) with z = x[0 : nA] (the front solve), into
// x[nA], x[nA + 1] and dtmp[0..1]
__global__ void __launch_bounds__(BORDER_THREADS) border_delta_kernel(int c0_end, int c1_end, const int32_t* col,
                                                                      const int32_t* q, const double* J,
                                                                      const double* b, double* x, int64_t nA,
                                                                      const double* Sb, double* dtmp) {
  __shared__ double red[BORDER_THREADS];
  double t[2];
  for (int i = 0; i < 2; ++i) {
    const int b0 = i == 0 ? 0 : c0_end, b1 = i == 0 ? c0_end : c1_end;
    double a = 0;
    for (int k = b0 + threadIdx.x; k < b1; k += BORDER_THREADS) a += J[q[k]] * x[col[k]];
    t[i] = b[nA + i] - block_sum(a, red);
  }
  if (threadIdx.x == 0) {
    const double d0 = Sb[4] * t[0] + Sb[5] * t[1], d1 = Sb[6] * t[0] + Sb[7] * t[1];
    x[nA] = d0;
    x[nA + 1] = d1;
    dtmp[0] = d0;
    dtmp[1] = d1;
  }
}

// x[0 : nA] -= Y delta
__global__ void border_back_kernel(int64_t nA, const double* Y, int64_t ldy, const double* dtmp, double* x) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nA) return;
  x[r] -= Y[r] * dtmp[0] + Y[ldy + r] * dtmp[1];
}

}  // namespace

void launch_norm2(const double* v, int64_t n, double* partial, double* out, cudaStream_t s) {
  {
    Launched L(K_VEC, s);
    sumsq_partial<<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(v, n, partial);
  }
  {
    Launched L(K_VEC, s);
    sumsq_final<<<1, NORM_THREADS, 0, s>>>(partial, NORM_BLOCKS, out);
  }
  VIV_CUDA(cudaGetLastError());
}

void launch_bdf_history(const Mesh& m, CaseState& st, double a_n, double a_nm1, bool, cudaStream_t s) {
  int64_t n2 = m.dim * m.n_nodes;
  Launched L(K_VEC, s);
  bdf_kernel<<<blocks_for(n2, 256), 256, 0, s>>>(n2, st.u_n, st.u_nm1, st.x_n, st.x_nm1, a_n, a_nm1, st.hu,
                                                   st.hx);
  VIV_CUDA(cudaGetLastError());
}

void launch_extrapolate(const Mesh& m, CaseState& st, double w, cudaStream_t s) {
  const int64_t n2 = m.dim * m.n_nodes;
  {
    Launched L(K_VEC, s);
    extrapolate_kernel<<<blocks_for(n2, 256), 256, 0, s>>>(n2, st.u_n, st.u_nm1, st.x_n, st.x_nm1, w, st.u, st.x);
  }
  if (m.n_faces > 0) {
    Launched L(K_VEC, s);
    delta_from_x_kernel<<<1, 32, 0, s>>>(m.faces[0], m.dim, m.d_X, st.x, st.delta);
  }
  VIV_CUDA(cudaGetLastError());
}

void launch_update(const Mesh& m, CaseState& st, const double* dU, cudaStream_t s) {
  {
    Launched L(K_VEC, s);
    update_kernel<<<blocks_for(m.n_nodes, 256), 256, 0, s>>>(m.n_nodes, m.dim, m.d_node_dof, m.d_tags, m.d_X,
                                                              m.d_delta_dof, st.delta, dU, st.u, st.p, st.x,
                                                              st.lam);
  }
  if (m.tri) launch_midside_positions(m, st.x, s);   // P1 position: midpoints follow the vertices
  {
    Launched L(K_VEC, s);
    delta_update_kernel<<<1, 32, 0, s>>>(m.d_delta_dof, dU, st.delta);
  }
  VIV_CUDA(cudaGetLastError());
}

void launch_spmv_residual(const Mesh& m, const double* J, const double* x, const double* b, double* r,
                          cudaStream_t s) {
  int64_t threads = m.n_dofs * 32;
  Launched L(K_SPMV, s);
  spmv_residual_kernel<<<blocks_for(threads, 256), 256, 0, s>>>(m.n_dofs, m.d_row_ptr, m.d_col, J, x, b, r);
  VIV_CUDA(cudaGetLastError());
}

void launch_axpy(double* y, const double* x, double a, int64_t n, cudaStream_t s) {
  Launched L(K_VEC, s);
  axpy_kernel<<<blocks_for(n, 256), 256, 0, s>>>(y, x, a, n);
  VIV_CUDA(cudaGetLastError());
}

void launch_scale_copy(double* y, const double* x, double a, int64_t n, cudaStream_t s) {
  Launched L(K_VEC, s);
  scale_copy_kernel<<<blocks_for(n, 256), 256, 0, s>>>(y, x, a, n);
  VIV_CUDA(cudaGetLastError());
}

void launch_f64_to_f32(float* y, const double* x, int64_t n, cudaStream_t s) {
  Launched L(K_VEC, s);
  f64_to_f32_kernel<<<blocks_for(n, 256), 256, 0, s>>>(y, x, n);
  VIV_CUDA(cudaGetLastError());
}

void launch_f32_to_f64(double* y, const float* x, int64_t n, cudaStream_t s) {
  Launched L(K_VEC, s);
  f32_to_f64_kernel<<<blocks_for(n, 256), 256, 0, s>>>(y, x, n);
  VIV_CUDA(cudaGetLastError());
}

// ---- border launchers --------------------------------------------------------
void launch_border_column(const Mesh& m, const double* J, int j, double* dst, cudaStream_t s) {
  VIV_CUDA(cudaMemsetAsync(dst, 0, (size_t)m.n_dofs * sizeof(double), s));
  const int b0 = m.bb_off[j], n = m.bb_off[j + 1] - b0;
  if (n > 0) {
    Launched L(K_VEC, s);
    border_scatter_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, m.d_bb_row + b0, m.d_bb_q + b0, J, dst);
  }
  VIV_CUDA(cudaGetLastError());
}

void launch_border_schur(const Mesh& m, const double* J, const double* Y, double* Sb, int32_t* flag,
                         cudaStream_t s) {
  Launched L(K_VEC, s);
  border_schur_kernel<<<1, BORDER_THREADS, 0, s>>>(m.bc_off[1], m.bc_off[2], m.d_bc_col, m.d_bc_q,
                                                   make_int4(m.bd_q[0], m.bd_q[1], m.bd_q[2], m.bd_q[3]), J, Y,
                                                   m.n_dofs, Sb, flag);
  VIV_CUDA(cudaGetLastError());
}

void launch_border_solve(const Mesh& m, const double* J, const double* b, double* x, const double* Y,
                         const double* Sb, double* dtmp, cudaStream_t s) {
  {
    Launched L(K_VEC, s);
    border_delta_kernel<<<1, BORDER_THREADS, 0, s>>>(m.bc_off[1], m.bc_off[2], m.d_bc_col, m.d_bc_q, J, b, x,
                                                     m.n_front_dofs, Sb, dtmp);
  }
  {
    Launched L(K_VEC, s);
    border_back_kernel<<<blocks_for(m.n_front_dofs, 256), 256, 0, s>>>(m.n_front_dofs, Y, m.n_dofs, dtmp, x);
  }
  VIV_CUDA(cudaGetLastError());
}

// Courant number dt max_e (max_a |u_a| / h_e) of the current state, read back
double launch_cfl(const Mesh& m, const CaseState& st, double dt, double* partial, double* out, double* host,
                  cudaStream_t s) {
  {
    Launched L(K_VEC, s);
    cfl_partial_kernel<<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(m.n_elems, m.d_conn, st.x, st.u, partial);
  }
  {
    Launched L(K_VEC, s);
    cfl_final_kernel<<<1, NORM_THREADS, 0, s>>>(partial, NORM_BLOCKS, dt, out);
  }
  VIV_CUDA(cudaGetLastError());
  VIV_CUDA(cudaMemcpyAsync(host, out, sizeof(double), cudaMemcpyDeviceToHost, s));
  VIV_CUDA(cudaStreamSynchronize(s));
  return *host;
}

}  // namespace viv
