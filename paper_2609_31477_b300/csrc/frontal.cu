// Multifrontal LU of the Jacobian on the GPU (replaces the sparse direct
// solver of Section 4.4).  Fronts are dense column-major blocks in one pool;
// each tree level is processed by batched launches over all of its fronts:
//
//   assemble : zero the front, place the original CSR entries, extend-add the
//              children's contribution blocks (children in a fixed order, so
//              the sums are deterministic)
//   panel    : partial LU of PANEL_NB pivot columns with threshold partial
//              pivoting restricted to the fully summed rows; a pivot below the
//              threshold is counted, an empty fully summed column is replaced
//              by a small static perturbation and counted
//   trsm     : U12 = L11^{-1} A12 for the panel rows
//   gemm     : A22 -= L21 U12 (the Schur-complement update)
//
// The forward and backward solves walk the same tree: each front gathers
// its children's update vectors (extend-add on vectors), so no global atomics
// are used and results do not depend on the launch order.
#include <cuda_runtime.h>

#include <cfloat>

#include "viv_internal.h"

namespace viv {
namespace {

template <class T>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double v = DBL_EPSILON;
};
template <>
struct Eps<float> {
  static constexpr float v = FLT_EPSILON;
};

struct FT {   // front tables passed by value
  const int64_t* off;
  const int32_t* m;
  const int32_t* p;
  const int32_t* first;
  const int64_t* idx_off;
  const int32_t* idx;
  const int64_t* nz_off;
  const int32_t* nz_csr;
  const int32_t* nz_pos;
  const int32_t* child_off;
  const int32_t* child;
  const int64_t* ea_off;
  const int32_t* ea;
  const int64_t* vec_off;
  const int32_t* piv_off;
  const int32_t* col_nz;
  const int64_t* col_nz_off;
};

FT make_ft(const Mesh& m) {
  const FrontTables& t = m.ft;
  return FT{t.off, t.m, t.p, t.first, t.idx_off, t.idx, t.nz_off, t.nz_csr, t.nz_pos, t.child_off,
            t.child, t.ea_off, t.ea, t.vec_off, t.piv_off, t.col_nz, t.col_nz_off};
}

__device__ __forceinline__ int lower_bound_i(const int32_t* a, int n, int v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

template <class T, class S>
__global__ void assemble_kernel(FT ft, const int32_t* work, const S* J, T* pool) {
  const int32_t* it = work + 3 * blockIdx.x;
  const int f = it[0], c0 = it[1];
  const int m = ft.m[f];
  const int c1 = min(c0 + ASM_COLS, m);
  T* F = pool + ft.off[f];
  const int64_t span = (int64_t)(c1 - c0) * m;
  for (int64_t q = threadIdx.x; q < span; q += blockDim.x) F[(int64_t)c0 * m + q] = T(0);
  __syncthreads();
  const int ch = c0 / ASM_COLS;
  const int64_t base = ft.nz_off[f];
  const int32_t* cn = ft.col_nz + ft.col_nz_off[f];
  for (int64_t q = base + cn[ch] + threadIdx.x; q < base + cn[ch + 1]; q += blockDim.x)
    F[ft.nz_pos[q]] = (T)J[ft.nz_csr[q]];
  __syncthreads();
  for (int cc = ft.child_off[f]; cc < ft.child_off[f + 1]; ++cc) {
    const int c = ft.child[cc];
    const int mc = ft.m[c], pc = ft.p[c], nc = mc - pc;
    if (nc == 0) continue;
    const int32_t* ea = ft.ea + ft.ea_off[c];
    const int lo = lower_bound_i(ea, nc, c0), hi = lower_bound_i(ea, nc, c1);
    const T* C = pool + ft.off[c];
    const int64_t cnt = (int64_t)(hi - lo) * nc;
    for (int64_t q = threadIdx.x; q < cnt; q += blockDim.x) {
      const int r = (int)(q % nc), k = lo + (int)(q / nc);
      F[ea[r] + (int64_t)ea[k] * m] += C[(pc + r) + (int64_t)(pc + k) * mc];
    }
    __syncthreads();
  }
}

constexpr int PANEL_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(PANEL_THREADS) panel_kernel(FT ft, const int32_t* work, int k, T* pool,
                                                              int32_t* piv, int32_t* stats, T thresh) {
  const int f = work[3 * blockIdx.x];
  const int m = ft.m[f], p = ft.p[f];
  T* F = pool + ft.off[f];
  int32_t* pv = piv + ft.piv_off[f];
  const int nbe = min(PANEL_NB, p - k);
  __shared__ T s_max[PANEL_THREADS / 32], s_best[PANEL_THREADS / 32];
  __shared__ int s_row[PANEL_THREADS / 32];
  __shared__ int s_piv;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = k; j < k + nbe; ++j) {
    const T* colj = F + (int64_t)j * m;
    T cmax = 0, best = -1;
    int brow = j;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
      T a = fabs(colj[i]);
      cmax = a > cmax ? a : cmax;
      if (i < p && (a > best || (a == best && i < brow))) {
        best = a;
        brow = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T om = __shfl_xor_sync(0xffffffffu, cmax, o);
      cmax = om > cmax ? om : cmax;
      T ob = __shfl_xor_sync(0xffffffffu, best, o);
      int orow = __shfl_xor_sync(0xffffffffu, brow, o);
      if (ob > best || (ob == best && orow < brow)) {
        best = ob;
        brow = orow;
      }
    }
    if (lane == 0) {
      s_max[wid] = cmax;
      s_best[wid] = best;
      s_row[wid] = brow;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      T cm = 0, bb = -1;
      int br = j;
      for (int w = 0; w < PANEL_THREADS / 32; ++w) {
        cm = s_max[w] > cm ? s_max[w] : cm;
        if (s_best[w] > bb || (s_best[w] == bb && s_row[w] < br)) {
          bb = s_best[w];
          br = s_row[w];
        }
      }
      T diag = fabs(colj[j]);
      int r;
      if (diag > 0 && diag >= thresh * cm) {
        r = j;
      } else if (bb > 0) {
        r = br;
        if (bb < thresh * cm) atomicAdd(&stats[1], 1);
      } else {
        // no usable pivot in the fully summed rows: static perturbation
        r = j;
        T scale = cm > 0 ? cm : T(1);
        F[(int64_t)j * m + j] = sqrt(Eps<T>::v) * scale;
        atomicAdd(&stats[0], 1);
      }
      pv[j] = r;
      s_piv = r;
    }
    __syncthreads();
    const int r = s_piv;
    if (r != j)
      for (int c = threadIdx.x; c < m; c += blockDim.x) {
        T a = F[(int64_t)c * m + j];
        F[(int64_t)c * m + j] = F[(int64_t)c * m + r];
        F[(int64_t)c * m + r] = a;
      }
    __syncthreads();
    const T inv = T(1) / F[(int64_t)j * m + j];
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) F[(int64_t)j * m + i] *= inv;
    __syncthreads();
    const int ncol = k + nbe - j - 1;
    const int nrow = m - j - 1;
    for (int q = threadIdx.x; q < ncol * nrow; q += blockDim.x) {
      const int i = j + 1 + q % nrow, l = j + 1 + q / nrow;
      F[(int64_t)l * m + i] -= F[(int64_t)j * m + i] * F[(int64_t)l * m + j];
    }
    __syncthreads();
  }
}

template <class T>
__global__ void trsm_kernel(FT ft, const int32_t* work, int k, T* pool) {
  const int32_t* it = work + 3 * blockIdx.x;
  const int f = it[0], c0 = it[1];
  const int m = ft.m[f], p = ft.p[f];
  const int nbe = min(PANEL_NB, p - k);
  const int c1 = min(c0 + TRSM_COLS, m);
  T* F = pool + ft.off[f];
  __shared__ T L[PANEL_NB][PANEL_NB + 1];
  __shared__ T B[PANEL_NB][TRSM_COLS + 1];
  for (int q = threadIdx.x; q < nbe * nbe; q += blockDim.x) {
    int i = q % nbe, l = q / nbe;
    L[i][l] = F[(int64_t)(k + l) * m + k + i];
  }
  const int nc = c1 - c0;
  for (int q = threadIdx.x; q < nbe * nc; q += blockDim.x) {
    int i = q % nbe, c = q / nbe;
    B[i][c] = F[(int64_t)(c0 + c) * m + k + i];
  }
  __syncthreads();
  if (threadIdx.x < nc) {
    const int c = threadIdx.x;
    for (int i = 1; i < nbe; ++i) {
      T s = B[i][c];
      for (int l = 0; l < i; ++l) s -= L[i][l] * B[l][c];
      B[i][c] = s;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nbe * nc; q += blockDim.x) {
    int i = q % nbe, c = q / nbe;
    F[(int64_t)(c0 + c) * m + k + i] = B[i][c];
  }
}

// C[r0 + 64 ti .., r0 + 64 tj ..] -= L21 * U12 with K = nbe <= 32
template <class T>
__global__ void __launch_bounds__(256) gemm_kernel(FT ft, const int32_t* work, int k, T* pool) {
  const int32_t* it = work + 3 * blockIdx.x;
  const int f = it[0], ti = it[1], tj = it[2];
  const int m = ft.m[f], p = ft.p[f];
  const int nbe = min(PANEL_NB, p - k);
  const int r0 = k + nbe;
  const int rb = r0 + ti * GEMM_TILE, cb = r0 + tj * GEMM_TILE;
  T* F = pool + ft.off[f];
  __shared__ T As[PANEL_NB][GEMM_TILE + 1];   // [kk][row]
  __shared__ T Bs[PANEL_NB][GEMM_TILE + 1];   // [kk][col]
  for (int q = threadIdx.x; q < PANEL_NB * GEMM_TILE; q += blockDim.x) {
    int r = q % GEMM_TILE, kk = q / GEMM_TILE;
    T a = 0, b = 0;
    if (kk < nbe) {
      if (rb + r < m) a = F[(int64_t)(k + kk) * m + rb + r];
      if (cb + r < m) b = F[(int64_t)(cb + r) * m + k + kk];
    }
    As[kk][r] = a;
    Bs[kk][r] = b;
  }
  __syncthreads();
  const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;
  T acc[4][4] = {};
  for (int kk = 0; kk < nbe; ++kk) {
    T a[4], b[4];
    for (int u = 0; u < 4; ++u) {
      a[u] = As[kk][tr + 16 * u];
      b[u] = Bs[kk][tc + 16 * u];
    }
    for (int u = 0; u < 4; ++u)
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
  }
  for (int v = 0; v < 4; ++v) {
    const int c = cb + tc + 16 * v;
    if (c >= m) continue;
    for (int u = 0; u < 4; ++u) {
      const int r = rb + tr + 16 * u;
      if (r < m) F[(int64_t)c * m + r] -= acc[u][v];
    }
  }
}

// ---- solves -----------------------------------------------------------------------
template <class T>
__global__ void fwd_kernel(FT ft, const int32_t* fronts, const T* pool, const int32_t* piv, const double* b,
                           T* vec, T* yv) {
  const int f = fronts[blockIdx.x];
  const int m = ft.m[f], p = ft.p[f], first = ft.first[f];
  T* w = vec + ft.vec_off[f];
  const T* F = pool + ft.off[f];
  for (int i = threadIdx.x; i < m; i += blockDim.x) w[i] = i < p ? (T)b[first + i] : T(0);
  __syncthreads();
  for (int cc = ft.child_off[f]; cc < ft.child_off[f + 1]; ++cc) {
    const int c = ft.child[cc];
    const int nc = ft.m[c] - ft.p[c];
    const int32_t* ea = ft.ea + ft.ea_off[c];
    const T* wc = vec + ft.vec_off[c] + ft.p[c];
    for (int r = threadIdx.x; r < nc; r += blockDim.x) w[ea[r]] += wc[r];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int32_t* pv = piv + ft.piv_off[f];
    for (int j = 0; j < p; ++j) {
      int r = pv[j];
      if (r != j) {
        T t = w[j];
        w[j] = w[r];
        w[r] = t;
      }
    }
  }
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    const T xj = w[j];
    const T* col = F + (int64_t)j * m;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) w[i] -= col[i] * xj;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < p; i += blockDim.x) yv[first + i] = w[i];
}

template <class T>
__global__ void bwd_kernel(FT ft, const int32_t* fronts, const T* pool, const T* yv, T* vec, double* x) {
  const int f = fronts[blockIdx.x];
  const int m = ft.m[f], p = ft.p[f], first = ft.first[f];
  T* v = vec + ft.vec_off[f];
  const T* F = pool + ft.off[f];
  const int32_t* idx = ft.idx + ft.idx_off[f];
  for (int i = threadIdx.x; i < m; i += blockDim.x) v[i] = i < p ? yv[first + i] : (T)x[idx[i]];
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    T s = v[i];
    for (int c = p; c < m; ++c) s -= F[(int64_t)c * m + i] * v[c];
    v[i] = s;
  }
  __syncthreads();
  for (int j = p - 1; j >= 0; --j) {
    if (threadIdx.x == 0) v[j] /= F[(int64_t)j * m + j];
    __syncthreads();
    const T xj = v[j];
    const T* col = F + (int64_t)j * m;
    for (int i = threadIdx.x; i < j; i += blockDim.x) v[i] -= col[i] * xj;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < p; i += blockDim.x) x[first + i] = (double)v[i];
}

}  // namespace

template <class T>
void factor_numeric(const Mesh& m, const double* J64, const float* J32, T* fronts, int32_t* piv,
                    int32_t* stats, double threshold, cudaStream_t s) {
  FT ft = make_ft(m);
  VIV_CUDA(cudaMemsetAsync(stats, 0, 2 * sizeof(int32_t), s));
  const int32_t* work = m.ft.work;
  for (const Launch& L : m.sched) {
    const int32_t* w = work + 3 * L.item0;
    const unsigned grid = (unsigned)L.count;
    static const int kk[4] = {K_FRONT_ASM, K_PANEL, K_TRSM, K_GEMM};
    Launched LL(kk[L.kind], s);
    switch (L.kind) {
      case L_ASSEMBLE:
        if (J32)
          assemble_kernel<T, float><<<grid, 256, 0, s>>>(ft, w, J32, fronts);
        else
          assemble_kernel<T, double><<<grid, 256, 0, s>>>(ft, w, J64, fronts);
        break;
      case L_PANEL:
        panel_kernel<T><<<grid, PANEL_THREADS, 0, s>>>(ft, w, L.k, fronts, piv, stats, (T)threshold);
        break;
      case L_TRSM:
        trsm_kernel<T><<<grid, TRSM_COLS, 0, s>>>(ft, w, L.k, fronts);
        break;
      case L_GEMM:
        gemm_kernel<T><<<grid, 256, 0, s>>>(ft, w, L.k, fronts);
        break;
    }
  }
  VIV_CUDA(cudaGetLastError());
}

template <class T>
void solve_fronts(const Mesh& m, const T* fronts, const int32_t* piv, const double* b, double* x, T* vec,
                  T* yv, cudaStream_t s) {
  FT ft = make_ft(m);
  for (int l = 0; l < m.n_levels; ++l) {
    int n = m.level_off[l + 1] - m.level_off[l];
    Launched L(K_FWD, s);
    fwd_kernel<T><<<n, 256, 0, s>>>(ft, m.d_level_fronts + m.level_off[l], fronts, piv, b, vec, yv);
  }
  for (int l = m.n_levels - 1; l >= 0; --l) {
    int n = m.level_off[l + 1] - m.level_off[l];
    Launched L(K_BWD, s);
    bwd_kernel<T><<<n, 256, 0, s>>>(ft, m.d_level_fronts + m.level_off[l], fronts, yv, vec, x);
  }
  VIV_CUDA(cudaGetLastError());
}

template void factor_numeric<double>(const Mesh&, const double*, const float*, double*, int32_t*, int32_t*,
                                     double, cudaStream_t);
template void factor_numeric<float>(const Mesh&, const double*, const float*, float*, int32_t*, int32_t*,
                                    double, cudaStream_t);
template void solve_fronts<double>(const Mesh&, const double*, const int32_t*, const double*, double*, double*,
                                   double*, cudaStream_t);
template void solve_fronts<float>(const Mesh&, const float*, const int32_t*, const double*, double*, float*,
                                  float*, cudaStream_t);

}  // namespace viv
