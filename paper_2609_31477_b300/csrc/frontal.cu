// Multifrontal LU of the Jacobian on the GPU (replaces the sparse direct
// solver of Section 4.3).  Fronts are dense column-major blocks in one pool;
// each tree level is processed by batched launches over all of its fronts, in
// 32-column panel steps:
//
//   assemble : zero the front, place the original CSR entries, extend-add the
//              children's contribution blocks (children in a fixed order, so
//              the sums are deterministic)
//   threshold pivoting (vivParams.pivoting = 0):
//     panel  : partial LU of PANEL_NB pivot columns with threshold partial
//              pivoting restricted to the fully summed rows; a pivot below the
//              threshold is counted, an empty fully summed column is replaced
//              by a small static perturbation and counted.  The m x PANEL_NB
//              panel is held in shared memory (one CTA, or the distributed
//              shared memory of a PANEL_CLUSTER-CTA cluster with a DSMEM pivot
//              reduction); row interchanges outside the panel follow (laswp)
//     trsm   : U12 = L11^{-1} A12 for the panel rows
//   windowed pivoting (vivParams.pivoting = 1):
//     diag   : one warp factors the 32 x 32 diagonal block with partial
//              pivoting inside it (run inside the previous panel's gemm tile
//              that covers the block when there is one)
//     window : L21 = A21 U11^{-1} and U12 = L11^{-1} P A12 in one launch
//   gemm     : A22 -= L21 U12 inside the front's 128-column outer block (SIMT)
//   tc       : the outer block's K = 128 Schur update of large fronts on the
//              tcgen05 tensor cores (3xTF32, tc_mma.cuh)
//
// After the factorisation every diagonal block's L11 and U11 are inverted in
// place and each front's interchanges are composed into one permutation.  The
// forward and backward solves walk the same tree: a CTA per front runs the
// triangular chain over its pivot rows, and multi-CTA slice products handle
// the off-diagonal blocks; each front gathers its children's update vectors,
// so no global atomics are used and results do not depend on launch order.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <mutex>
#include <type_traits>

#include "tc_pipe.cuh"
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
  const uint8_t* blk;   // solves: fronts whose 128-row diagonal blocks are stored inverted (or null)
  const uint8_t* fused; // solves: slice products formed in the chain CTA (1 forward, 2 backward)
};

FT make_ft(const Mesh& m, bool blk = false) {
  const FrontTables& t = m.ft;
  return FT{t.off, t.m, t.p, t.first, t.idx_off, t.idx, t.nz_off, t.nz_csr, t.nz_pos, t.child_off,
            t.child, t.ea_off, t.ea, t.vec_off, t.piv_off, t.col_nz, t.col_nz_off, blk ? m.d_blk_front : nullptr,
            m.d_solve_fused};
}


template <class T, class S>
__global__ void assemble_kernel(FT ft, const int32_t* work, const S* J, T* pool) {
  const int32_t* it = work + WORK_STRIDE * blockIdx.x;
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
  {   // the original entries, four per thread in flight (index loads, then the gathers, then the stores)
    const int64_t q1 = base + cn[ch + 1];
    for (int64_t q0 = base + cn[ch] + threadIdx.x; q0 < q1; q0 += 4 * (int64_t)blockDim.x) {
      int32_t pos[4], src[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t q = q0 + (int64_t)u * blockDim.x;
        pos[u] = q < q1 ? ft.nz_pos[q] : -1;
        src[u] = q < q1 ? ft.nz_csr[q] : 0;
      }
      T v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = pos[u] >= 0 ? (T)J[src[u]] : T(0);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (pos[u] >= 0) F[pos[u]] = v[u];
    }
  }
  __shared__ int64_t s_col[ASM_COLS];   // parent column offsets of the child columns in this chunk
  __syncthreads();
  for (int cc = ft.child_off[f]; cc < ft.child_off[f + 1]; ++cc) {
    const int c = ft.child[cc];
    const int mc = ft.m[c], pc = ft.p[c], nc = mc - pc;
    if (nc == 0) continue;
    const int32_t* ea = ft.ea + ft.ea_off[c];
    // the child's columns that map into [c0, c1): ea is increasing, so the
    // bounds are counts, taken in one parallel pass (no dependent loads)
    int lo = 0, hi = 0;
    for (int b0 = 0; b0 < nc; b0 += blockDim.x) {
      const int t = b0 + threadIdx.x;
      const int e = t < nc ? ea[t] : INT_MAX;
      lo += __syncthreads_count(e < c0);
      hi += __syncthreads_count(e < c1);
    }
    if (hi == lo) continue;   // (uniform)
    if (threadIdx.x < hi - lo) s_col[threadIdx.x] = (int64_t)ea[lo + threadIdx.x] * m;
    __syncthreads();
    const T* C = pool + ft.off[c] + pc + (int64_t)pc * mc;   // the child's contribution block
    // threads as (row, column group): R rows per pass, G groups of the (at
    // most ASM_COLS) child columns that map into this chunk; four columns at
    // a time per thread, all loads before the stores
    const int R = min(nc, (int)blockDim.x), G = blockDim.x / R;
    const int g = threadIdx.x / R;
    if (g < G)
      for (int r = threadIdx.x % R; r < nc; r += R) {
        const int er = ea[r];
        const T* Cr = C + r;
        for (int k0 = lo + g; k0 < hi; k0 += 4 * G) {
          T cv[4], fv[4];
          int64_t fo[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int k = k0 + u * G;
            if (k < hi) {
              fo[u] = er + s_col[k - lo];
              cv[u] = Cr[(int64_t)k * mc];
              fv[u] = F[fo[u]];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (k0 + u * G < hi) F[fo[u]] = fv[u] + cv[u];
        }
      }
    __syncthreads();
  }
}

constexpr int PANEL_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(PANEL_THREADS) panel_kernel(FT ft, const int32_t* work, int k, T* pool,
                                                              int32_t* piv, int32_t* stats, T thresh) {
  const int f = work[WORK_STRIDE * blockIdx.x];
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


namespace cg = cooperative_groups;

// Barrier and shared-memory addressing of a panel group: one CTA (CLN = 1) or
// a thread-block cluster of CLN CTAs with distributed shared memory.
template <int CLN>
struct Group {
  cg::cluster_group c;
  __device__ Group() : c(cg::this_cluster()) {}
  __device__ int rank() const { return (int)c.block_rank(); }
  __device__ void sync() { c.sync(); }
  template <class P>
  __device__ P* map(P* ptr, int r) {
    return c.map_shared_rank(ptr, r);
  }
};
template <>
struct Group<1> {
  __device__ Group() {}
  __device__ int rank() const { return 0; }
  __device__ void sync() { __syncthreads(); }
  template <class P>
  __device__ P* map(P* ptr, int) {
    return ptr;
  }
};

// Panel LU of one front in shared memory: CTA q of the group holds rows
// [k + q*chunk, k + (q+1)*chunk) of the panel columns [k, k + nbe).  Every CTA
// derives the same pivot from the group-wide maxima; row interchanges are
// applied inside the panel here and to the other columns by laswp_kernel.
template <class T, int CLN, int NT>
__global__ void __launch_bounds__(NT)
    panel_smem_kernel(FT ft, const int32_t* work, int k, T* pool, int32_t* piv, int32_t* stats, T thresh) {
  Group<CLN> grp;
  const int q = grp.rank();
  const int f = work[WORK_STRIDE * (blockIdx.x / CLN)];
  const int m = ft.m[f], p = ft.p[f];
  const int nbe = min(PANEL_NB, p - k);
  const int chunk = (m - k + CLN - 1) / CLN;
  const int r0 = k + q * chunk;
  const int nr = max(0, min(chunk, m - r0));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* P = reinterpret_cast<T*>(smem_raw);          // P[c * chunk + i]: panel column c, local row i
  __shared__ T s_cmax, s_best;
  __shared__ int s_brow;
  __shared__ T s_wm[NT / 32], s_wb[NT / 32];
  __shared__ int s_wr[NT / 32];
  __shared__ T s_prow[PANEL_NB], s_rowj[PANEL_NB], s_rowr[PANEL_NB];
  __shared__ int s_r, s_pert, s_pivs[PANEL_NB];
  __shared__ T s_pscale;
  T* F = pool + ft.off[f];
  for (int idx = threadIdx.x; idx < nr * nbe; idx += NT) {
    const int i = idx % nr, c = idx / nr;
    P[c * chunk + i] = F[(int64_t)(k + c) * m + r0 + i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int jj = 0; jj < nbe; ++jj) {
    const int j = k + jj;
    // 1. local column maximum over rows >= j, best fully summed candidate
    T cmax = 0, best = -1;
    int brow = INT_MAX;
    for (int i = threadIdx.x; i < nr; i += NT) {
      const int g = r0 + i;
      if (g < j) continue;
      const T a = fabs(P[jj * chunk + i]);
      cmax = a > cmax ? a : cmax;
      if (g < p && (a > best || (a == best && g < brow))) {
        best = a;
        brow = g;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T om = __shfl_xor_sync(0xffffffffu, cmax, o);
      cmax = om > cmax ? om : cmax;
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int orow = __shfl_xor_sync(0xffffffffu, brow, o);
      if (ob > best || (ob == best && orow < brow)) {
        best = ob;
        brow = orow;
      }
    }
    if (lane == 0) {
      s_wm[wid] = cmax;
      s_wb[wid] = best;
      s_wr[wid] = brow;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      T cm = 0, bb = -1;
      int br = INT_MAX;
      for (int w = 0; w < NT / 32; ++w) {
        cm = s_wm[w] > cm ? s_wm[w] : cm;
        if (s_wb[w] > bb || (s_wb[w] == bb && s_wr[w] < br)) {
          bb = s_wb[w];
          br = s_wr[w];
        }
      }
      s_cmax = cm;
      s_best = bb;
      s_brow = br;
    }
    grp.sync();
    // 2. the same decision in every CTA: lanes of warp 0 gather the CTAs'
    //    maxima (in parallel through DSMEM) and reduce them in a fixed order
    const int qj = (j - k) / chunk, lj = j - k - qj * chunk;
    if (wid == 0) {
      T cm = 0, bb = -1, diag = 0;
      int br = INT_MAX;
      if (lane < CLN) {
        cm = *grp.map(&s_cmax, lane);
        bb = *grp.map(&s_best, lane);
        br = *grp.map(&s_brow, lane);
      } else if (lane == CLN) {
        diag = fabs(grp.map(P, qj)[jj * chunk + lj]);
      }
      diag = __shfl_sync(0xffffffffu, diag, CLN);
      for (int o = CLN / 2; o > 0; o >>= 1) {
        const T om = __shfl_xor_sync(0xffffffffu, cm, o);
        const T ob = __shfl_xor_sync(0xffffffffu, bb, o);
        const int orr = __shfl_xor_sync(0xffffffffu, br, o);
        if (lane < CLN) {
          cm = om > cm ? om : cm;
          if (ob > bb || (ob == bb && orr < br)) {
            bb = ob;
            br = orr;
          }
        }
      }
      if (lane == 0) {
        int r, pert = 0;
        if (diag > 0 && diag >= thresh * cm) {
          r = j;
        } else if (bb > 0) {
          r = br;
          if (q == 0 && bb < thresh * cm) atomicAdd(&stats[1], 1);
        } else {
          r = j;
          pert = 1;
          if (q == 0) atomicAdd(&stats[0], 1);
        }
        s_r = r;
        s_pert = pert;
        s_pivs[jj] = r;
        s_pscale = cm;
      }
    }
    __syncthreads();
    const int r = s_r;
    const int qr = (r - k) / chunk, lr = r - k - qr * chunk;
    // 3. interchange rows j and r inside the panel (uniform branch: every CTA knows r)
    if (r != j) {
      if (threadIdx.x < nbe && (q == qj || q == qr)) {
        s_rowj[threadIdx.x] = grp.map(P, qj)[threadIdx.x * chunk + lj];
        s_rowr[threadIdx.x] = grp.map(P, qr)[threadIdx.x * chunk + lr];
      }
      grp.sync();
      if (threadIdx.x < nbe) {
        if (q == qj) P[threadIdx.x * chunk + lj] = s_rowr[threadIdx.x];
        if (q == qr) P[threadIdx.x * chunk + lr] = s_rowj[threadIdx.x];
      }
    } else if (s_pert && q == qj && threadIdx.x == 0) {
      const T scale = s_pscale > 0 ? s_pscale : T(1);
      P[jj * chunk + lj] = sqrt(Eps<T>::v) * scale;
    }
    grp.sync();
    // 4. pivot row from its owner, then scale and update the local rows below it
    if (threadIdx.x < nbe) s_prow[threadIdx.x] = grp.map(P, qj)[threadIdx.x * chunk + lj];
    __syncthreads();
    const T inv = T(1) / s_prow[jj];
    for (int i = threadIdx.x; i < nr; i += NT) {
      if (r0 + i <= j) continue;
      const T l = P[jj * chunk + i] * inv;
      P[jj * chunk + i] = l;
      for (int c = jj + 1; c < nbe; ++c) P[c * chunk + i] -= l * s_prow[c];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < nr * nbe; idx += NT) {
    const int i = idx % nr, c = idx / nr;
    F[(int64_t)(k + c) * m + r0 + i] = P[c * chunk + i];
  }
  if (q == 0 && threadIdx.x < nbe) piv[ft.piv_off[f] + k + threadIdx.x] = s_pivs[threadIdx.x];
  grp.sync();   // no CTA leaves while another may still read its shared memory
}

// ---- windowed pivoting ---------------------------------------------------------
// Pivots of a 32-column step are chosen inside the 32 x 32 diagonal block only
// (partial pivoting within the window, a counted perturbation when the window
// has no nonzero candidate).  The diagonal block is factored by one warp; the
// rows below (L21 = A21 U11^{-1}) and the columns to the right
// (U12 = L11^{-1} P A12) then need no cross-CTA reduction.
// ordered bits of |x|: the IEEE bits of a nonnegative float, or the high word
// of a nonnegative double (sign, exponent and 20 leading mantissa bits)
__device__ __forceinline__ uint32_t mag_bits(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }
__device__ __forceinline__ uint32_t mag_bits(double x) {
  return (uint32_t)(__double_as_longlong(x) >> 32) & 0x7FFFFFFFu;
}

// Factor the 32 x 32 diagonal block of front f at pivot index k with partial
// pivoting inside the block (one warp, lane = threadIdx.x & 31).  The block
// lives in shared memory (A[row][col], padded so that a row and a column are
// both conflict-free) and the elimination loop stays rolled: a fully unrolled
// 32-step elimination is too long for the instruction cache.
template <class T>
__device__ void diag_block_lu(const FT& ft, int f, int k, T* pool, int32_t* piv, int32_t* perm, int32_t* stats) {
  __shared__ T A[PANEL_NB][PANEL_NB + 1];
  __shared__ int s_piv[PANEL_NB];
  __shared__ int s_src[PANEL_NB];
  const int m = ft.m[f], p = ft.p[f];
  const int nbe = min(PANEL_NB, p - k);
  const int lane = threadIdx.x & 31;
  T* F = pool + ft.off[f] + (int64_t)k * m + k;
  T v[PANEL_NB];   // all 32 loads in flight together
#pragma unroll
  for (int c = 0; c < PANEL_NB; ++c) v[c] = (lane < nbe && c < nbe) ? F[(int64_t)c * m + lane] : T(0);
  T bmax = 0;   // largest entry of the block, the perturbation scale
#pragma unroll
  for (int c = 0; c < PANEL_NB; ++c) {
    A[lane][c] = v[c];
    bmax = fmax(bmax, fabs(v[c]));
  }
  for (int o = 16; o > 0; o >>= 1) bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
  __syncwarp();
  for (int jj = 0; jj < nbe; ++jj) {
    // pivot search in one warp reduction: the key is the magnitude's leading
    // bits (five low bits dropped) with the lane in the low bits, so the
    // largest magnitude wins and, among equal keys, the lowest lane
    const uint32_t key = (lane >= jj && lane < nbe) ? ((mag_bits(A[lane][jj]) & ~31u) | (31u - lane)) : 0u;
    const uint32_t best = __reduce_max_sync(0xffffffffu, key);
    const bool empty = (best & ~31u) == 0u;   // no nonzero candidate in the window column
    const int r = empty ? jj : (int)(31u - (best & 31u));
    if (r != jj) {   // warp-uniform: lane c exchanges column c of rows jj and r
      const T t1 = A[jj][lane], t2 = A[r][lane];
      A[jj][lane] = t2;
      A[r][lane] = t1;
    }
    if (lane == 0) {
      s_piv[jj] = r;
      if (empty) {
        A[jj][jj] = sqrt(Eps<T>::v) * (bmax > 0 ? bmax : T(1));
        atomicAdd(&stats[0], 1);
      }
    }
    __syncwarp();
    if (lane > jj && lane < nbe) {
      const T l = A[lane][jj] * (T(1) / A[jj][jj]);
      A[lane][jj] = l;
#pragma unroll 8
      for (int c = jj + 1; c < nbe; ++c) A[lane][c] -= l * A[jj][c];
    }
    __syncwarp();
  }
#pragma unroll 8
  for (int c = 0; c < PANEL_NB; ++c)
    if (lane < nbe && c < nbe) F[(int64_t)c * m + lane] = A[lane][c];
  // the block's interchanges composed: new row i of the block holds old row
  // s_src[i] (all interchanges of this pivoting stay inside the block)
  s_src[lane] = lane;
  __syncwarp();
  if (lane == 0)
    for (int jj = 0; jj < nbe; ++jj) {
      const int r = s_piv[jj], t = s_src[jj];
      s_src[jj] = s_src[r];
      s_src[r] = t;
    }
  __syncwarp();
  if (lane < nbe) {
    piv[ft.piv_off[f] + k + lane] = k + s_piv[lane];
    perm[ft.piv_off[f] + k + lane] = k + s_src[lane];
  }
}

// the diagonal blocks of the fronts of one launch (those not factored by the
// previous panel's Schur update)
template <class T>
__global__ void __launch_bounds__(32) diag_lu_kernel(FT ft, const int32_t* work, int k, T* pool, int32_t* piv,
                                                     int32_t* perm, int32_t* stats) {
  diag_block_lu<T>(ft, work[WORK_STRIDE * blockIdx.x], k, pool, piv, perm, stats);
}

// One launch, two kinds of items.  Kind 0 (f, r0): rows [r0, r0 + 256) of the
// panel below the diagonal block: L21 = A21 U11^{-1}.  Kind 1 (f, c0, c_end):
// columns [c0, c0 + 256) outside the panel: the block's row permutation and,
// for columns in [k + nbe, c_end), U12 = L11^{-1} P A12.
template <class T>
__global__ void __launch_bounds__(WINDOW_THREADS) window_kernel(FT ft, const int32_t* work, int k, T* pool,
                                                     const int32_t* perm, int32_t* stats, T thresh) {
  const int32_t* it = work + WORK_STRIDE * blockIdx.x;
  const int f = it[1];
  const int m = ft.m[f], p = ft.p[f];
  const int nbe = min(PANEL_NB, p - k);
  T* F = pool + ft.off[f];
  __shared__ T D[PANEL_NB][PANEL_NB + 1];   // the factored diagonal block (L11 \ U11)
  __shared__ T Dinv[PANEL_NB];              // reciprocals of U11's diagonal
  __shared__ int s_src[PANEL_NB];
  for (int e = threadIdx.x; e < PANEL_NB * PANEL_NB; e += blockDim.x) {
    const int i = e % PANEL_NB, c = e / PANEL_NB;
    D[i][c] = (i < nbe && c < nbe) ? F[(int64_t)(k + c) * m + k + i] : T(0);
  }
  if (threadIdx.x < PANEL_NB)
    Dinv[threadIdx.x] = threadIdx.x < nbe ? T(1) / F[(int64_t)(k + threadIdx.x) * m + k + threadIdx.x] : T(0);
  // the block's composed interchanges (written by its diagonal LU): new row i
  // takes old row s_src[i]
  if (threadIdx.x < PANEL_NB)
    s_src[threadIdx.x] = threadIdx.x < nbe ? perm[ft.piv_off[f] + k + threadIdx.x] - k : threadIdx.x;
  __syncthreads();
  if (it[0] == 0) {
    const int g = it[2] + threadIdx.x;
    const bool live = g < m;
    bool big = false;
    if (live) {
      T x[PANEL_NB];
#pragma unroll
      for (int c = 0; c < PANEL_NB; ++c) x[c] = c < nbe ? F[(int64_t)(k + c) * m + g] : T(0);
#pragma unroll
      for (int c = 0; c < PANEL_NB; ++c) {
        if (c < nbe) {
          x[c] *= Dinv[c];
          big = big || fabs(x[c]) * thresh > T(1);
#pragma unroll
          for (int c2 = c + 1; c2 < PANEL_NB; ++c2) x[c2] -= x[c] * D[c][c2];
        }
      }
#pragma unroll
      for (int c = 0; c < PANEL_NB; ++c)
        if (c < nbe) F[(int64_t)(k + c) * m + g] = x[c];
    }
    // a multiplier above 1/threshold: the window pivot missed the threshold test
    // that pivoting over all fully summed rows would have applied
    if (__syncthreads_or(big) && threadIdx.x == 0) atomicAdd(&stats[1], 1);
  } else {
    const int c = it[2] + threadIdx.x, c_end = it[3];
    if (c >= m || (c >= k && c < k + nbe)) return;
    T* col = F + (int64_t)c * m;
    T x[PANEL_NB];
#pragma unroll
    for (int i = 0; i < PANEL_NB; ++i) x[i] = i < nbe ? col[k + s_src[i]] : T(0);
    if (c >= k + nbe && c < c_end) {
#pragma unroll
      for (int l = 0; l < PANEL_NB - 1; ++l) {
        const T xl = x[l];
#pragma unroll
        for (int i = l + 1; i < PANEL_NB; ++i) x[i] -= D[i][l] * xl;
      }
    }
#pragma unroll
    for (int i = 0; i < PANEL_NB; ++i)
      if (i < nbe) col[k + i] = x[i];
  }
}

// ---- 128-column blocks of large fronts, windowed pivoting (FP32) -----------------
// One CTA factors the block's nb x nb diagonal part (nb = min(128, p - k2)) in
// shared memory, one 32-column window at a time:
//   window  one warp: LU with partial pivoting inside the 32 x 32 window, the
//           rows in registers (no interchanges: rows stay in place, a done
//           mask marks the pivotal ones; a row shifts left by one column per
//           step so that the current column is always register 0, and the
//           pivot row is broadcast by shuffles).
//   perm    the window rows put in pivot order on every block column.
//   inv     U11^{-1} and L11^{-1} of the window (one warp each, by
//           substitution): the diagonal blocks of the block's inverses.
//   panel   L21 = A21 U11^{-1} for the block rows below the window and
//           U12 = L11^{-1} P A12 for the block columns right of it, 4 x 4
//           register tiles.
//   rank    A22 -= L21 U12 for the rest of the block, 4 x 4 register tiles.
// It then completes U^{-1} and L^{-1} of the whole block (off-diagonal 32 x 32
// blocks by distance from the diagonal), stores them in place of the block's
// diagonal part (the solves of these fronts step over whole blocks), and
// writes (I - U^{-1}) and (I - L^{-1}) as hi/lo TF32 operand images, so that
// the tensor-core pipeline
// (C -= A B) turns the block's rows below into L21 = A21 - A21 (I - U^{-1}) and
// its columns to the right into U12 = P A12 - (I - L^{-1}) P A12.
// Item: {f, k2, a_blk, b_blk, nchunks} (image blocks of (I - L^{-1}) and
// (I - U^{-1}); -1 when the front has no rows below the block).  A launch runs
// 4 nn_max threads per CTA (nn = 32 nchunks) with three nn_max x (nn_max + 1)
// matrices in shared memory, so blocks of small fronts share an SM.
constexpr int BLK_MAX_THREADS = 4 * OUTER_NB;

__host__ __device__ constexpr size_t blk_smem_bytes(int nn_max) {
  return 3 * sizeof(float) * (size_t)nn_max * (nn_max + 1);
}

// operand image of a 128 x 128 matrix given by val(r, k) (r: M or N index,
// k: K index), chunks blk .. blk + nch - 1 (layout of tc_split_kernel)
template <class Val>
__device__ void write_operand_image(unsigned char* img, int blk, int nch, Val val) {
  for (int e = threadIdx.x; e < nch * OUTER_NB * (tcp::KC / 4); e += blockDim.x) {
    const int ch = e / (OUTER_NB * (tcp::KC / 4)), rem = e % (OUTER_NB * (tcp::KC / 4));
    const int r = rem % OUTER_NB, g = rem / OUTER_NB;
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float v = val(r, ch * tcp::KC + 4 * g + j);
      h[j] = tc::to_tf32(v);
      l[j] = tc::to_tf32(v - __uint_as_float(h[j]));
    }
    unsigned char* out = img + (int64_t)(blk + ch) * tcp::CHUNK_BYTES;
    const int o = g * tcp::KCORE_STRIDE + (r >> 3) * tcp::CORE_BYTES + (r & 7) * 16;
    *reinterpret_cast<uint4*>(out + o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(out + tcp::OPERAND_BYTES + o) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// 4 x 4 register tile of sum_{t < K} A(ia[a], ka + t) B(kb + t, jb[b]) over
// row-major shared matrices with leading dimension ld
__device__ __forceinline__ void blk_tile(const float* __restrict__ A, const float* __restrict__ B, int ld,
                                         const int (&ia)[4], int ka, int kb, const int (&jb)[4], int K,
                                         float (&acc)[4][4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 4
  for (int t = 0; t < K; ++t) {
    float x[4], y[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = A[ia[a] * ld + ka + t];
#pragma unroll
    for (int b = 0; b < 4; ++b) y[b] = B[(kb + t) * ld + jb[b]];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += x[a] * y[b];
  }
}

// hardware reciprocal (about 1 ulp); the multipliers of the FP32 window LU,
// whose rounding the FP64 refinement absorbs
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// One warp: LU with partial pivoting inside the w x w window P (row-major,
// leading dimension ld).  Lane r keeps row r in registers, shifted left by
// one column per step so that x[0] is always the current column.  At step jj
// the candidates are the rows not pivotal yet; the pivot row stores its
// registers (U(jj, jj + c) = x[c]) into Ub[jj], every lane reads them back as
// a broadcast, and the other candidates are eliminated (multiplier into
// Lb[row][jj]).  Rows stay in place; the caller writes the window in pivot
// order: row s = original row s_order[s], its multipliers left of column s and
// its U part from column s on.
__device__ void window_lu(float* P, int ld, int w, float (*Ub)[PANEL_NB + 4], float (*Lb)[PANEL_NB + 1],
                          int* s_order, int32_t* stats) {
  const int lane = threadIdx.x & 31;
  float x[PANEL_NB];
#pragma unroll
  for (int c = 0; c < PANEL_NB; ++c) x[c] = (lane < w && c < w) ? P[lane * ld + c] : 0.f;
  float bmax = 0.f;   // largest entry of the window, the perturbation scale
#pragma unroll
  for (int c = 0; c < PANEL_NB; ++c) bmax = fmaxf(bmax, fabsf(x[c]));
  for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
  uint32_t done = 0;
  int perturbed = 0;
  for (int jj = 0; jj < w; ++jj) {
    const bool cand = lane < w && !((done >> lane) & 1u);
    const uint32_t key = cand ? ((mag_bits(x[0]) & ~31u) | (31u - lane)) : 0u;
    const uint32_t best = __reduce_max_sync(0xffffffffu, key);
    const bool empty = (best & ~31u) == 0u;   // no nonzero candidate: perturbed pivot
    const int pr = empty ? __ffs(~done) - 1 : (int)(31u - (best & 31u));
    perturbed += empty;
    if (lane == pr) {
      if (empty) x[0] = sqrtf(FLT_EPSILON) * (bmax > 0.f ? bmax : 1.f);
      float4* dst = reinterpret_cast<float4*>(Ub[jj]);
#pragma unroll
      for (int q = 0; q < PANEL_NB / 4; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    }
    s_order[jj] = pr;   // (every lane, the same value)
    __syncwarp();
    float u[PANEL_NB];
    const float4* src = reinterpret_cast<const float4*>(Ub[jj]);
#pragma unroll
    for (int q = 0; q < PANEL_NB / 4; ++q) {
      const float4 t = src[q];
      u[4 * q] = t.x;
      u[4 * q + 1] = t.y;
      u[4 * q + 2] = t.z;
      u[4 * q + 3] = t.w;
    }
    const bool elim = cand && lane != pr;
    // (rows that are pivotal shift too: their U part is in Ub already)
    const float l = elim ? x[0] * rcp_approx(u[0]) : 0.f;
    Lb[lane][jj] = l;   // (0 for the other rows: never read)
#pragma unroll
    for (int c = 1; c < PANEL_NB; ++c) x[c - 1] = x[c] - l * u[c];
    x[PANEL_NB - 1] = 0.f;   // (beyond the window)
    done |= 1u << pr;
  }
  if (perturbed && lane == 0) atomicAdd(&stats[0], perturbed);
}

// U^{-1} into V and L^{-1} into W for the 32 x 32 diagonal block at o: the
// 8 x 8 diagonal blocks by substitution (one thread per column, registers),
// then the off-diagonal 8 x 8 blocks by distance from the diagonal (as for the
// 32 x 32 blocks below); the other triangles are zeroed (the products read
// whole blocks).  Every thread of the CTA takes part (blockDim >= 128).
__device__ void diag_inverse(const float* __restrict__ D, float* __restrict__ V, float* __restrict__ W, int ld,
                             int o) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int e = tid; e < PANEL_NB * PANEL_NB; e += nthr) {
    const int i = e & 31, j = e >> 5;
    if (i > j) V[(o + i) * ld + o + j] = 0.f;
    if (i < j) W[(o + i) * ld + o + j] = 0.f;
  }
  if (tid < 64) {
    const int task = tid >> 3, j = tid & 7, ob = o + 8 * (task & 3);
    float y[8];
    if (task < 4) {   // column j of U_bb^{-1}
#pragma unroll
      for (int i = 7; i >= 0; --i) {
        float s0 = i == j ? 1.f : 0.f;
#pragma unroll
        for (int t = i + 1; t < 8; ++t) s0 -= D[(ob + i) * ld + ob + t] * y[t];
        y[i] = i <= j ? s0 * rcp_approx(D[(ob + i) * ld + ob + i]) : 0.f;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i <= j) V[(ob + i) * ld + ob + j] = y[i];
    } else {          // column j of L_bb^{-1}
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float s0 = i == j ? 1.f : 0.f;
#pragma unroll
        for (int t = 0; t < i; ++t) s0 -= D[(ob + i) * ld + ob + t] * y[t];
        y[i] = i >= j ? s0 : 0.f;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i >= j) W[(ob + i) * ld + ob + j] = y[i];
    }
  }
  __syncthreads();
  for (int d = 1; d < 4; ++d) {
    const int nblk = 4 - d, nt = 2 * nblk * 64;   // outputs of this distance (<= 384)
    float r[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {   // sums, straight into the target blocks
      const int e = tid + q * nthr;
      if (e < nt) {
        const int task = e >> 6, i = e & 7, j = (e >> 3) & 7;
        const bool up = task < nblk;
        const int I = up ? task : task - nblk, J = I + d;
        float s0 = 0.f;
        if (up) {
          for (int t = 8 * (I + 1); t < 8 * (J + 1); ++t) s0 += D[(o + 8 * I + i) * ld + o + t] * V[(o + t) * ld + o + 8 * J + j];
          V[(o + 8 * I + i) * ld + o + 8 * J + j] = s0;
        } else {
          for (int t = 8 * I; t < 8 * J; ++t) s0 += D[(o + 8 * J + i) * ld + o + t] * W[(o + t) * ld + o + 8 * I + j];
          W[(o + 8 * J + i) * ld + o + 8 * I + j] = s0;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 3; ++q) {   // products with the diagonal inverses
      const int e = tid + q * nthr;
      if (e < nt) {
        const int task = e >> 6, i = e & 7, j = (e >> 3) & 7;
        const bool up = task < nblk;
        const int I = up ? task : task - nblk, J = I + d;
        float s0 = 0.f;
        if (up) {
#pragma unroll
          for (int t = 0; t < 8; ++t) s0 += V[(o + 8 * I + i) * ld + o + 8 * I + t] * V[(o + 8 * I + t) * ld + o + 8 * J + j];
        } else {
#pragma unroll
          for (int t = 0; t < 8; ++t) s0 += W[(o + 8 * J + i) * ld + o + 8 * J + t] * W[(o + 8 * J + t) * ld + o + 8 * I + j];
        }
        r[q] = -s0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int e = tid + q * nthr;
      if (e < nt) {
        const int task = e >> 6, i = e & 7, j = (e >> 3) & 7;
        const bool up = task < nblk;
        const int I = up ? task : task - nblk, J = I + d;
        if (up) V[(o + 8 * I + i) * ld + o + 8 * J + j] = r[q];
        else W[(o + 8 * J + i) * ld + o + 8 * I + j] = r[q];
      }
    }
    __syncthreads();
  }
}

// off-diagonal 32 x 32 blocks of V = U^{-1} and W = L^{-1} (diagonal blocks
// in place), by distance d = J - I from the diagonal, all of one distance at
// once (they need only blocks nearer the diagonal):
//   U^{-1}_IJ = -U_II^{-1} sum_{K=I+1..J} U_IK U^{-1}_KJ
//   L^{-1}_JI = -L_JJ^{-1} sum_{K=I..J-1} L_JK L^{-1}_KI
// The sums go straight into the target block (no task of this distance reads
// it); the products with the diagonal inverses are held in registers until
// every tile has read its sums.  64 tiles of 4 x 4 per block, at most
// 2 (nbk - 1) blocks: one tile per thread.
__device__ void offdiag_inverses(const float* __restrict__ D, float* __restrict__ V, float* __restrict__ W, int ld,
                                 int nbk) {
  for (int d = 1; d < nbk; ++d) {
    const int nt = 2 * (nbk - d) * 64;
    const int tile = threadIdx.x;
    const bool act = tile < nt;
    const int task = tile >> 6, ti = tile & 7, tj = (tile >> 3) & 7;
    const bool up = task < nbk - d;
    const int I = up ? task : task - (nbk - d), J = I + d;
    float* X = up ? V : W;
    int ia[4], jb[4];
    float acc[4][4];
    if (act) {
      const int r0 = up ? 32 * I : 32 * J, c0 = up ? 32 * J : 32 * I;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ia[a] = r0 + ti + 8 * a;
        jb[a] = c0 + tj + 8 * a;
      }
      if (up) blk_tile(D, V, ld, ia, 32 * (I + 1), 32 * (I + 1), jb, 32 * d, acc);
      else blk_tile(D, W, ld, ia, 32 * I, 32 * I, jb, 32 * d, acc);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) X[ia[a] * ld + jb[b]] = acc[a][b];
    }
    __syncthreads();
    if (act) {
      const int dg = up ? 32 * I : 32 * J;   // -U_II^{-1} sums(I, J) / -L_JJ^{-1} sums(J, I)
      blk_tile(X, X, ld, ia, dg, dg, jb, 32, acc);
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) X[ia[a] * ld + jb[b]] = -acc[a][b];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(BLK_MAX_THREADS, 1) block_lu_kernel(FT ft, const int32_t* work, float* pool,
                                                                      int32_t* perm, int32_t* stats, float thresh,
                                                                      unsigned char* img, int nn_max) {
  extern __shared__ __align__(16) float blk_sm[];
  const int ld = nn_max + 1;
  float* __restrict__ D = blk_sm;
  float* __restrict__ V = blk_sm + nn_max * ld;
  float* __restrict__ W = V + nn_max * ld;
  __shared__ int s_order[PANEL_NB];
  __shared__ __align__(16) float s_ub[PANEL_NB][PANEL_NB + 4];   // window pivot rows (16-byte rows)
  __shared__ float s_lb[PANEL_NB][PANEL_NB + 1];                 // window multipliers by original row
  const int32_t* it = work + WORK_STRIDE * blockIdx.x;
  const int f = it[0], k2 = it[1], a_blk = it[2], b_blk = it[3], nch = it[4];
  const int m = ft.m[f], p = ft.p[f];
  const int nb = min(OUTER_NB, p - k2), nn = 32 * nch;   // nb <= nn <= nn_max
  float* F = pool + ft.off[f] + (int64_t)k2 * m + k2;
  const int tid = threadIdx.x, warp = tid >> 5, nthr = blockDim.x;
  // the nn x nn block, identity outside nb x nb; column j of the front is
  // contiguous, so consecutive threads take consecutive rows (8 loads in flight)
  const int jstep = nthr / nn, li = tid % nn;   // threads at or beyond jstep nn take no part
  for (int jb = tid < jstep * nn ? tid / nn : nn; jb < nn; jb += 8 * jstep) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = jb + q * jstep;
      v[q] = (li < nb && j < nb) ? F[(int64_t)j * m + li] : (li == j ? 1.f : 0.f);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = jb + q * jstep;
      if (j < nn) D[li * ld + j] = v[q];
    }
  }
  __syncthreads();
  const int pc = tid & 127, pr0 = tid >> 7, prs = nthr >> 7;   // (row, column) pattern of the row moves
  bool big = false;
  for (int j0 = 0; j0 < nb; j0 += PANEL_NB) {
    const int w = min(PANEL_NB, nb - j0), r0 = j0 + w, cr = nb - r0;
    if (warp == 0) window_lu(D + j0 * ld + j0, ld, w, s_ub, s_lb, s_order, stats);
    __syncthreads();
    for (int e = tid; e < w * PANEL_NB; e += nthr) {   // the window in pivot order
      const int s = e >> 5, c = e & 31;
      if (c < w) D[(j0 + s) * ld + j0 + c] = c < s ? s_lb[s_order[s]][c] : s_ub[s][c - s];
    }
    if (nb == w) __syncthreads();   // (uniform; otherwise the row moves below end with one)
    // the composed permutation (new row s of the window holds old row
    // s_order[s]; windowed pivoting keeps no interchange sequence), and the
    // window rows in pivot order on the other block columns (rows j0.. of V
    // hold them meanwhile: V's diagonal block there is written only afterwards)
    if (tid < w) perm[ft.piv_off[f] + k2 + j0 + tid] = k2 + j0 + s_order[tid];
    if (nb > w) {   // (uniform)
      const bool col = pc < nb && (pc < j0 || pc >= j0 + w);
      if (col)
        for (int s = pr0; s < w; s += prs) V[(j0 + s) * ld + pc] = D[(j0 + s_order[s]) * ld + pc];
      __syncthreads();
      if (col)
        for (int s = pr0; s < w; s += prs) D[(j0 + s) * ld + pc] = V[(j0 + s) * ld + pc];
      __syncthreads();
    }
    diag_inverse(D, V, W, ld, j0);
    __syncthreads();
    if (cr > 0) {
      // L21 = A21 U11^{-1} (rows r0.., window columns) and U12 = L11^{-1} P A12
      // (window rows, columns r0..): one 4 x 4 tile per thread, written after
      // every tile has read its operands
      const int RT = (cr + 3) >> 2, nl = RT * 8;
      const int t = tid;
      const bool act = t < 2 * nl;
      const bool lower = t < nl;
      int ia[4], jb[4];
      float acc[4][4];
      if (act) {
        const int u = lower ? t : t - nl, ta = lower ? u % RT : u & 7, tb = lower ? u / RT : u >> 3;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          ia[a] = lower ? r0 + min(ta + RT * a, cr - 1) : j0 + ta + 8 * a;
          jb[a] = lower ? j0 + tb + 8 * a : r0 + min(tb + RT * a, cr - 1);
        }
        if (lower) blk_tile(D, V, ld, ia, j0, j0, jb, w, acc);
        else blk_tile(W, D, ld, ia, j0, j0, jb, w, acc);
      }
      __syncthreads();
      if (act) {
        const int u = lower ? t : t - nl, ta = lower ? u % RT : u & 7, tb = lower ? u / RT : u >> 3;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const bool ok = lower ? (ta + RT * a < cr && tb + 8 * b < w) : (ta + 8 * a < w && tb + RT * b < cr);
            if (ok) {
              D[ia[a] * ld + jb[b]] = acc[a][b];
              // a multiplier above 1/threshold: the window pivot missed the
              // threshold test that pivoting over all fully summed rows would apply
              big = big || (lower && fabsf(acc[a][b]) * thresh > 1.f);
            }
          }
      }
      __syncthreads();
      // rank-w update of the rest of the block: rows and columns r0 .. nb - 1
      for (int q = tid; q < RT * RT; q += nthr) {
        const int ti = q % RT, tj = q / RT;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          ia[a] = r0 + min(ti + RT * a, cr - 1);
          jb[a] = r0 + min(tj + RT * a, cr - 1);
        }
        blk_tile(D, D, ld, ia, j0, j0, jb, w, acc);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (ti + RT * a < cr && tj + RT * b < cr) D[ia[a] * ld + jb[b]] -= acc[a][b];
      }
      __syncthreads();
    }
  }
  if (__syncthreads_or(big) && tid == 0) atomicAdd(&stats[1], 1);
  offdiag_inverses(D, V, W, ld, nch);
  // the block's diagonal part is kept inverted (the solves step over whole
  // blocks): L^{-1} below the diagonal (unit diagonal implied), U^{-1} on and
  // above it
  if (li < nb && tid < jstep * nn)
    for (int j = tid / nn; j < nb; j += jstep) F[(int64_t)j * m + li] = li > j ? W[li * ld + j] : V[li * ld + j];
  if (a_blk < 0) return;   // (uniform) no rows below the block: no operand images
  // B operand (K x N: row k, column n of I - U^{-1}), A operand (M x K: row i,
  // column k of I - L^{-1}); zero outside nn x nn and outside the triangles
  write_operand_image(img, b_blk, nch, [&](int n, int k) {
    return (n < nn && k <= n) ? (k == n ? 1.f : 0.f) - V[k * ld + n] : 0.f;
  });
  write_operand_image(img, a_blk, nch, [&](int i, int k) { return (i < nn && i > k) ? -W[i * ld + k] : 0.f; });
}

// the block's row permutation (new row i of the block holds old row s_src[i],
// which stays inside its 32-row window) on the front's columns outside the
// block; item {f, k2, c0}: columns c0 .. c0 + 255.  Threads are rows of the
// block (coalesced within a column), two column groups per CTA, eight columns
// per thread in flight: all reads of a batch before its writes.
constexpr int PERM_THREADS = 2 * OUTER_NB;
__global__ void __launch_bounds__(PERM_THREADS) block_perm_kernel(FT ft, const int32_t* work, float* pool,
                                                                  const int32_t* perm) {
  const int32_t* it = work + WORK_STRIDE * blockIdx.x;
  const int f = it[0], k2 = it[1], c0 = it[2];
  const int m = ft.m[f], p = ft.p[f];
  const int nb = min(OUTER_NB, p - k2);
  const int i = threadIdx.x & (OUTER_NB - 1), g = threadIdx.x >> 7;
  const int src = i < nb ? perm[ft.piv_off[f] + k2 + i] : 0;   // absolute row
  float* F = pool + ft.off[f];
  const int c_end = min(c0 + 256, m);
  for (int cb = c0; cb < c_end; cb += 16) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = cb + 2 * u + g;
      const bool ok = i < nb && c < c_end && (c < k2 || c >= k2 + nb);
      v[u] = ok ? F[(int64_t)c * m + src] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = cb + 2 * u + g;
      if (i < nb && c < c_end && (c < k2 || c >= k2 + nb)) F[(int64_t)c * m + k2 + i] = v[u];
    }
  }
}

// row interchanges of a cluster panel applied to the columns outside it
template <class T>
__global__ void laswp_kernel(FT ft, const int32_t* work, int k, T* pool, const int32_t* piv) {
  const int32_t* it = work + WORK_STRIDE * blockIdx.x;
  const int f = it[0], c = it[1] + threadIdx.x;
  const int m = ft.m[f], p = ft.p[f];
  const int nbe = min(PANEL_NB, p - k);
  if (c >= m || (c >= k && c < k + nbe)) return;
  T* col = pool + ft.off[f] + (int64_t)c * m;
  const int32_t* pv = piv + ft.piv_off[f];
  for (int jj = 0; jj < nbe; ++jj) {
    const int j = k + jj, r = pv[j];
    if (r != j) {
      const T a = col[j];
      col[j] = col[r];
      col[r] = a;
    }
  }
}

// U12 rows [k, k + nbe) of columns [c0, min(c0 + TRSM_COLS, c_end)) := L11^{-1} A12
template <class T>
__global__ void trsm_kernel(FT ft, const int32_t* work, T* pool) {
  const int32_t* it = work + WORK_STRIDE * blockIdx.x;
  const int f = it[0], c0 = it[1], c_end = it[2], k = it[3];
  const int m = ft.m[f], p = ft.p[f];
  const int nbe = min(PANEL_NB, p - k);
  const int c1 = min(c0 + TRSM_COLS, c_end);
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

// F[rb.., cb..] -= F[rows, k_begin : k_begin + k_len] * F[k_begin : k_begin + k_len, cols]
// for one 64 x 64 tile clipped to rows < r_end and columns < c_end (SIMT).
// With item[7] set (windowed pivoting) the tile holds the next panel's
// diagonal block at (rb, rb): once the tile is updated, one warp factors it.
template <class T>
__global__ void __launch_bounds__(256) gemm_kernel(FT ft, const int32_t* work, T* pool, int32_t* piv,
                                                   int32_t* perm, int32_t* stats) {
  const int32_t* it = work + WORK_STRIDE * blockIdx.x;
  const int f = it[0], rb = it[1], cb = it[2], r_end = it[3], c_end = it[4], kb = it[5], kl = it[6];
  const int m = ft.m[f];
  T* F = pool + ft.off[f];
  __shared__ T As[PANEL_NB][GEMM_TILE + 1];   // [kk][row]
  __shared__ T Bs[PANEL_NB][GEMM_TILE + 1];   // [kk][col]
  const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;
  constexpr int LD = PANEL_NB * GEMM_TILE / 256;   // operand entries per thread and chunk = 8
  T acc[4][4] = {};
  for (int k0 = 0; k0 < kl; k0 += PANEL_NB) {
    const int kn = min(PANEL_NB, kl - k0);
    // A: rows vary fastest; B: k varies fastest (each column is contiguous in k)
    T ra[LD], rbv[LD];
#pragma unroll
    for (int t = 0; t < LD; ++t) {
      const int q = threadIdx.x + 256 * t;
      const int r = q % GEMM_TILE, kk = q / GEMM_TILE;
      const int kk2 = q % PANEL_NB, c2 = q / PANEL_NB;
      ra[t] = (kk < kn && rb + r < r_end) ? F[(int64_t)(kb + k0 + kk) * m + rb + r] : T(0);
      rbv[t] = (kk2 < kn && cb + c2 < c_end) ? F[(int64_t)(cb + c2) * m + kb + k0 + kk2] : T(0);
    }
#pragma unroll
    for (int t = 0; t < LD; ++t) {
      const int q = threadIdx.x + 256 * t;
      As[q / GEMM_TILE][q % GEMM_TILE] = ra[t];
      Bs[q % PANEL_NB][q / PANEL_NB] = rbv[t];
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kn; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][tr + 16 * u];
        b[u] = Bs[kk][tc + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int c = cb + tc + 16 * v;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = rb + tr + 16 * u;
      if (c < c_end && r < r_end) F[(int64_t)c * m + r] -= acc[u][v];
    }
  }
  if (it[7]) {
    __syncthreads();   // the whole tile is updated (block-scope visibility of its stores)
    if (threadIdx.x < 32) diag_block_lu<T>(ft, f, rb, pool, piv, perm, stats);
  }
}

// ---- solves -----------------------------------------------------------------------
// After the numeric factorisation, every 32 x 32 diagonal block of a front is
// replaced in place by the inverses of its unit-lower part L11 (strictly lower
// entries) and of its upper part U11 (upper entries, diagonal included), and
// the row interchanges of each front are composed into one permutation.
// A solve then walks the tree level by level:
//   forward, per level:  one CTA per front gathers the children's update
//     vectors, permutes the pivot rows and runs the triangular chain over the
//     pivot rows (x_blk = L11^{-1} w_blk, then the rows below the block); a
//     second, multi-CTA launch forms L21 x for the non-pivot rows in column
//     slices (partial sums per slice, summed in order by the parent);
//   backward, per level: a multi-CTA launch forms U12 x2 in column slices,
//     then one CTA per front subtracts the slices and runs the chain upwards
//     (x_blk = U11^{-1} v_blk, then the rows above the block).
// The chains are latency-bound (one barrier and one memory round trip per
// 32 rows); the slice launches carry the bandwidth-bound part of the solve.

// in-place inversion of the diagonal blocks; one warp per (front, block)
constexpr int INV_WARPS = 4;
template <class T>
__global__ void __launch_bounds__(INV_WARPS * 32) diag_inv_kernel(FT ft, const int32_t* items, int n, T* pool) {
  __shared__ T B[INV_WARPS][32][33];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int it = blockIdx.x * INV_WARPS + wid;
  if (it >= n) return;   // warp-uniform; the kernel uses no block barrier
  const int f = items[2 * it], jb = items[2 * it + 1];
  const int m = ft.m[f], p = ft.p[f];
  const int nb = min(32, p - jb);
  T* F = pool + ft.off[f] + (int64_t)jb * m + jb;
  T(*Bw)[33] = B[wid];
#pragma unroll 4
  for (int j = 0; j < 32; ++j) Bw[lane][j] = (lane < nb && j < nb) ? F[(int64_t)j * m + lane] : T(lane == j ? 1 : 0);
  __syncwarp();
  // column `lane` of L11^{-1} (unit lower): X[i] = -sum_{k<i} L[i][k] X[k] for i > lane
  T X[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) X[i] = i == lane ? T(1) : T(0);
#pragma unroll
  for (int i = 1; i < 32; ++i) {
    T s = 0;
#pragma unroll
    for (int k = 0; k < i; ++k) s += Bw[i][k] * X[k];
    if (i > lane) X[i] = -s;
  }
  // column `lane` of U11^{-1}: Y[i] = (delta_i,lane - sum_{k>i} U[i][k] Y[k]) / U[i][i] for i <= lane
  T Y[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) Y[i] = 0;
#pragma unroll
  for (int i = 31; i >= 0; --i) {
    T s = i == lane ? T(1) : T(0);
#pragma unroll
    for (int k = i + 1; k < 32; ++k) s -= Bw[i][k] * Y[k];
    if (i <= lane) Y[i] = s / Bw[i][i];
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) Bw[i][lane] = i > lane ? X[i] : Y[i];
  __syncwarp();
  if (lane < nb)
    for (int j = 0; j < nb; ++j) F[(int64_t)j * m + lane] = Bw[lane][j];
}

// Composition of a front's row interchanges (threshold pivoting): new pivot
// row i holds old row perm[i].  (With windowed pivoting each diagonal LU
// writes its block's composition itself.)
__global__ void perm_kernel(FT ft, const int32_t* piv, int32_t* perm) {
  extern __shared__ int32_t s_perm[];
  const int f = blockIdx.x;
  const int p = ft.p[f];
  const int32_t* pv = piv + ft.piv_off[f];
  int32_t* sp = s_perm;
  int32_t* sv = s_perm + p;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    sp[i] = i;
    sv[i] = pv[i];
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int j = 0; j < p; ++j) {
      const int r = sv[j];
      const int32_t t = sp[j];
      sp[j] = sp[r];
      sp[r] = t;
    }
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += blockDim.x) perm[ft.piv_off[f] + i] = sp[i];
}

constexpr int SOLVE_THREADS = 1024;
constexpr int SOLVE_SMEM_MAX = 160 * 1024;
// chain CTAs: up to 1024 threads for FP32 fronts, 512 for FP64 (two 32-entry
// register rows per thread)
template <class T>
constexpr int solve_threads_max() {
  return sizeof(T) == 8 ? 512 : 1024;
}
constexpr int GEMV_THREADS = SOLVE_ROWS;   // one row per thread, 32 rows per warp

// Every solve kernel handles NR right-hand sides at once (NR = 1 for the
// refinement sweeps, 2 for the border columns Y = A^{-1} B): vector r of b
// and x starts at r * ldv (doubles), of yv at r * ldv (T) and of the
// workspace at r * vstride (T); the factor entries are loaded once for all NR.

// slice partial sums of the non-pivot rows (FWD: L21 x) or of the pivot rows
// (!FWD: U12 x2) for one item (f, r0, s)
template <class T, bool FWD, int NR>
__global__ void __launch_bounds__(GEMV_THREADS) solve_gemv_kernel(FT ft, const int32_t* items, const T* __restrict__ pool,
                                                                  const T* __restrict__ yv,
                                                                  const double* __restrict__ x, T* vec, int64_t ldv,
                                                                  int64_t vstride) {
  __shared__ T xs[NR][SOLVE_SLICE];
  const int32_t* it = items + 4 * blockIdx.x;
  const int f = it[0], r0 = it[1], sl = it[2];
  const int m = ft.m[f], p = ft.p[f], first = ft.first[f];
  const int row_lo = FWD ? p : 0, row_hi = FWD ? m : p;
  const int col_lo = FWD ? 0 : p, col_hi = FWD ? p : m;
  const int c0 = col_lo + sl * SOLVE_SLICE, c1 = min(col_hi, c0 + SOLVE_SLICE);
  const int nrows = row_hi - row_lo;
  if (FWD) {
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x)
#pragma unroll
      for (int r = 0; r < NR; ++r) xs[r][c - c0] = yv[r * ldv + first + c];
  } else {
    const int32_t* idx = ft.idx + ft.idx_off[f];
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x)
#pragma unroll
      for (int r = 0; r < NR; ++r) xs[r][c - c0] = (T)x[r * ldv + idx[c]];
  }
  __syncthreads();
  const int i = row_lo + r0 + threadIdx.x;
  if (i >= row_hi) return;
  const T* col = pool + ft.off[f] + (int64_t)c0 * m + i;
  T a[NR][4];
#pragma unroll
  for (int r = 0; r < NR; ++r) a[r][0] = a[r][1] = a[r][2] = a[r][3] = T(0);
  int c = 0;
  const int nc = c1 - c0;
  for (; c + 32 <= nc; c += 32) {
    T v[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) v[u] = __ldg(col + (int64_t)(c + u) * m);
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int u = 0; u < 32; ++u) a[r][u & 3] += v[u] * xs[r][c + u];
  }
  for (; c < nc; ++c) {
    const T v = __ldg(col + (int64_t)c * m);
#pragma unroll
    for (int r = 0; r < NR; ++r) a[r][0] += v * xs[r][c];
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    T* part = vec + r * vstride + ft.vec_off[f] + m;
    part[(int64_t)sl * nrows + (i - row_lo)] = (a[r][0] + a[r][1]) + (a[r][2] + a[r][3]);
  }
}

// One 128-row step of a chain over a front whose 128 x 128 diagonal blocks
// are stored inverted (block-LU fronts).  FWD: x_b = L_bb^{-1} w_b (unit lower
// part of the stored inverse; x_b -> yv), then w_i -= L(i, b) x_b for the pivot
// rows below the block.  !FWD: x_b = U_bb^{-1} v_b (upper part with the
// diagonal; x_b -> xo, FP64), then v_i -= U(i, b) x_b for the pivot rows above
// it.  The block product is split over all threads (row of the block x 16-column
// group, partial sums in red = NR x 1024 shared entries), the row updates take
// one row per thread with 32 loads in flight.
template <class T, int NR, bool FWD>
__device__ void chain_block128(const T* __restrict__ F, int m, int p, int jb, T* const (&w)[NR], T* red,
                               T* yo, int64_t ldv, double* xo = nullptr) {
  __shared__ T xb[NR][OUTER_NB];
  const int nb = min(OUTER_NB, p - jb), nthr = blockDim.x;
  __syncthreads();   // w of the block final (row updates of the previous step)
  for (int e = threadIdx.x; e < OUTER_NB * 8; e += nthr) {
    const int rr = e & (OUTER_NB - 1), g = e >> 7;   // row of the block, 16-column group
    T a[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) a[r] = T(0);
    if (rr < nb) {
      const T* Dc = F + (int64_t)(jb + 16 * g) * m + jb + rr;
      T d[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = 16 * g + j;
        d[j] = (c < nb && (FWD ? c < rr : c >= rr)) ? Dc[(int64_t)j * m] : T(0);
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = min(16 * g + j, nb - 1);
          a[r] += d[j] * w[r][jb + c];
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) red[r * 1024 + g * OUTER_NB + rr] = a[r];
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < nb; rr += nthr)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      T s = FWD ? w[r][jb + rr] : T(0);   // (unit diagonal of L^{-1})
#pragma unroll
      for (int g = 0; g < 8; ++g) s += red[r * 1024 + g * OUTER_NB + rr];
      xb[r][rr] = s;
      if (FWD) yo[r * ldv + jb + rr] = s;
      else xo[r * ldv + jb + rr] = (double)s;
    }
  __syncthreads();
  const int i0 = FWD ? jb + OUTER_NB : 0, i1 = FWD ? p : jb;
  for (int i = i0 + threadIdx.x; i < i1; i += nthr) {
    const T* col = F + (int64_t)jb * m + i;
    T a[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) a[r] = T(0);
    for (int c0 = 0; c0 < nb; c0 += 32) {
      T v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = c0 + j < nb ? col[(int64_t)(c0 + j) * m] : T(0);
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < 32; ++j) a[r] += v[j] * xb[r][min(c0 + j, nb - 1)];
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) w[r][i] -= a[r];
  }
}

// forward chain of one front: gather, permute, L11^{-1} blocks and the pivot
// rows below them; the non-pivot rows keep the gathered values for the slices
template <class T, int NR>
__global__ void __launch_bounds__(solve_threads_max<T>(), 1) fwd_tri_kernel(FT ft, const int32_t* fronts, const T* __restrict__ pool,
                                                                const int32_t* perm, const double* b, T* vec, T* yv,
                                                                bool in_smem, int64_t ldv, int64_t vstride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T xw[NR][SOLVE_THREADS / 32][32];
  const int f = fronts[blockIdx.x];
  const int m = ft.m[f], p = ft.p[f], first = ft.first[f];
  // vector r: w[r] (m entries) and tmp[r] (p entries)
  T* const wsm = reinterpret_cast<T*>(smem_raw);
  T* w[NR];
  T* tmp[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    w[r] = in_smem ? wsm + (int64_t)r * m : vec + r * vstride + ft.vec_off[f];
    tmp[r] = in_smem ? wsm + (int64_t)NR * m + (int64_t)r * p : yv + r * ldv + first;
  }
  const T* F = pool + ft.off[f];
  for (int i = threadIdx.x; i < m; i += blockDim.x)
#pragma unroll
    for (int r = 0; r < NR; ++r) w[r][i] = i < p ? (T)b[r * ldv + first + i] : T(0);
  __syncthreads();
  for (int cc = ft.child_off[f]; cc < ft.child_off[f + 1]; ++cc) {
    const int c = ft.child[cc];
    const int mc = ft.m[c], pc = ft.p[c], nc = mc - pc;
    const int32_t* ea = ft.ea + ft.ea_off[c];
    const int ns = (pc + SOLVE_SLICE - 1) / SOLVE_SLICE;
    for (int rr = threadIdx.x; rr < nc; rr += blockDim.x) {
      const int e = ea[rr];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const T* wc = vec + r * vstride + ft.vec_off[c];
        const T* pc_part = wc + mc;
        T v = wc[pc + rr];
        for (int s2 = 0; s2 < ns; ++s2) v -= pc_part[(int64_t)s2 * nc + rr];
        w[r][e] += v;
      }
    }
    __syncthreads();
  }
  const int32_t* pm = perm + ft.piv_off[f];
  for (int i = threadIdx.x; i < p; i += blockDim.x)
#pragma unroll
    for (int r = 0; r < NR; ++r) tmp[r][i] = w[r][pm[i]];
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += blockDim.x)
#pragma unroll
    for (int r = 0; r < NR; ++r) w[r][i] = tmp[r][i];
  if (ft.blk && ft.blk[f] == 2) {   // the chain runs on many CTAs (chain_multi_kernel): w's pivot part -> yv
    for (int i = threadIdx.x; i < m; i += blockDim.x)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (i < p) yv[r * ldv + first + i] = w[r][i];
        else if (in_smem) vec[r * vstride + ft.vec_off[f] + i] = w[r][i];
      }
    return;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool b128 = ft.blk && ft.blk[f];   // (block-LU fronts: 128-row blocks stored inverted)
  for (int jb = 0; jb < p; jb += b128 ? OUTER_NB : 32) {
    if (b128) {
      chain_block128<T, NR, true>(F, m, p, jb, w, xw[0][0], yv + first, ldv);
      continue;
    }
    const int nb = min(32, p - jb);
    // row `lane` of L11^{-1} (strictly lower part), loaded before the barrier
    T d[32];
    const T* Db = F + (int64_t)jb * m + jb + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) d[j] = (j < lane && lane < nb) ? Db[(int64_t)j * m] : T(0);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const T wl = lane < nb ? w[r][jb + lane] : T(0);
      T xl = wl;
#pragma unroll
      for (int j = 0; j < 32; ++j) xl += d[j] * __shfl_sync(0xffffffffu, wl, j);
      xw[r][wid][lane] = xl;
      if (wid == 0 && lane < nb) yv[r * ldv + first + jb + lane] = xl;
    }
    __syncwarp();
    if (nb == 32) {
      for (int i = jb + 32 + threadIdx.x; i < p; i += blockDim.x) {
        const T* col = F + (int64_t)jb * m + i;
        T v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = col[(int64_t)j * m];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const T* xr = xw[r][wid];
          T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            a0 += v[j] * xr[j];
            a1 += v[j + 1] * xr[j + 1];
            a2 += v[j + 2] * xr[j + 2];
            a3 += v[j + 3] * xr[j + 3];
          }
          w[r][i] -= (a0 + a1) + (a2 + a3);
        }
      }
    }
    // (a short last block has no pivot rows below it)
  }
  if ((ft.fused[f] & 1) && m > p) {   // (uniform) L21 x of the non-pivot rows: slice 0 of the partial sums
    __syncthreads();   // the chain's x (yv) written
    if (in_smem) {     // x into the shared tmp (otherwise tmp is yv itself)
      for (int c = threadIdx.x; c < p; c += blockDim.x)
#pragma unroll
        for (int r = 0; r < NR; ++r) tmp[r][c] = yv[r * ldv + first + c];
      __syncthreads();
    }
    for (int i = p + threadIdx.x; i < m; i += blockDim.x) {
      const T* row = F + i;
      T a[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) a[r] = T(0);
#pragma unroll 8
      for (int c = 0; c < p; ++c) {
        const T l = row[(int64_t)c * m];
#pragma unroll
        for (int r = 0; r < NR; ++r) a[r] += l * tmp[r][c];
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) vec[r * vstride + ft.vec_off[f] + m + (i - p)] = a[r];
    }
  }
  if (in_smem)
    for (int i = p + threadIdx.x; i < m; i += blockDim.x)
#pragma unroll
      for (int r = 0; r < NR; ++r) vec[r * vstride + ft.vec_off[f] + i] = w[r][i];
}

// backward chain of one front: subtract the slice sums, U11^{-1} blocks from
// the last one up, and the rows above each block
template <class T, int NR>
__global__ void __launch_bounds__(solve_threads_max<T>(), 1) bwd_tri_kernel(FT ft, const int32_t* fronts, const T* __restrict__ pool,
                                                                T* yv, const T* vec, double* x, bool in_smem,
                                                                int64_t ldv, int64_t vstride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T xw[NR][SOLVE_THREADS / 32][32];
  const int f = fronts[blockIdx.x];
  const int m = ft.m[f], p = ft.p[f], first = ft.first[f];
  T* const vsm = reinterpret_cast<T*>(smem_raw);
  T* v[NR];   // in place in yv when not in shared memory
#pragma unroll
  for (int r = 0; r < NR; ++r) v[r] = in_smem ? vsm + (int64_t)r * p : yv + r * ldv + first;
  const T* F = pool + ft.off[f];
  const int ns = (m - p + SOLVE_SLICE - 1) / SOLVE_SLICE;
  if ((ft.fused[f] & 2) && m > p) {   // (uniform) U12 x2 formed here: x2 of the non-pivot columns first
    __shared__ T x2s[NR][SOLVE_SLICE];
    const int32_t* idx = ft.idx + ft.idx_off[f];
    for (int c = threadIdx.x; c < m - p; c += blockDim.x)
#pragma unroll
      for (int r = 0; r < NR; ++r) x2s[r][c] = (T)x[r * ldv + idx[p + c]];
    __syncthreads();
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
      const T* row = F + (int64_t)p * m + i;
      T a[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) a[r] = T(0);
#pragma unroll 8
      for (int c = 0; c < m - p; ++c) {
        const T u = row[(int64_t)c * m];
#pragma unroll
        for (int r = 0; r < NR; ++r) a[r] += u * x2s[r][c];
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) v[r][i] = yv[r * ldv + first + i] - a[r];
    }
  } else {
    for (int i = threadIdx.x; i < p; i += blockDim.x)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const T* part = vec + r * vstride + ft.vec_off[f] + m;
        T a = yv[r * ldv + first + i];
        for (int s2 = 0; s2 < ns; ++s2) a -= part[(int64_t)s2 * p + i];
        v[r][i] = a;
      }
  }
  if (ft.blk && ft.blk[f] == 2) {   // the chain runs on many CTAs (chain_multi_kernel): v -> yv
    if (in_smem)
      for (int i = threadIdx.x; i < p; i += blockDim.x)
#pragma unroll
        for (int r = 0; r < NR; ++r) yv[r * ldv + first + i] = v[r][i];
    return;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (ft.blk && ft.blk[f]) {   // (block-LU fronts: 128-row blocks stored inverted)
    for (int jb = ((p - 1) / OUTER_NB) * OUTER_NB; jb >= 0 && p > 0; jb -= OUTER_NB)
      chain_block128<T, NR, false>(F, m, p, jb, v, xw[0][0], nullptr, ldv, x + first);
    return;
  }
  for (int jb = ((p - 1) / 32) * 32; jb >= 0 && p > 0; jb -= 32) {
    const int nb = min(32, p - jb);
    // row `lane` of U11^{-1} (upper part, diagonal included)
    T d[32];
    const T* Db = F + (int64_t)jb * m + jb + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) d[j] = (j >= lane && j < nb) ? Db[(int64_t)j * m] : T(0);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const T vl = lane < nb ? v[r][jb + lane] : T(0);
      T xl = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) xl += d[j] * __shfl_sync(0xffffffffu, vl, j);
      xw[r][wid][lane] = xl;
      if (wid == 0 && lane < nb) x[r * ldv + first + jb + lane] = (double)xl;
    }
    __syncwarp();
    for (int i = threadIdx.x; i < jb; i += blockDim.x) {
      const T* col = F + (int64_t)jb * m + i;
      T u[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) u[j] = j < nb ? col[(int64_t)j * m] : T(0);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const T* xr = xw[r][wid];
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          a0 += u[j] * xr[j];
          a1 += u[j + 1] * xr[j + 1];
          a2 += u[j + 2] * xr[j + 2];
          a3 += u[j + 3] * xr[j + 3];
        }
        v[r][i] -= (a0 + a1) + (a2 + a3);
      }
    }
  }
}

// Multi-CTA chains of the large block-LU fronts of one level.  A persistent
// grid takes tasks (front f, block b of 128 pivot rows) from a counter in
// dependency order: forward, the blocks of every front top down; backward,
// bottom up.  A task applies the finished blocks of its front to its rows as
// their flags appear (w_b -= L(b, k) x_k; backward with U), then forms its
// own x_b with the stored inverse of its diagonal block (forward: unit lower
// part of L^{-1}; backward: U^{-1}), writes it (yv; backward also x in FP64)
// and releases its flag.  A task waits only on tasks taken before it, which
// are running or done, so the grid needs no co-residency.  Every wait is
// bounded: on expiry the task sets *err and goes on (the solve is then
// reported, not trusted).  chain[0] is the task counter, chain[1 + i] the
// flags; both are zeroed before the launch.
constexpr int MC_THREADS = 512;                  // 128 rows x 4 column quarters
constexpr long long MC_WAIT_LIMIT = 1LL << 24;   // polls (64 ns apart) before a wait gives up

__device__ __forceinline__ int ld_acquire_gpu(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <class T, int NR, bool FWD>
__global__ void __launch_bounds__(MC_THREADS) chain_multi_kernel(FT ft, const int32_t* __restrict__ tasks,
                                                                 int n_tasks, const T* __restrict__ pool, T* yv,
                                                                 double* x, int32_t* chain, int32_t* err,
                                                                 int64_t ldv) {
  __shared__ T wr[NR][OUTER_NB];       // the task's rows
  __shared__ T xs[NR][OUTER_NB];       // x of the block being applied
  __shared__ T red[NR][4][OUTER_NB];   // partial sums of the four column quarters
  __shared__ int s_task;
  int32_t* flags = chain + 1;
  const int tid = threadIdx.x, rr = tid & (OUTER_NB - 1), q = tid >> 7;
  for (;;) {
    if (tid == 0) s_task = atomicAdd(&chain[0], 1);
    __syncthreads();
    const int t = s_task;
    if (t >= n_tasks) break;   // (uniform)
    const int f = tasks[3 * t], b = tasks[3 * t + 1], fb = tasks[3 * t + 2];
    const int m = ft.m[f], p = ft.p[f], first = ft.first[f];
    const int nblk = (p + OUTER_NB - 1) / OUTER_NB, r0 = OUTER_NB * b, nr = min(OUTER_NB, p - r0);
    const T* F = pool + ft.off[f];
    if (tid < OUTER_NB)
#pragma unroll
      for (int r = 0; r < NR; ++r) wr[r][tid] = tid < nr ? yv[r * ldv + first + r0 + tid] : T(0);
    __syncthreads();
    const int n_apply = FWD ? b : nblk - 1 - b;
    // the factor lines this task reads next go to L2 ahead of time: thread
    // (column tid / 4, 32-row line tid % 4) of a 128 x 128 block
    auto prefetch_block = [&](int col0, int ncols) {
      const int c = tid >> 2, q2 = tid & 3;
      if (c < ncols && 32 * q2 < nr)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(F + (int64_t)(col0 + c) * m + r0 + 32 * q2));
    };
    prefetch_block(r0, nr);   // the own diagonal block's inverse
    for (int k = 0; k < n_apply; ++k) {
      const int kb = FWD ? k : nblk - 1 - k, c0 = OUTER_NB * kb, nc = min(OUTER_NB, p - c0);
      prefetch_block(c0, nc);   // (while the flag is awaited)
      if (tid == 0) {   // bounded wait for block kb
        long long it = 0;
        while (!ld_acquire_gpu(&flags[fb + kb])) {
          if (++it >= MC_WAIT_LIMIT) {
            atomicExch(err, 1);
            break;
          }
          __nanosleep(64);
        }
      }
      __syncthreads();
      if (tid < OUTER_NB)
#pragma unroll
        for (int r = 0; r < NR; ++r) xs[r][tid] = tid < nc ? __ldcg(&yv[r * ldv + first + c0 + tid]) : T(0);
      __syncthreads();
      T a[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) a[r] = T(0);
      if (rr < nr) {
        const T* col = F + (int64_t)(c0 + 32 * q) * m + r0 + rr;
        T v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 32 * q + j < nc ? col[(int64_t)j * m] : T(0);
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
          for (int j = 0; j < 32; ++j) a[r] += v[j] * xs[r][min(32 * q + j, nc - 1)];
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) red[r][q][rr] = a[r];
      __syncthreads();
      if (tid < OUTER_NB)
#pragma unroll
        for (int r = 0; r < NR; ++r) wr[r][tid] -= (red[r][0][tid] + red[r][1][tid]) + (red[r][2][tid] + red[r][3][tid]);
      __syncthreads();
    }
    // x_b = L_bb^{-1} w_b (forward) / U_bb^{-1} v_b (backward) with the stored inverse
    T a[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) a[r] = T(0);
    if (rr < nr) {
      const T* col = F + (int64_t)(r0 + 32 * q) * m + r0 + rr;
      T v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = 32 * q + j;
        v[j] = (c < nr && (FWD ? c < rr : c >= rr)) ? col[(int64_t)j * m] : T(0);
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < 32; ++j) a[r] += v[j] * wr[r][min(32 * q + j, nr - 1)];
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) red[r][q][rr] = a[r];
    __syncthreads();
    if (tid < nr) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const T s = (FWD ? wr[r][tid] : T(0)) + (red[r][0][tid] + red[r][1][tid]) + (red[r][2][tid] + red[r][3][tid]);
        yv[r * ldv + first + r0 + tid] = s;
        if (!FWD) x[r * ldv + first + r0 + tid] = (double)s;
      }
      __threadfence();
    }
    __syncthreads();
    if (tid == 0) st_release_gpu(&flags[fb + b], 1);
  }
}

}  // namespace

// kernel attributes (dynamic shared memory limits) of one precision
template <class T>
static void set_kernel_attributes() {
  if constexpr (std::is_same<T, float>::value) {
    tcp::prepare();
    VIV_CUDA(cudaFuncSetAttribute(block_lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)blk_smem_bytes(OUTER_NB)));
  }
  VIV_CUDA(cudaFuncSetAttribute(panel_smem_kernel<T, 1, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                PANEL_SMEM_BYTES));
  VIV_CUDA(cudaFuncSetAttribute(panel_smem_kernel<T, PANEL_CLUSTER, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                PANEL_SMEM_BYTES));
  VIV_CUDA(cudaFuncSetAttribute(fwd_tri_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX));
  VIV_CUDA(cudaFuncSetAttribute(bwd_tri_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX));
  VIV_CUDA(cudaFuncSetAttribute(fwd_tri_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX));
  VIV_CUDA(cudaFuncSetAttribute(bwd_tri_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX));
  VIV_CUDA(cudaFuncSetAttribute(perm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, PERM_SMEM_MAX));
}

// set once per device and precision, before any launch (including before a
// stream capture); the serving loop's worker threads get here concurrently,
// hence call_once (an exception leaves the flag unset, so a later call retries)
template <class T>
void prepare_kernels() {
  constexpr int MAX_DEV = 64;
  static std::once_flag once[MAX_DEV];
  int dev = 0;
  VIV_CUDA(cudaGetDevice(&dev));
  VIV_CHECK(dev >= 0 && dev < MAX_DEV, VIV_ERR_ARG, "device index out of range");
  std::call_once(once[dev], [] { set_kernel_attributes<T>(); });
}
template void prepare_kernels<float>();
template void prepare_kernels<double>();

template <class T>
void factor_numeric(const Mesh& m, const double* J64, const float* J32, T* fronts, int32_t* piv, int32_t* perm,
                    int32_t* stats, double threshold, bool window, unsigned char* tc_img, cudaStream_t s) {
  FT ft = make_ft(m);
  prepare_kernels<T>();
  VIV_CUDA(cudaMemsetAsync(stats, 0, 4 * sizeof(int32_t), s));
  const int32_t* work = m.ft.work;
  for (const Launch& L : m.sched[(sizeof(T) == 8) + 2 * (window ? 1 : 0)]) {
    prof_level(L.level);
    const int32_t* w = work + (int64_t)WORK_STRIDE * L.item0;
    const unsigned grid = (unsigned)L.count;
    static const int kk[13] = {K_FRONT_ASM, K_PANEL,  K_TRSM,   K_GEMM,    K_PANEL, K_TRSM, K_PANEL,
                               K_TCGEMM,    K_PANEL, K_TRSM, K_TCSPLIT, K_PANEL, K_TRSM};
    Launched LL(kk[L.kind], s);
    switch (L.kind) {
      case L_ASSEMBLE:
        if (J32)
          assemble_kernel<T, float><<<grid, L.aux, 0, s>>>(ft, w, J32, fronts);
        else
          assemble_kernel<T, double><<<grid, L.aux, 0, s>>>(ft, w, J64, fronts);
        break;
      case L_PANEL:
        panel_kernel<T><<<grid, PANEL_THREADS, 0, s>>>(ft, w, L.k, fronts, piv, stats, (T)threshold);
        break;
      case L_TRSM:
        trsm_kernel<T><<<grid, TRSM_COLS, 0, s>>>(ft, w, fronts);
        break;
      case L_GEMM:
        gemm_kernel<T><<<grid, 256, 0, s>>>(ft, w, fronts, piv, perm, stats);
        break;
      case L_BLOCK_LU:   // aux: the launch's largest block width nn (a multiple of 32)
        if constexpr (std::is_same<T, float>::value)
          block_lu_kernel<<<grid, 4 * L.aux, blk_smem_bytes(L.aux), s>>>(ft, w, fronts, perm, stats,
                                                                        (float)threshold, tc_img, L.aux);
        break;
      case L_BLOCK_PERM:
        if constexpr (std::is_same<T, float>::value)
          block_perm_kernel<<<grid, PERM_THREADS, 0, s>>>(ft, w, fronts, perm);
        break;
      case L_TC_SPLIT:
        if constexpr (std::is_same<T, float>::value) tcp::split_launch(w, (int)L.count, fronts, ft.off, ft.m, tc_img, stats, (float)threshold, s);
        break;
      case L_TC_GEMM:
        if constexpr (std::is_same<T, float>::value)
          tcp::pipe_launch(w, (int)L.count, tc_img, fronts, ft.off, ft.m, stats + 2, s);
        break;
      case L_PANEL_1: {
        const size_t smem = (size_t)L.aux * PANEL_NB * sizeof(T);
        panel_smem_kernel<T, 1, 512><<<grid, 512, smem, s>>>(ft, w, L.k, fronts, piv, stats, (T)threshold);
        break;
      }
      case L_PANEL_CL: {
        const size_t smem = (size_t)L.aux * PANEL_NB * sizeof(T);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid * PANEL_CLUSTER);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = PANEL_CLUSTER;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        VIV_CUDA(cudaLaunchKernelEx(&cfg, panel_smem_kernel<T, PANEL_CLUSTER, 256>, ft, w, L.k, fronts, piv, stats,
                                    (T)threshold));
        break;
      }
      case L_DIAG:
        diag_lu_kernel<T><<<grid, 32, 0, s>>>(ft, w, L.k, fronts, piv, perm, stats);
        break;
      case L_WINDOW:
        window_kernel<T><<<grid, WINDOW_THREADS, 0, s>>>(ft, w, L.k, fronts, perm, stats, (T)threshold);
        break;
      case L_LASWP:
        laswp_kernel<T><<<grid, LASWP_COLS, 0, s>>>(ft, w, L.k, fronts, piv);
        break;
    }
  }
  VIV_CUDA(cudaGetLastError());
  prof_level(-1);
  // solve preparation: composed row permutations, inverted diagonal blocks
  if (!window) {   // (windowed pivoting: the diagonal LUs wrote the permutations)
    Launched LL(K_TRSM, s);
    perm_kernel<<<m.n_fronts, 128, 2 * (size_t)std::max(1, m.max_p) * sizeof(int32_t), s>>>(ft, piv, perm);
  }
  // (the block LU stored its blocks' diagonal parts inverted already)
  const bool blk = std::is_same<T, float>::value && window && m.block_lu;
  const std::vector<int32_t>& inv = blk ? m.inv_items_blk : m.inv_items;
  if (!inv.empty()) {
    Launched LL(K_TRSM, s);
    const int n = (int)(inv.size() / 2);
    diag_inv_kernel<T><<<(n + INV_WARPS - 1) / INV_WARPS, INV_WARPS * 32, 0, s>>>(
        ft, blk ? m.d_inv_items_blk : m.d_inv_items, n, fronts);
  }
  VIV_CUDA(cudaGetLastError());
}

// NR right-hand sides: vector r of b and x at r * ldv (doubles), of yv at
// r * ldv (T), of the workspace vec at r * vstride (T)
template <class T, int NR>
void solve_fronts_nr(const Mesh& m, const T* fronts, const int32_t* perm, const double* b, double* x, T* vec, T* yv,
                     int64_t ldv, int64_t vstride, bool blk, int32_t* chain, int32_t* err, cudaStream_t s) {
  FT ft = make_ft(m, blk);
  VIV_CHECK(!blk || (chain && err), VIV_ERR_ARG, "block-LU solves need the case's chain flags");
  // the level's multi-CTA chains (block-LU fronts of order >= MULTI_CHAIN_P)
  auto multi = [&](int l, bool fwd) {
    if constexpr (std::is_same<T, float>::value) {
      const int n = blk ? m.mc_off[l + 1] - m.mc_off[l] : 0;
      if (!n) return;
      VIV_CUDA(cudaMemsetAsync(chain, 0, (1 + (size_t)m.mc_flags) * sizeof(int32_t), s));
      Launched L(fwd ? K_FWD : K_BWD, s);
      const int grid = std::min(n, device_sm_count());
      const int32_t* tasks = (fwd ? m.d_mc_fwd : m.d_mc_bwd) + 3 * (int64_t)m.mc_off[l];
      if (fwd)
        chain_multi_kernel<T, NR, true><<<grid, MC_THREADS, 0, s>>>(ft, tasks, n, fronts, yv, x, chain, err, ldv);
      else
        chain_multi_kernel<T, NR, false><<<grid, MC_THREADS, 0, s>>>(ft, tasks, n, fronts, yv, x, chain, err, ldv);
    }
  };
  prepare_kernels<T>();
  for (int l = 0; l < m.n_levels; ++l) {
    prof_level(l);
    const int n = m.level_off[l + 1] - m.level_off[l];
    const size_t need = (size_t)NR * (m.level_maxm[l] + m.level_maxp[l]) * sizeof(T);
    const bool sm = need <= (size_t)SOLVE_SMEM_MAX;
    {
      Launched L(K_FWD, s);
      fwd_tri_kernel<T, NR><<<n, std::min(m.level_threads[l], solve_threads_max<T>()), sm ? need : 0, s>>>(
          ft, m.d_level_fronts + m.level_off[l], fronts, perm, b, vec, yv, sm, ldv, vstride);
    }
    multi(l, true);
    const int ng = m.fg_off[l + 1] - m.fg_off[l];
    if (ng) {
      Launched L(K_FWD, s);
      solve_gemv_kernel<T, true, NR><<<ng, GEMV_THREADS, 0, s>>>(ft, m.d_fg_items + 4 * (int64_t)m.fg_off[l], fronts,
                                                                  yv, x, vec, ldv, vstride);
    }
  }
  for (int l = m.n_levels - 1; l >= 0; --l) {
    prof_level(l);
    const int ng = m.bg_off[l + 1] - m.bg_off[l];
    if (ng) {
      Launched L(K_BWD, s);
      solve_gemv_kernel<T, false, NR><<<ng, GEMV_THREADS, 0, s>>>(ft, m.d_bg_items + 4 * (int64_t)m.bg_off[l],
                                                                   fronts, yv, x, vec, ldv, vstride);
    }
    const int n = m.level_off[l + 1] - m.level_off[l];
    const size_t need = (size_t)NR * m.level_maxp[l] * sizeof(T);
    const bool sm = need <= (size_t)SOLVE_SMEM_MAX;
    {
      Launched L(K_BWD, s);
      bwd_tri_kernel<T, NR><<<n, std::min(m.level_threads[l], solve_threads_max<T>()), sm ? need : 0, s>>>(
          ft, m.d_level_fronts + m.level_off[l], fronts, yv, vec, x, sm, ldv, vstride);
    }
    multi(l, false);
  }
  prof_level(-1);
  VIV_CUDA(cudaGetLastError());
}

template <class T>
void solve_fronts(const Mesh& m, const T* fronts, const int32_t* perm, const double* b, double* x, T* vec, T* yv,
                  bool blk, int32_t* chain, int32_t* err, cudaStream_t s) {
  solve_fronts_nr<T, 1>(m, fronts, perm, b, x, vec, yv, m.n_dofs, m.vec_entries, blk, chain, err, s);
}

// two right-hand sides in one pass (the border columns): b, x, yv hold two
// vectors of m.n_dofs, vec two workspaces of m.vec_entries
template <class T>
void solve_fronts2(const Mesh& m, const T* fronts, const int32_t* perm, const double* b, double* x, T* vec, T* yv,
                   bool blk, int32_t* chain, int32_t* err, cudaStream_t s) {
  solve_fronts_nr<T, 2>(m, fronts, perm, b, x, vec, yv, m.n_dofs, m.vec_entries, blk, chain, err, s);
}

template void factor_numeric<double>(const Mesh&, const double*, const float*, double*, int32_t*, int32_t*,
                                     int32_t*, double, bool, unsigned char*, cudaStream_t);
template void factor_numeric<float>(const Mesh&, const double*, const float*, float*, int32_t*, int32_t*, int32_t*,
                                    double, bool, unsigned char*, cudaStream_t);
template void solve_fronts<double>(const Mesh&, const double*, const int32_t*, const double*, double*, double*,
                                   double*, bool, int32_t*, int32_t*, cudaStream_t);
template void solve_fronts<float>(const Mesh&, const float*, const int32_t*, const double*, double*, float*,
                                  float*, bool, int32_t*, int32_t*, cudaStream_t);
template void solve_fronts2<double>(const Mesh&, const double*, const int32_t*, const double*, double*, double*,
                                    double*, bool, int32_t*, int32_t*, cudaStream_t);
template void solve_fronts2<float>(const Mesh&, const float*, const int32_t*, const double*, double*, float*,
                                   float*, bool, int32_t*, int32_t*, cudaStream_t);

}  // namespace viv
