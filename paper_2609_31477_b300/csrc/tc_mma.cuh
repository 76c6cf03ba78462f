// tcgen05 (kind::tf32, 3xTF32) tile update shared by the standalone GEMM
// entry point and the front-batched Schur updates of the factorisation.
//
// C -= A * B for one 128 x 128 tile, A: M x K, B: K x N, C: M x N, all
// column-major FP32.  Every FP32 operand is split into hi = tf32(x) and
// lo = tf32(x - hi); the product is accumulated in FP32 in tensor memory as
// lo*hi + hi*lo + hi*hi, which keeps close to FP32 accuracy.  Operands are
// staged in shared memory in the canonical K-major, no-swizzle core-matrix
// layout (8 rows x 16 bytes per core matrix); one elected thread issues the
// MMAs and commits them to an mbarrier; every wait is bounded and on expiry
// the tile is skipped and an error flag is raised instead of hanging.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace viv {
namespace tc {

constexpr int BM = 128, BN = 128, KC = 32;        // tile and K chunk
constexpr int THREADS = 256;                     // 8 warps stage operands; one thread issues MMAs
constexpr int CORE_BYTES = 128;                   // 8 rows x 16 bytes
constexpr int KCORE_STRIDE = (BM / 8) * CORE_BYTES;   // bytes between K-adjacent core matrices (LBO)
constexpr int OPERAND_BYTES = BM * KC * 4;        // one 128 x 32 FP32 operand chunk
constexpr uint32_t TMEM_COLS = 128;
constexpr long long WAIT_LIMIT = 1LL << 24;       // bounded mbarrier polling

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// shared-memory matrix descriptor: start, LBO (K direction), SBO (M/N
// direction), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// bounded wait for the phase with the given parity; false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// byte offset of element (row r, k) of a 128 x 32 K-major chunk
__device__ __forceinline__ int kmajor_off(int r, int k) {
  return (k >> 2) * KCORE_STRIDE + (r >> 3) * CORE_BYTES + (r & 7) * 16 + (k & 3) * 4;
}

struct Stage {
  alignas(1024) unsigned char a_hi[OPERAND_BYTES];
  alignas(1024) unsigned char a_lo[OPERAND_BYTES];
  alignas(1024) unsigned char b_hi[OPERAND_BYTES];
  alignas(1024) unsigned char b_lo[OPERAND_BYTES];
};

// One operand stage (64 KB) so that three CTAs fit on an SM; the next K
// chunk waits in registers while the MMAs of the current one run.
struct Smem {
  Stage st;
  uint64_t bar;         // completed by tcgen05.commit of the stage's MMAs
  uint32_t tmem_base;
};

constexpr int PER = BM * (KC / 4) / THREADS;   // (row, k-group) pairs per thread = 4
struct ChunkRegs {
  float va[PER][4], vb[PER][4];
};

// (row, k-group) pair t of this thread for A (rows contiguous in memory: the
// row index runs fastest across a warp) and for B (k contiguous: the k-group
// runs fastest, so eight lanes read one 128-byte column segment)
__device__ __forceinline__ void pair_a(int t, int& r, int& g) {
  const int idx = threadIdx.x + t * THREADS;
  r = idx % BM;
  g = idx / BM;
}
__device__ __forceinline__ void pair_b(int t, int& r, int& g) {
  const int idx = threadIdx.x + t * THREADS;
  g = idx % (KC / 4);
  r = idx / (KC / 4);
}

// global loads of K-chunk [k0, k0 + KC) of A (rows rb..) and B (columns
// cb..), read-only path (A and B are never written by the update)
__device__ __forceinline__ void load_chunk(ChunkRegs& R, const float* __restrict__ A, int lda,
                                           const float* __restrict__ B, int ldb, int M, int N, int K, int rb, int cb,
                                           int k0) {
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    int r, g;
    pair_a(t, r, g);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + 4 * g + j;
      R.va[t][j] = (rb + r < M && k < K) ? __ldg(A + (int64_t)k * lda + rb + r) : 0.f;
    }
    pair_b(t, r, g);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + 4 * g + j;
      R.vb[t][j] = (cb + r < N && k < K) ? __ldg(B + (int64_t)(cb + r) * ldb + k) : 0.f;
    }
  }
}

// hi/lo TF32 split of a loaded chunk into the stage; every thread writes
// whole 16-byte core-matrix rows
__device__ __forceinline__ void store_chunk(Stage& S, const ChunkRegs& R) {
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    uint32_t h[4], l[4];
    int r, g;
    pair_a(t, r, g);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[j] = to_tf32(R.va[t][j]);
      l[j] = to_tf32(R.va[t][j] - __uint_as_float(h[j]));
    }
    int off = g * KCORE_STRIDE + (r >> 3) * CORE_BYTES + (r & 7) * 16;
    *reinterpret_cast<uint4*>(S.a_hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(S.a_lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    pair_b(t, r, g);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[j] = to_tf32(R.vb[t][j]);
      l[j] = to_tf32(R.vb[t][j] - __uint_as_float(h[j]));
    }
    off = g * KCORE_STRIDE + (r >> 3) * CORE_BYTES + (r & 7) * 16;
    *reinterpret_cast<uint4*>(S.b_hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(S.b_lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// C[rb.., cb..] -= A[rb.., 0:K] * B[0:K, cb..] for one 128 x 128 tile
static __device__ void tile_update(Smem& sm, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                                   int M, int N, int K, int rb, int cb, int* err) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&sm.bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sm.tmem_base;
  constexpr uint32_t idesc = make_idesc(BM, BN);
  uint32_t ph = 0u;        // parity of the barrier phase the next wait is for
  bool ok = true;
  bool pending = false;     // a commit (the MMAs of one chunk) not yet seen complete
  const int nchunks = (K + KC - 1) / KC;
  ChunkRegs R;
  load_chunk(R, A, lda, B, ldb, M, N, K, rb, cb, 0);
  for (int ch = 0; ch < nchunks; ++ch) {
    if (ch > 0) {   // the MMAs of chunk ch - 1 still read the stage: wait for them
      const bool w = mbar_wait(&sm.bar, ph);
      if (!__syncthreads_and(w)) {
        ok = false;   // the commit of chunk ch - 1 is still pending (phase ph)
        break;
      }
      ph ^= 1u;
      pending = false;
    }
    store_chunk(sm.st, R);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ah = smem_u32(sm.st.a_hi), al = smem_u32(sm.st.a_lo);
      const uint32_t bh = smem_u32(sm.st.b_hi), bl = smem_u32(sm.st.b_lo);
#pragma unroll
      for (int q = 0; q < KC / 8; ++q) {
        const uint32_t koff = (uint32_t)(2 * q * KCORE_STRIDE);   // 8 tf32 = 2 core matrices along K
        const uint64_t dah = make_desc(ah + koff, KCORE_STRIDE, CORE_BYTES);
        const uint64_t dal = make_desc(al + koff, KCORE_STRIDE, CORE_BYTES);
        const uint64_t dbh = make_desc(bh + koff, KCORE_STRIDE, CORE_BYTES);
        const uint64_t dbl = make_desc(bl + koff, KCORE_STRIDE, CORE_BYTES);
        mma_tf32(tmem, dal, dbh, idesc, (ch > 0 || q > 0) ? 1u : 0u);   // small terms first
        mma_tf32(tmem, dah, dbl, idesc, 1u);
        mma_tf32(tmem, dah, dbh, idesc, 1u);
      }
      mma_commit(&sm.bar);
    }
    pending = true;
    __syncwarp();
    if (ch + 1 < nchunks) load_chunk(R, A, lda, B, ldb, M, N, K, rb, cb, (ch + 1) * KC);   // overlaps the MMAs
  }
  if (ok && pending) {   // the last commit
    const bool w = mbar_wait(&sm.bar, ph);
    asm volatile("tcgen05.fence::after_thread_sync;");
    ok = __syncthreads_and(w) != 0;
    if (ok) pending = false;
  }
  if (!ok) {
    // Expired wait: flag the tile, then wait once more (bounded) for the MMAs
    // still in flight - a commit tracks every earlier MMA of the issuing
    // thread, so the pending phase completing means none is left - before
    // the accumulator is released below.  A commit that never completes
    // means the tensor core stopped; the tile is then abandoned as well.
    if (tid == 0) atomicExch(err, 1);
    if (pending) {
      const bool w = mbar_wait(&sm.bar, ph);
      asm volatile("tcgen05.fence::after_thread_sync;");
      (void)__syncthreads_and(w);
    }
  } else {
    // epilogue: warp w reads accumulator lanes 32 (w % 4) .. (tile rows) and
    // column half w / 4; each thread owns one row
    const int quarter = warp & 3, half = warp >> 2;
    const int r = rb + quarter * 32 + lane;
    for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
            "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < M) {
        // all 16 loads of C first, then the 16 stores: loads stay in flight together
        float cv[16];
        float* cr = C + (int64_t)(cb + c0) * ldc + r;
#pragma unroll
        for (int j = 0; j < 16; ++j) cv[j] = (cb + c0 + j < N) ? cr[(int64_t)j * ldc] : 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (cb + c0 + j < N) cr[(int64_t)j * ldc] = cv[j] - __uint_as_float(v[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace tc
}  // namespace viv
