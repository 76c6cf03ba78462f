// Kernels of the pipelined tcgen05 Schur-complement update (see tc_pipe.cuh)
// with their host launchers, and the standalone update C -= A B behind
// viv_tc_schur_update, which runs through the same two kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "tc_pipe.cuh"
#include "viv_internal.h"

namespace viv {
namespace tcp {

// ---- split ---------------------------------------------------------------------
__global__ void __launch_bounds__(SPLIT_THREADS) tc_split_kernel(const int32_t* __restrict__ items,
                                                                 const float* __restrict__ pool,
                                                                 const int64_t* __restrict__ off,
                                                                 const int32_t* __restrict__ ld,
                                                                 unsigned char* __restrict__ img,
                                                                 int* __restrict__ stats, float thresh) {
  const int32_t* it = items + (int64_t)ITEM * blockIdx.x;
  const int f = it[0], start = it[1], kind = it[2], k0 = it[3], klen = it[4], blk = it[5], limit = it[6];
  const int check = it[7];
  const float* base = pool + off[f];
  const int64_t L = ld[f];
  unsigned char* out = img + (int64_t)blk * CHUNK_BYTES;
  constexpr int PER = BM * (KC / 4) / SPLIT_THREADS;   // (row, k-group) pairs per thread: 4
  float v[PER][4];
  int rr[PER], gg[PER];
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int idx = threadIdx.x + t * SPLIT_THREADS;
    // A: rows contiguous in memory (row fastest across lanes); B: k contiguous
    const int r = kind == 0 ? idx % BM : idx / (KC / 4);
    const int g = kind == 0 ? idx / BM : idx % (KC / 4);
    rr[t] = r;
    gg[t] = g;
    const bool row_ok = start + r < limit;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * g + j;
      const bool ok = row_ok && k < klen;
      const int64_t e = kind == 0 ? (int64_t)(k0 + k) * L + start + r : (int64_t)(start + r) * L + k0 + k;
      v[t][j] = ok ? __ldg(base + e) : 0.f;
    }
  }
  if (check) {   // (uniform per CTA)
    bool big = false;
#pragma unroll
    for (int t = 0; t < PER; ++t)
#pragma unroll
      for (int j = 0; j < 4; ++j) big = big || fabsf(v[t][j]) * thresh > 1.f;
    if (__syncthreads_or(big) && threadIdx.x == 0) atomicAdd(&stats[1], 1);
  }
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[j] = tc::to_tf32(v[t][j]);
      l[j] = tc::to_tf32(v[t][j] - __uint_as_float(h[j]));
    }
    const int o = gg[t] * KCORE_STRIDE + (rr[t] >> 3) * CORE_BYTES + (rr[t] & 7) * 16;
    *reinterpret_cast<uint4*>(out + o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(out + OPERAND_BYTES + o) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// ---- persistent pipelined update -------------------------------------------------
__global__ void __launch_bounds__(THREADS, 1) tc_pipe_kernel(const int32_t* __restrict__ items, int n_items,
                                                            const unsigned char* __restrict__ img, float* pool,
                                                            const int64_t* __restrict__ off,
                                                            const int32_t* __restrict__ ld, int* err) {
  extern __shared__ unsigned char smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&sm.full[s], 1);
      tc::mbar_init(&sm.empty[s], 1);
    }
    for (int s = 0; s < A_SLOTS; ++s) {
      tc::mbar_init(&sm.a_full[s], 1);
      tc::mbar_init(&sm.a_empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&sm.acc_full[a], 1);
      tc::mbar_init(&sm.acc_empty[a], EPI_WARPS);
    }
    tc::mbar_init(&sm.drain, 1);
    sm.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&sm.tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sm.tmem_base;
  // this CTA's tiles: blockIdx.x, + gridDim.x, ... (round robin: the CTAs work
  // on neighbouring tiles at any moment, which keeps the shared A and B image
  // chunks and the C columns in L2; measured faster than contiguous ranges)
  const int t0 = blockIdx.x, t1 = n_items, tstep = gridDim.x;

  if (warp == 0) {
    // ---- producer: a segment's A chunks once (interleaved with its first
    // tile's B chunks), then the B chunks of its other tiles ----
    if (lane == 0) {
      uint32_t issued = 0, issued_parity = 0;       // per B slot: a fill was issued / its phase parity
      uint32_t a_issued = 0, a_issued_parity = 0;   // the same per A slot
      uint32_t u = 0, ua = 0;                       // B and A chunks of this CTA
      int prev_a = -1, prev_nch = 0;
      bool ok = true;
      for (int t = t0; t < t1 && ok; t += tstep) {
        const int32_t* it = items + (int64_t)ITEM * t;
        const int a_blk = it[5], b_blk = it[6], nch = it[7];
        const bool new_seg = a_blk != prev_a;
        if (new_seg) ua += (uint32_t)prev_nch;
        prev_a = a_blk;
        prev_nch = nch;
        {
          for (int ch = 0; ch < nch; ++ch) {
            if (new_seg) {
              const int x = (int)((ua + ch) % A_SLOTS);
              const uint32_t round = (ua + ch) / A_SLOTS;
              if (!wait_phase(sm, &sm.a_empty[x], (round & 1u) ^ 1u, true)) {
                raise_abort(sm, err);
                ok = false;
                break;
              }
              arrive_expect_tx(&sm.a_full[x], CHUNK_BYTES);
              bulk_copy(sm.a[x], img + (int64_t)(a_blk + ch) * CHUNK_BYTES, CHUNK_BYTES, &sm.a_full[x]);
              a_issued |= 1u << x;
              a_issued_parity = (a_issued_parity & ~(1u << x)) | ((round & 1u) << x);
            }
            const int s = (int)(u % STAGES);
            const uint32_t round = u / STAGES;
            if (!wait_phase(sm, &sm.empty[s], (round & 1u) ^ 1u, true)) {
              raise_abort(sm, err);
              ok = false;
              break;
            }
            arrive_expect_tx(&sm.full[s], CHUNK_BYTES);
            bulk_copy(sm.b[s], img + (int64_t)(b_blk + ch) * CHUNK_BYTES, CHUNK_BYTES, &sm.full[s]);
            issued |= 1u << s;
            issued_parity = (issued_parity & ~(1u << s)) | ((round & 1u) << s);
            ++u;
          }
        }
      }
      // no CTA leaves while copies into its shared memory are in flight
      for (int x = 0; x < A_SLOTS; ++x)
        if (((a_issued >> x) & 1u) && !wait_phase(sm, &sm.a_full[x], (a_issued_parity >> x) & 1u, false))
          atomicExch(err, 1);
      for (int s = 0; s < STAGES; ++s)
        if (((issued >> s) & 1u) && !wait_phase(sm, &sm.full[s], (issued_parity >> s) & 1u, false))
          atomicExch(err, 1);
    }
  } else if (warp == 1) {
    // ---- MMA issue ----
    if (lane == 0) {
      constexpr uint32_t idesc = tc::make_idesc(BM, BN);
      uint32_t u = 0, ua = 0, v = 0;
      int prev_a = -1, prev_nch = 0;
      bool ok = true;
      for (int t = t0; t < t1 && ok; t += tstep) {
        const int32_t* it = items + (int64_t)ITEM * t;
        const int a_blk = it[5], nch = it[7];
        if (a_blk != prev_a) ua += (uint32_t)prev_nch;
        prev_a = a_blk;
        prev_nch = nch;
        // the segment's last tile releases its A slots
        const bool last = t + tstep >= t1 || items[(int64_t)ITEM * (t + tstep) + 5] != a_blk;
        {
          const int acc = (int)(v & 1u);
          const uint32_t use = v >> 1;
          if (!wait_phase(sm, &sm.acc_empty[acc], (use & 1u) ^ 1u, true)) {
            raise_abort(sm, err);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t d = tmem + (uint32_t)(acc * BN);
          for (int ch = 0; ch < nch; ++ch, ++u) {
            const int x = (int)((ua + ch) % A_SLOTS);
            const uint32_t around = (ua + ch) / A_SLOTS;
            const int s = (int)(u % STAGES);
            const uint32_t round = u / STAGES;
            // (the A slot stays filled for the whole segment: later waits return at once)
            if (!wait_phase(sm, &sm.a_full[x], around & 1u, true) || !wait_phase(sm, &sm.full[s], round & 1u, true)) {
              raise_abort(sm, err);
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ah = tc::smem_u32(sm.a[x]), al = ah + OPERAND_BYTES;
            const uint32_t bh = tc::smem_u32(sm.b[s]), bl = bh + OPERAND_BYTES;
#pragma unroll
            for (int q = 0; q < KC / 8; ++q) {
              const uint32_t koff = (uint32_t)(2 * q * KCORE_STRIDE);   // 8 tf32 = 2 core matrices along K
              const uint64_t dah = tc::make_desc(ah + koff, KCORE_STRIDE, CORE_BYTES);
              const uint64_t dal = tc::make_desc(al + koff, KCORE_STRIDE, CORE_BYTES);
              const uint64_t dbh = tc::make_desc(bh + koff, KCORE_STRIDE, CORE_BYTES);
              const uint64_t dbl = tc::make_desc(bl + koff, KCORE_STRIDE, CORE_BYTES);
              tc::mma_tf32(d, dal, dbh, idesc, (ch > 0 || q > 0) ? 1u : 0u);   // small terms first
              tc::mma_tf32(d, dah, dbl, idesc, 1u);
              tc::mma_tf32(d, dah, dbh, idesc, 1u);
            }
            tc::mma_commit(&sm.empty[s]);                // the B slot may be refilled
            if (last) tc::mma_commit(&sm.a_empty[x]);   // the segment's last tile: the A slot too
          }
          if (!ok) break;
          tc::mma_commit(&sm.acc_full[acc]);
          ++v;
        }
      }
      // every MMA this thread issued has completed once this commit arrives
      tc::mma_commit(&sm.drain);
      if (!wait_phase(sm, &sm.drain, 0u, false)) atomicExch(err, 1);
    }
  } else {
    // ---- epilogue: warp w reads accumulator lanes 32 (w % 4) .. + 31 (its TMEM
    // lane quarter); each thread owns one tile row and its 128 columns, in
    // four groups of 32 with the loads of C two groups ahead ----
    const int quarter = warp & 3;
    int v = 0;
    bool ok = true;
    for (int t = t0; t < t1 && ok; t += tstep, ++v) {
      const int32_t* it = items + (int64_t)ITEM * t;
      const int f = it[0], rb = it[1], cb = it[2], r_end = it[3], c_end = it[4];
      const int64_t ldc = ld[f];
      const int row = rb + quarter * 32 + lane;
      // columns of the tile that exist for this row (none past the last row)
      const int ncol = row < r_end ? max(0, min(BN, c_end - cb)) : 0;
      float* const crow = pool + off[f] + (int64_t)cb * ldc + row;
      float c0v[32], c1v[32];   // C of group g: even g in c0v, odd g in c1v
      auto load_group = [&](float* dst, int g) {
        const float* src = crow + (int64_t)(32 * g) * ldc;
#pragma unroll
        for (int j = 0; j < 32; ++j, src += ldc) dst[j] = 32 * g + j < ncol ? *src : 0.f;
      };
      load_group(c0v, 0);   // before the accumulator is ready: overlaps the MMAs
      load_group(c1v, 1);
      // this warp's rows of the next tiles' C into L2 while this tile completes
      // (lane l: columns l, l + 32, l + 64, l + 96; a 32-row column segment
      // spans at most two 128-byte lines)
      for (int ahead = 1; ahead <= PREFETCH_TILES && t + ahead * tstep < t1; ++ahead) {
        const int32_t* nx = items + (int64_t)ITEM * (t + ahead * tstep);
        const int nf = nx[0], row0 = nx[1] + quarter * 32, ncb = nx[2], nr_end = nx[3], nc_end = nx[4];
        if (row0 < nr_end) {
          const int64_t nld = ld[nf];
          const float* nbase = pool + off[nf] + (int64_t)ncb * nld + row0;
          const int last = min(32, nr_end - row0) - 1;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = lane + 32 * q;
            if (ncb + j < nc_end) {
              const float* p0 = nbase + (int64_t)j * nld;
              asm volatile("prefetch.global.L2 [%0];" ::"l"(p0));
              asm volatile("prefetch.global.L2 [%0];" ::"l"(p0 + last));
            }
          }
        }
      }
      const int acc = v & 1;
      const uint32_t use = (uint32_t)(v >> 1);
      int got = 0;
      if (lane == 0) got = wait_phase(sm, &sm.acc_full[acc], use & 1u, true) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) {
        if (lane == 0) raise_abort(sm, err);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float* cur = (g & 1) ? c1v : c0v;
        uint32_t a[32];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * BN + 32 * g);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
              "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]),
              "=r"(a[15]), "=r"(a[16]), "=r"(a[17]), "=r"(a[18]), "=r"(a[19]), "=r"(a[20]), "=r"(a[21]),
              "=r"(a[22]), "=r"(a[23]), "=r"(a[24]), "=r"(a[25]), "=r"(a[26]), "=r"(a[27]), "=r"(a[28]),
              "=r"(a[29]), "=r"(a[30]), "=r"(a[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float* dst = crow + (int64_t)(32 * g) * ldc;
#pragma unroll
        for (int j = 0; j < 32; ++j, dst += ldc)
          if (32 * g + j < ncol) *dst = cur[j] - __uint_as_float(a[j]);
        if (g + 2 < 4) load_group(cur, g + 2);
      }
      // the accumulator may be overwritten once every epilogue warp has read it
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) arrive(&sm.acc_empty[acc]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}


void prepare() {
  constexpr int MAX_DEV = 64;
  static std::once_flag once[MAX_DEV];   // per device; callers may be concurrent threads
  int dev = 0;
  VIV_CUDA(cudaGetDevice(&dev));
  VIV_CHECK(dev >= 0 && dev < MAX_DEV, VIV_ERR_ARG, "device index out of range");
  std::call_once(once[dev], [] {
    VIV_CUDA(cudaFuncSetAttribute(tc_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
  });
}

void split_launch(const int32_t* items, int n_items, const float* pool, const int64_t* off, const int32_t* ld,
                  unsigned char* img, int* stats, float thresh, cudaStream_t s) {
  if (n_items > 0)
    tc_split_kernel<<<(unsigned)n_items, SPLIT_THREADS, 0, s>>>(items, pool, off, ld, img, stats, thresh);
}

// persistent: one CTA per SM at most (the ring and the two accumulators fill
// an SM's shared and tensor memory budget for this kernel)
void pipe_launch(const int32_t* items, int n_items, const unsigned char* img, float* pool, const int64_t* off,
                 const int32_t* ld, int* err, cudaStream_t s) {
  if (n_items > 0)
    tc_pipe_kernel<<<(unsigned)std::min(n_items, device_sm_count()), THREADS, SMEM_BYTES, s>>>(items, n_items, img,
                                                                                             pool, off, ld, err);
}

}  // namespace tcp

// streaming multiprocessors of the current device (queried once per device)
int device_sm_count() {
  constexpr int MAX_DEV = 64;
  static std::once_flag once[MAX_DEV];
  static int count[MAX_DEV];
  int dev = 0;
  VIV_CUDA(cudaGetDevice(&dev));
  VIV_CHECK(dev >= 0 && dev < MAX_DEV, VIV_ERR_ARG, "device index out of range");
  std::call_once(once[dev], [&] { VIV_CUDA(cudaDeviceGetAttribute(&count[dev], cudaDevAttrMultiProcessorCount, dev)); });
  return count[dev];
}

// The three matrices are addressed as "fronts" 0 (A), 1 (B), 2 (C) of one
// pool based at C: off[] holds A - C and B - C in floats.  The work items,
// the tables and the operand images live in one stream-ordered allocation
// that is released on the stream after the update.
void tc_gemm_update(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int M, int N, int K,
                    int* err, cudaStream_t s) {
  tcp::prepare();
  if (M <= 0 || N <= 0 || K <= 0) return;
  // one update takes K <= 128 (the resident A chunks); larger K runs as
  // successive updates over 128-wide slices of K
  if (K > tcp::MAX_CHUNKS * tcp::KC) {
    for (int k0 = 0; k0 < K; k0 += tcp::MAX_CHUNKS * tcp::KC)
      tc_gemm_update(A + (int64_t)k0 * lda, lda, B + k0, ldb, C, ldc, M, N,
                     std::min(tcp::MAX_CHUNKS * tcp::KC, K - k0), err, s);
    return;
  }
  const int nch = (K + tcp::KC - 1) / tcp::KC, nrb = (M + tcp::BM - 1) / tcp::BM, ncb = (N + tcp::BN - 1) / tcp::BN;
  std::vector<int32_t> split, tiles;
  int blk = 0;
  for (int i = 0; i < nrb; ++i)
    for (int ch = 0; ch < nch; ++ch)
      split.insert(split.end(), {0, i * tcp::BM, 0, ch * tcp::KC, std::min(tcp::KC, K - ch * tcp::KC), blk++, M, 0});
  const int b0 = blk;
  for (int j = 0; j < ncb; ++j)
    for (int ch = 0; ch < nch; ++ch)
      split.insert(split.end(), {1, j * tcp::BN, 1, ch * tcp::KC, std::min(tcp::KC, K - ch * tcp::KC), blk++, N, 0});
  for (int i = 0; i < nrb; ++i)
    for (int j = 0; j < ncb; ++j) tiles.insert(tiles.end(), {2, i * tcp::BM, j * tcp::BN, M, N, i * nch, b0 + j * nch, nch});
  const int64_t offs[3] = {(int64_t)(A - C), (int64_t)(B - C), 0};
  const int32_t lds[3] = {lda, ldb, ldc};
  const size_t img_bytes = (size_t)blk * tcp::CHUNK_BYTES;
  const size_t items_bytes = (split.size() + tiles.size()) * sizeof(int32_t);
  const size_t tab_bytes = sizeof(offs) + sizeof(lds);
  unsigned char* buf = nullptr;
  VIV_CUDA(cudaMallocAsync((void**)&buf, img_bytes + items_bytes + tab_bytes + 256, s));
  unsigned char* img = buf;   // 256-byte aligned (allocation start)
  int32_t* d_split = reinterpret_cast<int32_t*>(buf + img_bytes);
  int32_t* d_tiles = d_split + split.size();
  int64_t* d_off = reinterpret_cast<int64_t*>(buf + ((img_bytes + items_bytes + 15) & ~size_t(15)));
  int32_t* d_ld = reinterpret_cast<int32_t*>(d_off + 3);
  std::vector<unsigned char> host(items_bytes);
  std::copy(reinterpret_cast<const unsigned char*>(split.data()),
            reinterpret_cast<const unsigned char*>(split.data() + split.size()), host.begin());
  std::copy(reinterpret_cast<const unsigned char*>(tiles.data()),
            reinterpret_cast<const unsigned char*>(tiles.data() + tiles.size()),
            host.begin() + split.size() * sizeof(int32_t));
  VIV_CUDA(cudaMemcpyAsync(d_split, host.data(), items_bytes, cudaMemcpyHostToDevice, s));
  VIV_CUDA(cudaMemcpyAsync(d_off, offs, sizeof(offs), cudaMemcpyHostToDevice, s));
  VIV_CUDA(cudaMemcpyAsync(d_ld, lds, sizeof(lds), cudaMemcpyHostToDevice, s));
  {
    Launched L(K_TCSPLIT, s);
    tcp::split_launch(d_split, blk, C, d_off, d_ld, img, nullptr, 0.f, s);
  }
  {
    Launched L(K_TCGEMM, s);
    tcp::pipe_launch(d_tiles, nrb * ncb, img, C, d_off, d_ld, err, s);
  }
  VIV_CUDA(cudaGetLastError());
  // the host copies above are synchronous with respect to `host` (pageable
  // memory is staged before cudaMemcpyAsync returns), so it may go out of scope
  VIV_CUDA(cudaFreeAsync(buf, s));
}

}  // namespace viv
