// Pipelined tcgen05 Schur-complement update (kind::tf32, 3xTF32) of the mixed
// path: C -= A B for lists of 128 x 128 tiles of column-major FP32 matrices.
//
// Two kernels per batch of tiles:
//   split : every 128 x 32 operand chunk (a row block of A or a column block
//           of B, one 32-wide slice of K) is read once, split into
//           hi = tf32(x) and lo = tf32(x - hi), and written to an image buffer
//           in the exact shared-memory layout the MMAs read (canonical K-major,
//           no swizzle: core matrices of 8 rows x 16 bytes): 32 KB per chunk,
//           hi then lo.
//   pipe  : persistent, warp-specialised.  One thread streams the image chunks
//           with bulk async copies (cp.async.bulk, completion counted in bytes
//           on an mbarrier): B through a three-stage ring, A through a
//           four-slot ring (kept while consecutive tiles share the row block);
//           one thread issues the MMAs (lo*hi + hi*lo + hi*hi per 8-wide K
//           step, FP32 accumulation in tensor memory) and commits each stage
//           back to the producer; four epilogue warps read finished
//           accumulators (tcgen05.ld) and update C in global memory.  Two
//           accumulators of 128 columns alternate, so the epilogue of one tile
//           (the C read-modify-write, the dominant memory traffic) overlaps the
//           MMAs of the next; each epilogue thread owns one tile row and keeps
//           64 loads of C in flight (two groups of 32 columns ahead), the first
//           of them issued before it waits for the accumulator, together with
//           L2 prefetches of its warp's rows of the next tile's C.
//
// Every wait is bounded.  A wait that expires sets *err and a shared abort
// flag that ends the other roles' waits; the MMA thread then waits (bounded)
// for its issued MMAs through one more commit, the producer for its bulk
// copies still in flight, and only then is tensor memory released.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tc_mma.cuh"

namespace viv {
namespace tcp {

using tc::BM;
using tc::BN;
using tc::CORE_BYTES;
using tc::KC;
using tc::KCORE_STRIDE;
using tc::OPERAND_BYTES;

constexpr int CHUNK_BYTES = 2 * OPERAND_BYTES;   // hi + lo of one 128 x 32 chunk: 32 KB
constexpr int MAX_CHUNKS = 4;                    // K <= 128 per update (the outer block)
constexpr int STAGES = 3;                        // ring of B chunks
// Six warps: with at most two warps per SM sub-partition each thread may use
// up to 255 registers, which the epilogue's C prefetch needs (no spills).
constexpr int EPI_WARPS = 4;
constexpr int THREADS = 32 * (2 + EPI_WARPS);    // warp 0 producer, warp 1 MMA, 2..5 epilogue
constexpr uint32_t TMEM_COLS = 256;              // two 128-column FP32 accumulators
constexpr int SPLIT_THREADS = 256;
constexpr int ITEM = 8;                          // ints per work item
constexpr long long WAIT_LIMIT = 1LL << 26;      // polls before a wait gives up
constexpr int PREFETCH_TILES = 1;                // tiles ahead whose C the epilogue prefetches into L2 (2: slower)

// work items
//   split: {f, start, kind (0: rows of A, 1: columns of B), k0, klen, block, limit, check}
//          operand element (r, k) of kind 0 is base[(k0 + k) ld + start + r],
//          of kind 1 base[(start + r) ld + k0 + k]; base = pool + off[f], ld = ld[f];
//          rows (columns) at or beyond `limit` and k >= klen are written as 0;
//          with check != 0 an element above 1 / thresh in magnitude (a
//          multiplier that fails the threshold test) adds 1 to stats[1]
//   pipe:  {f, rb, cb, r_end, c_end, a_block, b_block, nchunks}: one tile; C =
//          pool + off[f] with leading dimension ld[f]; rows < r_end and
//          columns < c_end of the tile are updated; chunk ch of A (B) is image
//          block a_block + ch (b_block + ch), nchunks <= MAX_CHUNKS.  CTA b
//          takes tiles b, b + grid, b + 2 grid, ...; two of them in a row with
//          the same a_block share the loaded A chunks.

// A chunks go through a ring of A_SLOTS slots: consecutive tiles of a CTA
// that share a row block (a segment) load its nchunks A chunks once into
// consecutive slots and keep them (segments with two chunks or fewer are
// double-buffered, longer ones refill slot by slot as their last tile
// releases it); B chunks go through a ring of STAGES slots.
constexpr int A_SLOTS = MAX_CHUNKS;
struct Smem {
  unsigned char a[A_SLOTS][CHUNK_BYTES];      // ring of A chunks [hi | lo], resident per segment
  unsigned char b[STAGES][CHUNK_BYTES];       // ring of B chunks [hi | lo]
  uint64_t full[STAGES];                      // bulk copy of the B slot landed (tx bytes)
  uint64_t empty[STAGES];                     // the B slot's MMAs finished (tcgen05.commit)
  uint64_t a_full[A_SLOTS];                   // bulk copy of the A slot landed
  uint64_t a_empty[A_SLOTS];                  // the last MMAs reading the A slot finished
  uint64_t acc_full[2];                       // accumulator complete (tcgen05.commit)
  uint64_t acc_empty[2];                      // accumulator read out (one arrival per epilogue warp)
  uint64_t drain;                             // final commit of the MMA thread
  uint32_t tmem_base;
  int abort_flag;
};
constexpr size_t SMEM_BYTES = sizeof(Smem) + 1024;   // + alignment of the ring to 1 KB

__device__ __forceinline__ bool aborted(const Smem& sm) {
  return *reinterpret_cast<const volatile int*>(&sm.abort_flag) != 0;
}

// bounded wait for the phase of the given parity; with `abortable` it also
// gives up as soon as another role has aborted
__device__ __forceinline__ bool wait_phase(Smem& sm, uint64_t* bar, uint32_t parity, bool abortable) {
  const uint32_t a = tc::smem_u32(bar);
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (abortable && (it & 255) == 255 && aborted(sm)) return false;
  }
  return false;
}

__device__ __forceinline__ void raise_abort(Smem& sm, int* err) {
  atomicExch(&sm.abort_flag, 1);
  atomicExch(err, 1);
}

__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst_smem)),
               "l"(src_gmem), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}

// host launchers (tc_pipe.cu); both enqueue on stream s
void split_launch(const int32_t* items, int n_items, const float* pool, const int64_t* off, const int32_t* ld,
                  unsigned char* img, int* stats, float thresh, cudaStream_t s);
void pipe_launch(const int32_t* items, int n_items, const unsigned char* img, float* pool, const int64_t* off,
                 const int32_t* ld, int* err, cudaStream_t s);
void prepare();   // kernel attributes of the current device (once per device)

}  // namespace tcp
}  // namespace viv
