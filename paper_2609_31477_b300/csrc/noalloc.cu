// Allocation-free variant of the multifrontal triangular solve.
//
// Some callers must not allocate device memory while they run: a host
// framework that has already committed its memory pool and forbids growth
// during a time step, or a latency-sensitive loop that cannot afford
// cudaMalloc/cudaFree, which synchronise the device and stall other work.
// viv_lu_solve_noalloc serves them: it runs one forward + backward solve with
// the case's current factors, and the solve workspace (the front-local update
// vectors and the forward-solve vector) lives in the fixed array below
// instead of memory from the case's allocator.  The caller still provides
// the right-hand side and the solution buffers.
//
// The array is a module global: a GPU holds its NOALLOC_SCRATCH_BYTES from
// the moment this file's module is loaded on it until the process exits.
// Under lazy module loading (the CUDA default) that moment would be the first
// address lookup, which would make the first allocation-free call allocate;
// so every viv_case_create looks the address up (noalloc_prepare), once per
// device, while allocating is still allowed.  All calls share the array, and
// it keeps whatever the last call left in it.  The solve kernels write every
// workspace entry before reading it, so nothing needs clearing between
// calls.  Calls whose GPU work overlaps in time (different streams or
// threads) race on the array; callers must order them.
#include <cuda_runtime.h>

#include <mutex>

#include "viv_internal.h"

namespace viv {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(8) << 20;   // 8 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device (first call on that device) and cached.
void* scratch_address() {
  int dev = -1;
  VIV_CUDA(cudaGetDevice(&dev));
  VIV_CHECK(dev >= 0 && dev < MAX_DEVICES, VIV_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    VIV_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}
}  // namespace

// called by viv_case_create: commits the array on the current device
void noalloc_prepare() { (void)scratch_address(); }

void lu_solve_noalloc(vivCase* c, const double* b, double* x) {
  const Mesh& m = c->mesh->m;
  const bool f32 = c->prm.precision == VIV_MIXED;
  const size_t tsz = f32 ? sizeof(float) : sizeof(double);
  const size_t vec_bytes = ((size_t)m.vec_entries * tsz + 255) & ~size_t(255);
  const size_t yv_bytes = ((size_t)m.n_dofs * tsz + 255) & ~size_t(255);
  const bool border = m.n_front_dofs < m.n_dofs;
  const size_t need = vec_bytes + yv_bytes + (border ? 256 : 0);   // + the border's delta
  VIV_CHECK(need <= NOALLOC_SCRATCH_BYTES, VIV_ERR_ARG,
            "viv_lu_solve_noalloc: this mesh needs " + std::to_string(need) +
                " bytes of solve workspace, more than the fixed " + std::to_string(NOALLOC_SCRATCH_BYTES) +
                "-byte array; use viv_solve_rhs");
  unsigned char* base = static_cast<unsigned char*>(scratch_address());
  if (f32)
    solve_fronts<float>(m, (const float*)c->s.fronts, c->s.perm, b, x, (float*)base, (float*)(base + vec_bytes),
                        block_factors(c), c->s.chain, c->s.stats + 2, c->stream);
  else
    solve_fronts<double>(m, (const double*)c->s.fronts, c->s.perm, b, x, (double*)base,
                         (double*)(base + vec_bytes), false, nullptr, nullptr, c->stream);
  // the cylinder position through the FP64 border Schur block formed at factorisation
  if (border)
    launch_border_solve(m, c->s.J64, b, x, c->s.Y, c->s.Sb, (double*)(base + vec_bytes + yv_bytes), c->stream);
}

}  // namespace viv
