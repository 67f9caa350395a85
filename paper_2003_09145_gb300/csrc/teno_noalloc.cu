// teno_noalloc.cu -- teno_rhs_noalloc: the right-hand side for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's allocator or memory pool, plugin hosts that forbid device
// allocation on their threads, or deployments that must keep a fixed memory
// footprint.  They can still pass their own input and output arrays, but not
// the workspace that teno_rhs takes.  This entry point runs the same kernels
// as teno_rhs with the workspace carved from one file-scope device array of
// fixed size, so it never allocates.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "teno.h"
#include "teno_device.cuh"
#include "teno_launch.h"

namespace {

// The scratch array.  Every GPU that loads the library holds these bytes
// until the process exits.  Layout (all offsets 256-byte aligned):
//   [0, 256)        status word and the LF wave speeds (bit patterns)
//   [256, ...)      per-cell primitive variables, aux_fields(ndim) * ncell doubles
//   [..., end)      interface fluxes, nvar * max_d(#interfaces_d) doubles
static __device__ __align__(256) unsigned char g_noalloc_scratch[TENO_NOALLOC_SCRATCH_BYTES];

constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Device address of the scratch array on the current device.  In host code
// the symbol g_noalloc_scratch is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.  The cache
// does not survive cudaDeviceReset (the context that held the array is gone):
// a process that resets a device must not call teno_rhs_noalloc on it again.
teno_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TENO_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return TENO_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return TENO_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return TENO_OK;
}

bool grid_valid(const teno_grid* g) {
  if (!g || g->ndim < 1 || g->ndim > 3) return false;
  for (int k = 0; k < 3; ++k) {
    if (g->n[k] < 1 || (k >= g->ndim && g->n[k] != 1)) return false;
    if (k < g->ndim && (!(g->dx[k] > 0.0) || !(g->dx[k] < 1e300))) return false;
    if (k < g->ndim && g->bc[k] != TENO_BC_PERIODIC && g->bc[k] != TENO_BC_TRANSMISSIVE &&
        g->bc[k] != TENO_BC_REFLECTIVE)
      return false;
  }
  if (!(g->gamma > 1.0) || !(g->H > 0.0) || !(g->eps > 0.0)) return false;
  if (!std::isfinite(g->gamma) || !std::isfinite(g->H) || !std::isfinite(g->eps)) return false;
  if (g->b_l < 0 || g->b_u > 15 || g->b_u <= g->b_l) return false;
  if (!teno::scheme_fields_ok(g)) return false;
  for (int k = 0; k < g->ndim; ++k)
    if (!std::isfinite(g->grav[k])) return false;
  return true;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Bytes of the scratch array one call needs for grid g (SIZE_MAX if huge).
size_t scratch_needed(const teno_grid* g) {
  const double cells = double(g->n[0]) * double(g->n[1]) * double(g->n[2]);
  if (cells > double(TENO_NOALLOC_SCRATCH_BYTES)) return SIZE_MAX;
  const size_t ncell = size_t(g->n[0] * g->n[1] * g->n[2]);
  size_t maxifc = 0;
  for (int d = 0; d < g->ndim; ++d) {
    size_t m = 1;
    for (int k = 0; k < 3; ++k) m *= size_t(g->n[k] + (k == d ? 1 : 0));
    if (m > maxifc) maxifc = m;
  }
  return kAlign + round_up(sizeof(double) * teno::aux_fields(g->ndim) * ncell) +
         round_up(sizeof(double) * (g->ndim + 2) * maxifc);
}

}  // namespace

extern "C" teno_status teno_rhs_noalloc(const teno_grid* g, const double* U, double* dUdt,
                                        void* stream) {
  // fixed-state faces need a ghost block this variant does not hold
  if (g && g->ndim >= 1 && g->ndim <= 3)
    for (int k = 0; k < g->ndim; ++k)
      if (g->bc[k] == TENO_BC_DIRICHLET) return TENO_ERR_UNSUPPORTED;
  if (!grid_valid(g) || !U || !dUdt || U == dUdt) return TENO_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(U) % 16 || reinterpret_cast<uintptr_t>(dUdt) % 16)
    return TENO_ERR_INVALID_ARG;
  const size_t need = scratch_needed(g);
  if (need > TENO_NOALLOC_SCRATCH_BYTES) return TENO_ERR_WORKSPACE;
  if (!on_device(U) || !on_device(dUdt)) return TENO_ERR_INVALID_ARG;
  void* base = nullptr;
  teno_status s = scratch_address(&base);
  if (s != TENO_OK) return s;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(base);
  int* status = reinterpret_cast<int*>(ws);
  auto* alpha = reinterpret_cast<unsigned long long*>(ws + 64);
  const size_t ncell = size_t(g->n[0] * g->n[1] * g->n[2]);
  double* aux = reinterpret_cast<double*>(ws + kAlign);
  double* Fhat = reinterpret_cast<double*>(ws + kAlign + round_up(sizeof(double) * teno::aux_fields(g->ndim) * ncell));

  teno::Grid G;
  for (int k = 0; k < 3; ++k) {
    G.n[k] = g->n[k];
    G.bc[k] = k < g->ndim ? g->bc[k] : 0;
    G.dx[k] = k < g->ndim ? g->dx[k] : 1.0;
    G.inv_dx[k] = 1.0 / G.dx[k];
    G.rdx[k] = G.dx[0] / G.dx[k];
  }
  G.ncell = int64_t(ncell);
  for (int k = 0; k < g->ndim; ++k) {
    G.grav[k] = g->grav[k];
    if (g->grav[k] != 0.0) G.has_grav = 1;
  }
  const teno::Scheme S = teno::scheme_of(g);

  int nsm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    nsm = 152;

  // The array keeps the previous call's contents: the status word and the
  // wave-speed maxima must start from zero.
  if (cudaMemsetAsync(status, 0, 64 + sizeof(unsigned long long) * 9, st) != cudaSuccess)
    return TENO_ERR_CUDA;
  if (teno::launch_cell(g->ndim, U, aux, nullptr, alpha, status, G.ncell, g->gamma, nsm, st) != cudaSuccess)
    return TENO_ERR_CUDA;
  for (int d = 0; d < g->ndim; ++d) {
    if (teno::launch_flux(g->ndim, d, U, aux, nullptr, alpha, Fhat, nullptr, nullptr, nullptr, status, G, S, nsm, st,
                          nullptr) != cudaSuccess)
      return TENO_ERR_CUDA;
    if (teno::launch_diff(g->ndim, d, Fhat, dUdt, nullptr, nullptr, nullptr, nullptr, G, 0, nsm, st,
                          U) != cudaSuccess)
      return TENO_ERR_CUDA;
  }
  return TENO_OK;
}
