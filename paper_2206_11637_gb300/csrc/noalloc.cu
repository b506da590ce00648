// Allocation-free variant of the phase-field reduction (pfl_phi_moments_static).
//
// Some callers of this library may not allocate device memory at all: a host
// application or framework that owns every byte of the GPU through its own
// pool or caching allocator (a cudaMalloc behind its back fragments the pool
// and can fail once the pool has claimed the memory), a plugin that is handed
// fixed buffers at set-up and no right to allocate afterwards, and a tight
// loop that cannot afford cudaMalloc's implicit device synchronisation.  For
// them this entry point computes the same sums as pfl_diag on a phi field they
// already hold, with its scratch in an array that is part of the loaded
// library image rather than in a workspace.
//
// The scratch is one file-scope __device__ array of PFL_STATIC_PARTIALS * 9 +
// 16 doubles (about 88 KB).  Every GPU that loads the library keeps its own
// copy until the process exits.  All calls on one device share it: calls whose
// kernels overlap on that GPU (different streams, or threads racing) corrupt
// each other's partial sums, so callers must order them.
#include <cmath>
#include <string>

#include "../../include/pflbm.h"
#include "errors.h"
#include "kernels.cuh"

using namespace pfl;

namespace {

constexpr int PFL_STATIC_PARTIALS = DIAG_BLOCKS;
constexpr long long PFL_STATIC_MAX_CELLS = 2147483647LL;  // coordinates are 32-bit

static __device__ __align__(256) double g_static_scratch[PFL_STATIC_PARTIALS * 9 + 16];

pfl_status sfail(pfl_status s, const std::string& m) {
  pfl_internal::set_error(m);
  return s;
}

// Device address of the static scratch on the current device.  Host code only
// sees a host-side stand-in for g_static_scratch; handing that to a kernel
// would fault or address the wrong memory, so the address is looked up with
// cudaGetSymbolAddress, with the device that holds phi current.  The lookup is
// repeated on every call (it is a table lookup once the library's module is
// loaded on the device): an address kept from an earlier call would be stale
// after the device's primary context was destroyed and created again
// (cudaDeviceReset).  The first call on a device loads the module there, so
// it belongs before any stream capture.
pfl_status scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return sfail(PFL_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = (double*)p;
  return PFL_OK;
}

// Makes `device` current for the lifetime of the guard and gives the caller's
// current device back on every return path.
struct DeviceGuard {
  int saved = -1;
  cudaError_t set(int device) {
    cudaError_t e = cudaGetDevice(&saved);
    if (e != cudaSuccess) {
      saved = -1;
      return e;
    }
    return saved == device ? cudaSuccess : cudaSetDevice(device);
  }
  ~DeviceGuard() {
    int now = -1;
    if (saved >= 0 && cudaGetDevice(&now) == cudaSuccess && now != saved) cudaSetDevice(saved);
  }
};

}  // namespace

extern "C" {

pfl_status pfl_phi_moments_static(const void* phi, int phi_fp64, int nx, int ny, int nz, double out[8],
                                  long long* nonfinite, void* stream) {
  if (!phi) return sfail(PFL_ERR_ARG, "phi is NULL");
  if (!out) return sfail(PFL_ERR_ARG, "out is NULL");
  if (nx < 1 || ny < 1 || nz < 1) return sfail(PFL_ERR_ARG, "dimensions must be >= 1");
  const long long N = (long long)nx * ny * nz;
  if (N > PFL_STATIC_MAX_CELLS)
    return sfail(PFL_ERR_ARG, "lattice has " + std::to_string(N) + " cells; this entry point accepts at most " +
                                  std::to_string(PFL_STATIC_MAX_CELLS));
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, phi) != cudaSuccess || (a.type != cudaMemoryTypeDevice &&
                                                           a.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return sfail(PFL_ERR_ARG, "phi must be device memory");
  }
  DeviceGuard dg;  // the kernels run on phi's device; the caller's current device is restored
  cudaError_t e = dg.set(a.device);
  if (e != cudaSuccess) return sfail(PFL_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  double* scratch = nullptr;
  pfl_status st = scratch_address(&scratch);
  if (st != PFL_OK) return st;

  Geo geo;
  geo.nx = nx;
  geo.ny = ny;
  geo.nz = nz;
  geo.wall[0] = geo.wall[1] = geo.wall[2] = 0;
  geo.N = N;
  cudaStream_t s = (cudaStream_t)stream;
  double* part = scratch;
  double* res = scratch + PFL_STATIC_PARTIALS * 9;
  // every partial slot is written by its block before the final sum reads it,
  // so the previous call's contents need no clearing
  if (phi_fp64)
    k_diag<double><<<PFL_STATIC_PARTIALS, DIAG_THREADS, 0, s>>>(geo, (const double*)phi, part);
  else
    k_diag<float><<<PFL_STATIC_PARTIALS, DIAG_THREADS, 0, s>>>(geo, (const float*)phi, part);
  k_diag_final<<<9, 32, 0, s>>>(part, PFL_STATIC_PARTIALS, res);
  e = cudaGetLastError();
  if (e != cudaSuccess) return sfail(PFL_ERR_CUDA, std::string("reduction launch: ") + cudaGetErrorString(e));
  double host[9];
  e = cudaMemcpyAsync(host, res, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return sfail(PFL_ERR_CUDA, std::string("reduction result: ") + cudaGetErrorString(e));
  for (int k = 0; k < 8; ++k) out[k] = host[k];
  const long long nf = (long long)host[8];
  if (nonfinite) *nonfinite = nf;
  if (nf > 0) return sfail(PFL_ERR_UNSTABLE, std::to_string(nf) + " cells hold a non-finite phi");
  return PFL_OK;
}

}  // extern "C"
