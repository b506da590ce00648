// Host helpers shared by the library's translation units: parameter checks,
// pointer kinds, sizes.
#pragma once
#include <cmath>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pflbm.h"

namespace pfl_host {

// The device of a context (the one that holds its workspace) is made current
// for the duration of a library call, and the caller's current device is
// given back when the call returns, on every return path, so that the
// caller's own CUDA calls keep going to the device it chose.  Nothing is
// switched when the two are the same device.
class DeviceScope {
 public:
  DeviceScope() = default;
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
  cudaError_t enter(int device) {
    cudaError_t e = cudaGetDevice(&saved_);
    if (e != cudaSuccess) {
      saved_ = -1;
      return e;
    }
    return saved_ == device ? cudaSuccess : cudaSetDevice(device);
  }
  ~DeviceScope() {
    int now = -1;
    if (saved_ >= 0 && cudaGetDevice(&now) == cudaSuccess && now != saved_) cudaSetDevice(saved_);
  }

 private:
  int saved_ = -1;
};

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

inline size_t pop_bytes(int prec) { return prec == PFL_FP64 ? 8 : prec == PFL_FP32 ? 4 : 2; }
inline size_t phi_bytes(int prec) { return prec == PFL_FP64 ? 8 : 4; }

// Velocities of the phase-field lattice: 27 (D3Q27), 9 (D2Q9, 2-D) or 15
// (D3Q15, also for 0); the hydrodynamic lattice is D2Q9 in 2-D, else D3Q27.
inline int qh_of(const pfl_params* p) { return p->h_lattice == 27 ? 27 : (p->h_lattice == 9 ? 9 : 15); }
inline int qg_of(const pfl_params* p) { return qh_of(p) == 9 ? 9 : 27; }

// The fused two-array step applies to MRT lattices with 32-bit indices.
inline bool uses_two_arrays(const pfl_params* p) {
  return p->engine == PFL_ENGINE_AUTO && p->collision == PFL_MRT &&
         27ull * (unsigned long long)p->nx * p->ny * p->nz < (1ull << 32);
}

inline std::string check_params(const pfl_params* p) {
  if (!p) return "params is NULL";
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return "dimensions must be >= 1";
  for (int a = 0; a < 3; ++a) {
    int lo = p->bc[2 * a], hi = p->bc[2 * a + 1];
    if ((lo != PFL_PERIODIC && lo != PFL_NOSLIP) || (hi != PFL_PERIODIC && hi != PFL_NOSLIP))
      return "unknown boundary kind";
    if (lo != hi) return "both faces of one axis must have the same kind";
  }
  if (!(p->rho_h > 0) || !(p->rho_l > 0)) return "densities must be > 0";
  if (!(p->mobility > 0)) return "mobility must be > 0";
  if (!(p->xi > 0)) return "interface width xi must be > 0";
  if (!(p->sigma >= 0)) return "sigma must be >= 0";
  const double wh = 1.0 / (3.0 * p->nu_h + 0.5), wl = 1.0 / (3.0 * p->nu_l + 0.5);
  const double wp = 1.0 / (3.0 * p->mobility + 0.5);
  if (!(wh > 0 && wh < 2) || !(wl > 0 && wl < 2)) return "relaxation rates of both phases must lie in (0, 2)";
  if (!(wp > 0 && wp < 2)) return "phase-field relaxation rate must lie in (0, 2)";
  if (p->precision < PFL_FP64 || p->precision > PFL_FP16S) return "unknown precision";
  if (p->collision != PFL_MRT && p->collision != PFL_BGK) return "unknown collision model";
  if (p->engine != PFL_ENGINE_AUTO && p->engine != PFL_ENGINE_INPLACE) return "unknown engine";
  if (p->h_lattice != 0 && p->h_lattice != 15 && p->h_lattice != 27 && p->h_lattice != 9)
    return "h_lattice must be 0, 15, 27 or 9";
  if (p->solids != 0 && p->solids != 1) return "solids must be 0 or 1";
  if (p->solids && !uses_two_arrays(p)) return "solid cells need the fused engine (MRT, engine AUTO)";
  if (p->h_lattice == 9 && (p->nz != 1 || p->bc[4] != PFL_PERIODIC))
    return "the 2-D lattices (h_lattice 9) need nz = 1 with periodic z faces";
  if (!std::isfinite(p->gravity[0]) || !std::isfinite(p->gravity[1]) || !std::isfinite(p->gravity[2]))
    return "gravity must be finite";
  if (p->hydrostatic != 0 && p->hydrostatic != 1) return "hydrostatic must be 0 or 1";
  if (p->hydrostatic) {
    const int axes = (p->gravity[0] != 0) + (p->gravity[1] != 0) + (p->gravity[2] != 0);
    if (axes != 1) return "the hydrostatic start needs gravity along exactly one axis";
    if (!std::isfinite(p->p_level)) return "p_level must be finite";
  }
  return "";
}

inline bool is_device_ptr(const void* ptr, int* device = nullptr) {
  if (!ptr) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (device) *device = a.device;
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Normalised pressure p* = p / (rho(phi) c_s^2) of the fluid at rest under
// gravity (the hydrostatic start of the paper's gravity cases): along every
// line of cells parallel to the gravity axis a, dp/ds = rho(phi) g_a is
// integrated by the trapezoid rule between cell centres,
//   P_0 = 0,  P_j = g_a * sum_{k < j} (rho_k + rho_{k+1}) / 2,
// then shifted so that p = 0 at s = level (linear interpolation between the
// cells j and j + 1 around it, j clamped to [0, n_a - 2]).  phi0 and out are
// N host doubles, x-fastest.
inline void hydrostatic_pstar(const pfl_params* p, const double* phi0, std::vector<double>& out) {
  const long long n[3] = {p->nx, p->ny, p->nz};
  const long long N = n[0] * n[1] * n[2];
  out.assign((size_t)N, 0.0);
  int a = 0;
  while (a < 2 && p->gravity[a] == 0) ++a;
  const double ga = p->gravity[a];
  const long long stride[3] = {1, n[0], n[0] * n[1]};
  const long long na = n[a];
  // the two axes across the lines
  const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
  std::vector<double> rho((size_t)na), P((size_t)na);
  long long j0 = (long long)std::floor(p->p_level);
  if (j0 > na - 2) j0 = na - 2;
  if (j0 < 0) j0 = 0;
  const double t = p->p_level - (double)j0;
  for (long long ic = 0; ic < n[c]; ++ic)
    for (long long ib = 0; ib < n[b]; ++ib) {
      const long long base = ib * stride[b] + ic * stride[c];
      for (long long j = 0; j < na; ++j)
        rho[(size_t)j] = p->rho_l + phi0[base + j * stride[a]] * (p->rho_h - p->rho_l);
      double acc = 0.0;
      P[0] = 0.0;
      for (long long j = 1; j < na; ++j) {
        acc += 0.5 * (rho[(size_t)j] + rho[(size_t)(j - 1)]);
        P[(size_t)j] = ga * acc;
      }
      const double ref = na > 1 ? (1.0 - t) * P[(size_t)j0] + t * P[(size_t)(j0 + 1)] : 0.0;
      for (long long j = 0; j < na; ++j) out[(size_t)(base + j * stride[a])] = 3.0 * (P[(size_t)j] - ref) / rho[(size_t)j];
    }
}

inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace pfl_host
