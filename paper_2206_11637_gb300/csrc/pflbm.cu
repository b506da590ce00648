// C interface of the PFLBM library (declared in include/pflbm.h).
//
// The library never allocates device memory: the caller hands in one
// workspace buffer, carved here into
//   [h populations | g populations | phi (two buffers) | FP64 staging (N) | reduction scratch]
// each section 256-byte aligned.  All kernels are queued on the caller's
// stream; calls returning data to the host synchronise that stream.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/pflbm.h"
#include "errors.h"
#include "kernels.cuh"
#include "step.cuh"

using namespace pfl;

namespace {

thread_local std::string g_err;

pfl_status fail(pfl_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

}  // namespace

namespace pfl_internal {
void set_error(const std::string& msg) { g_err = msg; }
}  // namespace pfl_internal

namespace {

pfl_status cuda_fail(cudaError_t e, const char* what) {
  return fail(PFL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

size_t pop_bytes(int prec) { return prec == PFL_FP64 ? 8 : prec == PFL_FP32 ? 4 : 2; }
size_t phi_bytes(int prec) { return prec == PFL_FP64 ? 8 : 4; }

struct Layout {
  size_t h, g, phi[2], stage, red, total;
};

Layout layout_of(const pfl_params* p) {
  Layout L;
  const size_t N = (size_t)p->nx * p->ny * p->nz;
  size_t off = 0;
  L.h = off;
  off = align256(off + 15 * N * pop_bytes(p->precision));
  L.g = off;
  off = align256(off + 27 * N * pop_bytes(p->precision));
  for (int b = 0; b < 2; ++b) {
    L.phi[b] = off;
    off = align256(off + N * phi_bytes(p->precision));
  }
  L.stage = off;
  off = align256(off + (N + 16) * sizeof(double));
  L.red = off;
  off = align256(off + (DIAG_BLOCKS * 9 + 16) * sizeof(double));
  L.total = off;
  return L;
}

std::string check_params(const pfl_params* p) {
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
  if (!std::isfinite(p->gravity[0]) || !std::isfinite(p->gravity[1]) || !std::isfinite(p->gravity[2]))
    return "gravity must be finite";
  return "";
}

bool is_device_ptr(const void* ptr, int* device = nullptr) {
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

unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

struct pfl_ctx {
  pfl_params p;
  Geo geo;
  Geo32 g32;
  bool idx32;    // 27 N < 2^32: the 32-bit indexed kernels apply
  Phys ph;
  Layout L;
  char* ws;
  cudaStream_t stream;
  int device;
  int cur;       // phi buffer holding phi^t; the other holds the shifts of the stored h
  long long t;   // steps taken
  int swapped;   // 1 after an even step (populations await the gather read)
};

namespace {

template <int PREC>
typename Store<PREC>::S* hbuf(pfl_ctx* c) {
  return (typename Store<PREC>::S*)(c->ws + c->L.h);
}
template <int PREC>
typename Store<PREC>::S* gbuf(pfl_ctx* c) {
  return (typename Store<PREC>::S*)(c->ws + c->L.g);
}
template <int PREC>
typename Store<PREC>::PhiT* phibuf(pfl_ctx* c, int b) {
  return (typename Store<PREC>::PhiT*)(c->ws + c->L.phi[b]);
}
template <int PREC>
typename Store<PREC>::PhiT* phicur(pfl_ctx* c) {
  return phibuf<PREC>(c, c->cur);
}
template <int PREC>
typename Store<PREC>::PhiT* phishift(pfl_ctx* c) {
  return phibuf<PREC>(c, 1 - c->cur);
}
double* stage(pfl_ctx* c) { return (double*)(c->ws + c->L.stage); }

// phi of the stored state into the spare buffer, then make it current.  The
// stored h carry the shifts of buffer `cur` (after a step) -- the spare buffer
// is free.
template <int PREC>
void launch_phi(pfl_ctx* c) {
  const unsigned nb = blocks_for(c->geo.N, 256);
  if (c->idx32) {
    if (c->swapped)
      k_phi32<PREC, 1><<<nb, 256, 0, c->stream>>>(c->g32, hbuf<PREC>(c), phicur<PREC>(c), phishift<PREC>(c));
    else
      k_phi32<PREC, 0><<<nb, 256, 0, c->stream>>>(c->g32, hbuf<PREC>(c), phicur<PREC>(c), phishift<PREC>(c));
  } else if (c->swapped)
    k_phi<PREC, 1><<<nb, 256, 0, c->stream>>>(c->geo, hbuf<PREC>(c), phicur<PREC>(c), phishift<PREC>(c));
  else
    k_phi<PREC, 0><<<nb, 256, 0, c->stream>>>(c->geo, hbuf<PREC>(c), phicur<PREC>(c), phishift<PREC>(c));
  c->cur = 1 - c->cur;
}

// One collide-stream launch (without the phi pass that completes the step).
// MRT runs the pair-based kernel; the BGK test mode, and lattices too large
// for 32-bit indices, the generic one.
template <int PREC, int BGK>
void step_only(pfl_ctx* c) {
  const unsigned nb = blocks_for(c->geo.N, 256);
  if (BGK || !c->idx32) {
    if (c->swapped)
      k_step<PREC, 1, 1><<<nb, 256, 0, c->stream>>>(c->geo, c->ph, hbuf<PREC>(c), gbuf<PREC>(c), phicur<PREC>(c),
                                                     phishift<PREC>(c));
    else
      k_step<PREC, 0, 1><<<nb, 256, 0, c->stream>>>(c->geo, c->ph, hbuf<PREC>(c), gbuf<PREC>(c), phicur<PREC>(c),
                                                     phishift<PREC>(c));
  } else {
    const unsigned nbm = blocks_for(c->geo.N, PFL_STEP_THREADS);
    if (c->swapped)
      k_step_mrt<PREC, 1><<<nbm, PFL_STEP_THREADS, 0, c->stream>>>(c->g32, c->ph, hbuf<PREC>(c), gbuf<PREC>(c), phicur<PREC>(c),
                                                      phishift<PREC>(c));
    else
      k_step_mrt<PREC, 0><<<nbm, PFL_STEP_THREADS, 0, c->stream>>>(c->g32, c->ph, hbuf<PREC>(c), gbuf<PREC>(c), phicur<PREC>(c),
                                                      phishift<PREC>(c));
  }
  c->swapped ^= 1;
  c->t += 1;
}

template <int PREC, int BGK>
void launch_steps(pfl_ctx* c, int n) {
  for (int s = 0; s < n; ++s) {
    step_only<PREC, BGK>(c);
    launch_phi<PREC>(c);
  }
}

// Fresh populations carry zero shifts (init / import).  Zero buffer 1, make it
// current so that launch_phi reads its shifts from it, and let launch_phi
// write phi into buffer 0 and make that one current.
template <int PREC>
pfl_status fresh_phi(pfl_ctx* c) {
  c->cur = 1;
  CUDA_TRY(cudaMemsetAsync(phicur<PREC>(c), 0, c->geo.N * sizeof(typename Store<PREC>::PhiT), c->stream));
  c->swapped = 0;
  launch_phi<PREC>(c);  // reads shifts from buffer 1 (zeros), writes phi into buffer 0, cur = 0
  CUDA_TRY(cudaGetLastError());
  return PFL_OK;
}

template <int PREC>
void launch_fields(pfl_ctx* c, double* o[6]) {
  const unsigned nb = blocks_for(c->geo.N, 256);
  if (c->swapped)
    k_fields<PREC, 1><<<nb, 256, 0, c->stream>>>(c->geo, c->ph, gbuf<PREC>(c), phicur<PREC>(c), o[0], o[1], o[2],
                                                  o[3], o[4], o[5]);
  else
    k_fields<PREC, 0><<<nb, 256, 0, c->stream>>>(c->geo, c->ph, gbuf<PREC>(c), phicur<PREC>(c), o[0], o[1], o[2],
                                                  o[3], o[4], o[5]);
}

template <int PREC>
void launch_export(pfl_ctx* c, int q, int i, double* out) {
  const unsigned nb = blocks_for(c->geo.N, 256);
  const typename Store<PREC>::S* f = (q == 27) ? gbuf<PREC>(c) : hbuf<PREC>(c);
  if (c->swapped)
    k_export<PREC, 1><<<nb, 256, 0, c->stream>>>(c->geo, f, phishift<PREC>(c), q, i, out);
  else
    k_export<PREC, 0><<<nb, 256, 0, c->stream>>>(c->geo, f, phishift<PREC>(c), q, i, out);
}

template <int PREC>
void launch_import(pfl_ctx* c, int q, int i, const double* in) {
  const unsigned nb = blocks_for(c->geo.N, 256);
  typename Store<PREC>::S* f = (q == 27) ? gbuf<PREC>(c) : hbuf<PREC>(c);
  k_import<PREC><<<nb, 256, 0, c->stream>>>(c->geo, f, q, i, in);
}

template <int PREC>
void launch_init(pfl_ctx* c, long long c0, long long count, const double* phi0, const double* ux, const double* uy,
                 const double* uz, const double* p0) {
  k_init<PREC><<<blocks_for(count, 256), 256, 0, c->stream>>>(c->geo, hbuf<PREC>(c), gbuf<PREC>(c), c0, count, phi0,
                                                               ux, uy, uz, p0);
}

template <int PREC>
void launch_diag(pfl_ctx* c, double* part, double* out) {
  k_diag<typename Store<PREC>::PhiT><<<DIAG_BLOCKS, DIAG_THREADS, 0, c->stream>>>(c->geo, phicur<PREC>(c), part);
  k_diag_final<<<9, 32, 0, c->stream>>>(part, DIAG_BLOCKS, out);
}

#define DISPATCH_PREC(c, fn, ...)                 \
  do {                                            \
    switch ((c)->p.precision) {                   \
      case PFL_FP64: fn<0>(__VA_ARGS__); break;   \
      case PFL_FP32: fn<1>(__VA_ARGS__); break;   \
      default: fn<2>(__VA_ARGS__); break;         \
    }                                             \
  } while (0)

// Copy n doubles from a host or device source into the device at dst.
pfl_status to_device(pfl_ctx* c, double* dst, const double* src, size_t n) {
  CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, c->stream));
  return PFL_OK;
}

}  // namespace

extern "C" {

int pfl_version(void) { return 1; }

const char* pfl_last_error(void) { return g_err.c_str(); }

size_t pfl_workspace_bytes(const pfl_params* p) {
  if (!check_params(p).empty()) return 0;
  return layout_of(p).total;
}

pfl_status pfl_init(const pfl_params* p, const double* phi0, const double* u0, const double* p0, void* workspace,
                    size_t workspace_bytes, void* stream, pfl_ctx** out) {
  if (!out) return fail(PFL_ERR_ARG, "out is NULL");
  *out = nullptr;
  std::string why = check_params(p);
  if (!why.empty()) return fail(PFL_ERR_ARG, why);
  if (!phi0) return fail(PFL_ERR_ARG, "phi0 is NULL");
  if (!workspace) return fail(PFL_ERR_ARG, "workspace is NULL");
  if (((uintptr_t)workspace & 255) != 0) return fail(PFL_ERR_ARG, "workspace must be 256-byte aligned");
  Layout L = layout_of(p);
  if (workspace_bytes < L.total)
    return fail(PFL_ERR_OOM, "workspace holds " + std::to_string(workspace_bytes) + " bytes, needs " +
                                 std::to_string(L.total));
  int device = 0;
  if (!is_device_ptr(workspace, &device)) return fail(PFL_ERR_ARG, "workspace is not device memory");
  CUDA_TRY(cudaSetDevice(device));

  pfl_ctx* c = new pfl_ctx();
  c->p = *p;
  c->device = device;
  c->L = L;
  c->ws = (char*)workspace;
  c->stream = (cudaStream_t)stream;
  c->t = 0;
  c->swapped = 0;
  c->cur = 0;
  c->geo.nx = p->nx;
  c->geo.ny = p->ny;
  c->geo.nz = p->nz;
  for (int a = 0; a < 3; ++a) c->geo.wall[a] = p->bc[2 * a] == PFL_NOSLIP ? 1 : 0;
  c->geo.N = (long long)p->nx * p->ny * p->nz;
  c->idx32 = 27ull * (unsigned long long)c->geo.N < (1ull << 32);
  c->g32.nx = p->nx;
  c->g32.ny = p->ny;
  c->g32.nz = p->nz;
  c->g32.N = (unsigned)(c->idx32 ? c->geo.N : 0);
  c->g32.dx = make_fastdiv((unsigned)p->nx);
  c->g32.dy = make_fastdiv((unsigned)p->ny);
  for (int a = 0; a < 3; ++a) c->g32.wall[a] = c->geo.wall[a];
  if (c->idx32 && (!fastdiv_ok((unsigned)p->nx, (unsigned)c->geo.N) ||
                   !fastdiv_ok((unsigned)p->ny, (unsigned)(c->geo.N / p->nx)))) {
    delete c;
    return fail(PFL_ERR_STATE, "integer divider self-check failed");
  }
  c->ph.rho_h = p->rho_h;
  c->ph.rho_l = p->rho_l;
  c->ph.tau_h = 3.0 * p->nu_h + 0.5;
  c->ph.tau_l = 3.0 * p->nu_l + 0.5;
  c->ph.beta = 12.0 * p->sigma / p->xi;
  c->ph.kappa = 1.5 * p->sigma * p->xi;
  c->ph.inv_xi = 1.0 / p->xi;
  c->ph.omega_phi = 1.0 / (3.0 * p->mobility + 0.5);
  c->ph.gx = p->gravity[0];
  c->ph.gy = p->gravity[1];
  c->ph.gz = p->gravity[2];

  // Initial state, in chunks through the FP64 staging area (5 arrays per chunk).
  const long long N = c->geo.N;
  const long long chunk = N / 5 > 0 ? N / 5 : 1;  // 5 * chunk <= N + 16 staging doubles
  double* st = stage(c);
  for (long long c0 = 0; c0 < N; c0 += chunk) {
    const long long cnt = (N - c0 < chunk) ? N - c0 : chunk;
    double* a_phi = st;
    double* a_ux = st + cnt;
    double* a_uy = st + 2 * cnt;
    double* a_uz = st + 3 * cnt;
    double* a_p = st + 4 * cnt;
    pfl_status s;
    if ((s = to_device(c, a_phi, phi0 + c0, cnt)) != PFL_OK) {
      delete c;
      return s;
    }
    if (u0) {
      if ((s = to_device(c, a_ux, u0 + c0, cnt)) != PFL_OK || (s = to_device(c, a_uy, u0 + N + c0, cnt)) != PFL_OK ||
          (s = to_device(c, a_uz, u0 + 2 * N + c0, cnt)) != PFL_OK) {
        delete c;
        return s;
      }
    }
    if (p0) {
      if ((s = to_device(c, a_p, p0 + c0, cnt)) != PFL_OK) {
        delete c;
        return s;
      }
    }
    DISPATCH_PREC(c, launch_init, c, c0, cnt, a_phi, u0 ? a_ux : nullptr, u0 ? a_uy : nullptr, u0 ? a_uz : nullptr,
                  p0 ? a_p : nullptr);
    // the staging area is reused by the next chunk: wait for this one
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "initialisation");
    }
  }
  pfl_status s = PFL_OK;
  switch (c->p.precision) {
    case PFL_FP64: s = fresh_phi<0>(c); break;
    case PFL_FP32: s = fresh_phi<1>(c); break;
    default: s = fresh_phi<2>(c); break;
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (s != PFL_OK || e != cudaSuccess) {
    delete c;
    return s != PFL_OK ? s : cuda_fail(e, "initial phi");
  }
  *out = c;
  return PFL_OK;
}

pfl_status pfl_step(pfl_ctx* c, int n) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  CUDA_TRY(cudaSetDevice(c->device));
  if (n < 0) return fail(PFL_ERR_ARG, "n_steps must be >= 0");
  if (n == 0) return PFL_OK;
  const bool bgk = c->p.collision == PFL_BGK;
  switch (c->p.precision) {
    case PFL_FP64: bgk ? launch_steps<0, 1>(c, n) : launch_steps<0, 0>(c, n); break;
    case PFL_FP32: bgk ? launch_steps<1, 1>(c, n) : launch_steps<1, 0>(c, n); break;
    default: bgk ? launch_steps<2, 1>(c, n) : launch_steps<2, 0>(c, n); break;
  }
  CUDA_TRY(cudaGetLastError());
  return PFL_OK;
}

pfl_status pfl_fields(pfl_ctx* c, double* phi, double* rho, double* p, double* u) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  CUDA_TRY(cudaSetDevice(c->device));
  const long long N = c->geo.N;
  double* want[6] = {phi, rho, p, u, u ? u + N : nullptr, u ? u + 2 * N : nullptr};
  double* dev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool host[6];
  for (int k = 0; k < 6; ++k) {
    host[k] = want[k] && !is_device_ptr(want[k]);
    if (want[k] && !host[k]) dev[k] = want[k];
  }
  // device outputs in one pass
  bool any_dev = false;
  for (int k = 0; k < 6; ++k) any_dev |= dev[k] != nullptr;
  if (any_dev) DISPATCH_PREC(c, launch_fields, c, dev);
  // host outputs one at a time through the staging area
  for (int k = 0; k < 6; ++k) {
    if (!host[k]) continue;
    double* o[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    o[k] = stage(c);
    DISPATCH_PREC(c, launch_fields, c, o);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(want[k], stage(c), N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PFL_OK;
}

pfl_status pfl_populations(pfl_ctx* c, double* h, double* g) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  CUDA_TRY(cudaSetDevice(c->device));
  const long long N = c->geo.N;
  for (int set = 0; set < 2; ++set) {
    double* dst = set == 0 ? h : g;
    if (!dst) continue;
    const int q = set == 0 ? 15 : 27;
    const bool dev = is_device_ptr(dst);
    for (int i = 0; i < q; ++i) {
      double* o = dev ? dst + (size_t)i * N : stage(c);
      DISPATCH_PREC(c, launch_export, c, q, i, o);
      CUDA_TRY(cudaGetLastError());
      if (!dev) {
        CUDA_TRY(cudaMemcpyAsync(dst + (size_t)i * N, o, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
      }
    }
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PFL_OK;
}

pfl_status pfl_set_populations(pfl_ctx* c, const double* h, const double* g) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  CUDA_TRY(cudaSetDevice(c->device));
  if (!h || !g) return fail(PFL_ERR_ARG, "both population sets are required");
  const long long N = c->geo.N;
  // read the complete current state first when only part would change: not
  // needed, both sets are replaced; the layout becomes the normal one.
  for (int set = 0; set < 2; ++set) {
    const double* src = set == 0 ? h : g;
    const int q = set == 0 ? 15 : 27;
    for (int i = 0; i < q; ++i) {
      CUDA_TRY(cudaMemcpyAsync(stage(c), src + (size_t)i * N, N * sizeof(double), cudaMemcpyDefault, c->stream));
      DISPATCH_PREC(c, launch_import, c, q, i, stage(c));
      CUDA_TRY(cudaGetLastError());
      CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
  }
  pfl_status s = PFL_OK;
  switch (c->p.precision) {
    case PFL_FP64: s = fresh_phi<0>(c); break;
    case PFL_FP32: s = fresh_phi<1>(c); break;
    default: s = fresh_phi<2>(c); break;
  }
  if (s != PFL_OK) return s;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PFL_OK;
}

pfl_status pfl_diag(pfl_ctx* c, double out[8], long long* nonfinite) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  CUDA_TRY(cudaSetDevice(c->device));
  double* part = (double*)(c->ws + c->L.red);
  double* res = part + DIAG_BLOCKS * 9;
  DISPATCH_PREC(c, launch_diag, c, part, res);
  CUDA_TRY(cudaGetLastError());
  double host[9];
  CUDA_TRY(cudaMemcpyAsync(host, res, sizeof(host), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (out)
    for (int k = 0; k < 8; ++k) out[k] = host[k];
  long long nf = (long long)host[8];
  if (nonfinite) *nonfinite = nf;
  if (nf > 0) return fail(PFL_ERR_UNSTABLE, std::to_string(nf) + " cells hold a non-finite phi");
  return PFL_OK;
}

pfl_status pfl_kernel_times(pfl_ctx* c, int n, double ms[2]) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  if (n <= 0 || !ms) return fail(PFL_ERR_ARG, "n_steps must be > 0 and ms non-NULL");
  CUDA_TRY(cudaSetDevice(c->device));
  cudaEvent_t ev[3];
  for (int k = 0; k < 3; ++k) CUDA_TRY(cudaEventCreate(&ev[k]));
  double acc[2] = {0, 0};
  const bool bgk = c->p.collision == PFL_BGK;
  pfl_status st = PFL_OK;
  for (int s = 0; s < n && st == PFL_OK; ++s) {
    cudaEventRecord(ev[0], c->stream);
    switch (c->p.precision) {
      case PFL_FP64: bgk ? step_only<0, 1>(c) : step_only<0, 0>(c); break;
      case PFL_FP32: bgk ? step_only<1, 1>(c) : step_only<1, 0>(c); break;
      default: bgk ? step_only<2, 1>(c) : step_only<2, 0>(c); break;
    }
    cudaEventRecord(ev[1], c->stream);
    DISPATCH_PREC(c, launch_phi, c);
    cudaEventRecord(ev[2], c->stream);
    cudaError_t e = cudaEventSynchronize(ev[2]);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      st = cuda_fail(e, "timed step");
      break;
    }
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    acc[0] += a;
    acc[1] += b;
  }
  for (int k = 0; k < 3; ++k) cudaEventDestroy(ev[k]);
  ms[0] = acc[0];
  ms[1] = acc[1];
  return st;
}

long long pfl_time(const pfl_ctx* c) { return c ? c->t : -1; }

void pfl_destroy(pfl_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  delete c;
}

}  // extern "C"
