// C interface of the PFLBM library (declared in include/pflbm.h).
//
// The library never allocates device memory: the caller hands in one
// workspace buffer, carved here into
//   [h populations | g populations | phi (two buffers) | FP64 staging (N) | reduction scratch]
// each section 256-byte aligned.  All kernels are queued on the caller's
// stream; calls returning data to the host synchronise that stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pflbm.h"
#include "errors.h"
#include "host_common.h"
#include "kernels.cuh"
#include "step.cuh"
#include "adjoint.cuh"

using namespace pfl;
using namespace pfl_host;

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



struct Layout {
  size_t h, g, h2, g2, phi[2], pg[2], links, stage, red, clock, total;
};

Layout layout_of(const pfl_params* p) {
  Layout L;
  const size_t N = (size_t)p->nx * p->ny * p->nz;
  size_t off = 0;
  const size_t QH = (size_t)qh_of(p);
  L.h = off;
  off = align256(off + QH * N * pop_bytes(p->precision));
  L.g = off;
  off = align256(off + (size_t)qg_of(p) * N * pop_bytes(p->precision));
  L.h2 = L.g2 = 0;
  if (uses_two_arrays(p)) {  // second array pair of the fused two-array step
    L.h2 = off;
    off = align256(off + QH * N * pop_bytes(p->precision));
    L.g2 = off;
    off = align256(off + (size_t)qg_of(p) * N * pop_bytes(p->precision));
  }
  for (int b = 0; b < 2; ++b) {
    L.phi[b] = off;
    off = align256(off + N * phi_bytes(p->precision));
  }
  // FP16S: the p* shifts of the stored g (one FP16 per cell, double-buffered
  // like phi)
  for (int b = 0; b < 2; ++b) {
    L.pg[b] = off;
    if (p->precision == PFL_FP16S) off = align256(off + N * sizeof(__half));
  }
  L.links = off;  // blocked-link words of solid lattices
  if (p->solids) off = align256(off + N * sizeof(unsigned));
  L.stage = off;
  off = align256(off + (N + 16) * sizeof(double));
  L.red = off;  // phi partials (9 per block), results, flow-speed partials (1 per block), result
  off = align256(off + (DIAG_BLOCKS * 10 + 32) * sizeof(double));
  L.clock = off;  // step count read by graph-replayed steps
  off = align256(off + sizeof(unsigned long long));
  L.total = off;
  return L;
}




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
  bool zm;       // fused two-array step (else in-place AA + phi pass)
  int ab;        // two-array step: 0 = first pair current, 1 = second
  bool stale;    // two-array step: phi of the current state not yet materialised
  int zc;        // two-array step: z planes per block
  long long t;   // steps taken
  int swapped;   // 1 after an even step (populations await the gather read)
  int qh;        // phase-field lattice: 15, 27 or 9 velocities
  int qg;        // hydrodynamic lattice: 27, or 9 in 2-D
  bool solid;    // solid cells set (pfl_set_solid): the fused step reads the link words
  // CUDA graphs of graph_k fused steps, one per (ab, cur) state at capture;
  // replays read the step count from the workspace clock
  int graph_k;
  cudaGraphExec_t gx[4];
  cudaStream_t cap;         // capture stream (created on first use)
  bool capturing;           // launches are being captured: pass the clock
  long long cap_t0;         // step count when the capture began
  long long clock_t;        // step count the device clock holds (-1: unknown)
};

namespace {

// current populations (the two-array step alternates between two pairs)
template <int PREC>
typename Store<PREC>::S* hbuf(pfl_ctx* c) {
  return (typename Store<PREC>::S*)(c->ws + (c->zm && c->ab ? c->L.h2 : c->L.h));
}
template <int PREC>
typename Store<PREC>::S* gbuf(pfl_ctx* c) {
  return (typename Store<PREC>::S*)(c->ws + (c->zm && c->ab ? c->L.g2 : c->L.g));
}
template <int PREC>
typename Store<PREC>::S* hnext(pfl_ctx* c) {
  return (typename Store<PREC>::S*)(c->ws + (c->ab ? c->L.h : c->L.h2));
}
template <int PREC>
typename Store<PREC>::S* gnext(pfl_ctx* c) {
  return (typename Store<PREC>::S*)(c->ws + (c->ab ? c->L.g : c->L.g2));
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
// FP16S p* shifts: pgshift holds those of the stored g (read by a step),
// pgcur receives those of the g a step writes (same parity as phi); NULL for
// the other precisions.
__half* pgbuf(pfl_ctx* c, int b) { return c->p.precision == PFL_FP16S ? (__half*)(c->ws + c->L.pg[b]) : nullptr; }
__half* pgcur(pfl_ctx* c) { return pgbuf(c, c->cur); }
__half* pgshift(pfl_ctx* c) { return pgbuf(c, 1 - c->cur); }
double* stage(pfl_ctx* c) { return (double*)(c->ws + c->L.stage); }

// seed of the FP16 stochastic rounding of one step
unsigned step_seed(const pfl_ctx* c) { return step_seed_of((unsigned long long)c->t); }
unsigned long long* clock_of(pfl_ctx* c) { return (unsigned long long*)(c->ws + c->L.clock); }

// the device step count: set (add = 0) or advance (add = 1)
__global__ void k_clock(unsigned long long* t, long long v, int add) {
  if (add)
    *t += (unsigned long long)v;
  else
    *t = (unsigned long long)v;
}

// phi of the stored state into the spare buffer, then make it current.  The
// stored h carry the shifts of buffer `cur` (after a step) -- the spare buffer
// is free.
template <int PREC, int QH>
void launch_phi(pfl_ctx* c) {
  const unsigned nb = blocks_for(c->geo.N, 256);
  if (c->idx32) {
    const unsigned* links = c->solid ? (const unsigned*)(c->ws + c->L.links) : nullptr;
    if (c->swapped)
      k_phi32<PREC, QH, 1><<<nb, 256, 0, c->stream>>>(c->g32, hbuf<PREC>(c), phicur<PREC>(c), phishift<PREC>(c), links);
    else
      k_phi32<PREC, QH, 0><<<nb, 256, 0, c->stream>>>(c->g32, hbuf<PREC>(c), phicur<PREC>(c), phishift<PREC>(c), links);
  } else if (c->swapped)
    k_phi<PREC, QH, 1><<<nb, 256, 0, c->stream>>>(c->geo, hbuf<PREC>(c), phicur<PREC>(c), phishift<PREC>(c));
  else
    k_phi<PREC, QH, 0><<<nb, 256, 0, c->stream>>>(c->geo, hbuf<PREC>(c), phicur<PREC>(c), phishift<PREC>(c));
  c->cur = 1 - c->cur;
}

// One collide-stream launch (without the phi pass that completes an in-place
// step).  Two-array contexts run the fused kernel; MRT in place the pair-based
// kernel; the BGK test mode, and lattices too large for 32-bit indices, the
// generic one.
template <int PREC, int QH, int BGK>
void step_only(pfl_ctx* c) {
  const unsigned nb = blocks_for(c->geo.N, 256);
  if (c->zm) {
    const int ty = zm_ty(c->p.nz == 1);
    const dim3 grid((c->p.nx + ZM_TX - 1) / ZM_TX, (c->p.ny + ty - 1) / ty, (c->p.nz + c->zc - 1) / c->zc);
    const dim3 block(ZM_TX, ty);
    const unsigned* links = (const unsigned*)(c->ws + c->L.links);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = c->stream;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = PFL_ZM_PDL ? 1 : 0;
    const typename Store<PREC>::S* ha = hbuf<PREC>(c);
    const typename Store<PREC>::S* ga = gbuf<PREC>(c);
    const typename Store<PREC>::PhiT* shift = phishift<PREC>(c);
    const unsigned long long* tclock = c->capturing ? clock_of(c) : nullptr;
    const int tofs = (int)(c->t - c->cap_t0);
#define PFL_ZM(FLAT, SOLID)                                                                                   \
  cudaLaunchKernelEx(&cfg, k_step_zm<PREC, QH, FLAT, SOLID>, c->g32, c->ph, ha, ga, hnext<PREC>(c),           \
                     gnext<PREC>(c), shift, phicur<PREC>(c), c->zc, step_seed(c), links, tclock, tofs,       \
                     (const __half*)pgshift(c), pgcur(c))
    if (c->p.nz == 1) {
      if (c->solid)
        PFL_ZM(1, 1);
      else
        PFL_ZM(1, 0);
    } else {
      if (c->solid)
        PFL_ZM(0, 1);
      else
        PFL_ZM(0, 0);
    }
#undef PFL_ZM
    // phicur now holds phi^t, the shift of the populations just written
    c->ab ^= 1;
    c->cur = 1 - c->cur;
    c->stale = true;
    c->t += 1;
    return;
  }
  if (BGK || !c->idx32) {
    if (c->swapped)
      k_step<PREC, QH, 1, BGK><<<nb, 256, 0, c->stream>>>(c->geo, c->ph, hbuf<PREC>(c), gbuf<PREC>(c), phicur<PREC>(c),
                                                       phishift<PREC>(c), pgshift(c), pgcur(c));
    else
      k_step<PREC, QH, 0, BGK><<<nb, 256, 0, c->stream>>>(c->geo, c->ph, hbuf<PREC>(c), gbuf<PREC>(c), phicur<PREC>(c),
                                                       phishift<PREC>(c), pgshift(c), pgcur(c));
  } else {
    const unsigned nbm = blocks_for(c->geo.N, PFL_STEP_THREADS);
    if (c->swapped)
      k_step_mrt<PREC, QH, 1><<<nbm, PFL_STEP_THREADS, 0, c->stream>>>(c->g32, c->ph, hbuf<PREC>(c), gbuf<PREC>(c),
                                                                    phicur<PREC>(c), phishift<PREC>(c), step_seed(c),
                                                                    pgshift(c), pgcur(c));
    else
      k_step_mrt<PREC, QH, 0><<<nbm, PFL_STEP_THREADS, 0, c->stream>>>(c->g32, c->ph, hbuf<PREC>(c), gbuf<PREC>(c),
                                                                    phicur<PREC>(c), phishift<PREC>(c), step_seed(c),
                                                                    pgshift(c), pgcur(c));
  }
  c->swapped ^= 1;
  c->t += 1;
}

// phi of the current state of a two-array context into the current buffer
// (the same sum the next fused step forms in shared memory).
template <int PREC, int QH>
void ensure_phi(pfl_ctx* c) {
  if (!c->zm || !c->stale) return;
  k_phi32<PREC, QH, 0><<<blocks_for(c->geo.N, 256), 256, 0, c->stream>>>(
      c->g32, hbuf<PREC>(c), phishift<PREC>(c), phicur<PREC>(c),
      c->solid ? (const unsigned*)(c->ws + c->L.links) : nullptr);
  c->stale = false;
}

// completes a step: the phi pass in place, nothing for the fused step
template <int PREC, int QH>
void after_step(pfl_ctx* c) {
  if (!c->zm) launch_phi<PREC, QH>(c);
}

// one collide-stream launch in the context's collision mode
template <int PREC, int QH>
void step_any(pfl_ctx* c) {
  if (c->p.collision == PFL_BGK)
    step_only<PREC, QH, 1>(c);
  else
    step_only<PREC, QH, 0>(c);
}

template <int PREC, int QH>
void launch_steps(pfl_ctx* c, int n) {
  for (int s = 0; s < n; ++s) {
    step_any<PREC, QH>(c);
    after_step<PREC, QH>(c);
  }
}

// Fresh populations (init, import) carry the shifts of buffer 1: the
// initial phi and p* written by k_init, or zeros (zero_shifts, for imported
// populations).  Make buffer 1 current so that launch_phi reads its shifts from
// it, and let launch_phi write phi into buffer 0 and make that one current.
template <int PREC, int QH>
pfl_status fresh_phi(pfl_ctx* c, bool zero_shifts) {
  c->stale = false;
  c->cur = 1;
  if (zero_shifts) {
    CUDA_TRY(cudaMemsetAsync(phicur<PREC>(c), 0, c->geo.N * sizeof(typename Store<PREC>::PhiT), c->stream));
    if (pgbuf(c, 1)) CUDA_TRY(cudaMemsetAsync(pgbuf(c, 1), 0, c->geo.N * sizeof(__half), c->stream));
  }
  c->swapped = 0;
  launch_phi<PREC, QH>(c);  // reads shifts from buffer 1 (zeros), writes phi into buffer 0, cur = 0
  CUDA_TRY(cudaGetLastError());
  return PFL_OK;
}

template <int PREC, int QH>
void launch_fields(pfl_ctx* c, double* o[6]) {
  const unsigned nb = blocks_for(c->geo.N, 256);
  const unsigned* links = (const unsigned*)(c->ws + c->L.links);
  if (c->swapped)
    k_fields<PREC, QH, 1><<<nb, 256, 0, c->stream>>>(c->geo, c->ph, gbuf<PREC>(c), phicur<PREC>(c), o[0],
                                                  o[1], o[2], o[3], o[4], o[5], c->solid ? links : nullptr,
                                                  pgshift(c));
  else
    k_fields<PREC, QH, 0><<<nb, 256, 0, c->stream>>>(c->geo, c->ph, gbuf<PREC>(c), phicur<PREC>(c), o[0],
                                                  o[1], o[2], o[3], o[4], o[5], c->solid ? links : nullptr,
                                                  pgshift(c));
}

template <int PREC, int QH>
void launch_export(pfl_ctx* c, int is_g, int i, double* out) {
  const unsigned nb = blocks_for(c->geo.N, 256);
  const typename Store<PREC>::S* f = is_g ? gbuf<PREC>(c) : hbuf<PREC>(c);
  if (c->swapped)
    k_export<PREC, QH, 1><<<nb, 256, 0, c->stream>>>(c->geo, f, phishift<PREC>(c), is_g, i, out, pgshift(c));
  else
    k_export<PREC, QH, 0><<<nb, 256, 0, c->stream>>>(c->geo, f, phishift<PREC>(c), is_g, i, out, pgshift(c));
}

template <int PREC, int QH>
void launch_import(pfl_ctx* c, int is_g, int i, const double* in) {
  const unsigned nb = blocks_for(c->geo.N, 256);
  typename Store<PREC>::S* f = is_g ? gbuf<PREC>(c) : hbuf<PREC>(c);
  k_import<PREC, QH><<<nb, 256, 0, c->stream>>>(c->geo, f, is_g, i, in);
}

template <int PREC, int QH>
void launch_init(pfl_ctx* c, long long c0, long long count, const double* phi0, const double* ux, const double* uy,
                 const double* uz, const double* p0) {
  // FP16S: stored against the writers' shifts, which k_init_shift has put into
  // buffer 1 (fresh_phi reads them there)
  const float* hs = PREC == 2 ? (const float*)phibuf<PREC>(c, 1) : nullptr;
  k_init<PREC, QH><<<blocks_for(count, 256), 256, 0, c->stream>>>(c->geo, hbuf<PREC>(c), gbuf<PREC>(c), c0, count, phi0,
                                                               ux, uy, uz, p0, hs, pgbuf(c, 1));
}

template <int PREC>
void launch_diag(pfl_ctx* c, double* part, double* out) {
  k_diag<typename Store<PREC>::PhiT><<<DIAG_BLOCKS, DIAG_THREADS, 0, c->stream>>>(c->geo, phicur<PREC>(c), part);
  k_diag_final<<<9, 32, 0, c->stream>>>(part, DIAG_BLOCKS, out);
}

// Largest |u| of the current state into out[0] (partials in part[0 .. DIAG_BLOCKS)).
template <int PREC, int QH>
void launch_umax(pfl_ctx* c, double* part, double* out) {
  const unsigned* links = c->solid ? (const unsigned*)(c->ws + c->L.links) : nullptr;
  if (c->swapped)
    k_umax<PREC, QH, 1><<<DIAG_BLOCKS, DIAG_THREADS, 0, c->stream>>>(c->geo, c->ph, gbuf<PREC>(c), phicur<PREC>(c),
                                                                     part, links, pgshift(c));
  else
    k_umax<PREC, QH, 0><<<DIAG_BLOCKS, DIAG_THREADS, 0, c->stream>>>(c->geo, c->ph, gbuf<PREC>(c), phicur<PREC>(c),
                                                                     part, links, pgshift(c));
  k_max_final<<<1, 32, 0, c->stream>>>(part, DIAG_BLOCKS, out);
}

#define DISPATCH_PREC(c, fn, ...)                 \
  do {                                            \
    switch ((c)->p.precision) {                   \
      case PFL_FP64: fn<0>(__VA_ARGS__); break;   \
      case PFL_FP32: fn<1>(__VA_ARGS__); break;   \
      default: fn<2>(__VA_ARGS__); break;         \
    }                                             \
  } while (0)

// fn<PREC, QH>(...) for the context's precision and phase-field lattice
#define DISPATCH(c, fn, ...)                                                  \
  do {                                                                        \
    const int qh_ = (c)->qh;                                                  \
    switch ((c)->p.precision) {                                               \
      case PFL_FP64:                                                          \
        if (qh_ == 27) fn<0, 27>(__VA_ARGS__);                                \
        else if (qh_ == 9) fn<0, 9>(__VA_ARGS__);                             \
        else fn<0, 15>(__VA_ARGS__);                                          \
        break;                                                                \
      case PFL_FP32:                                                          \
        if (qh_ == 27) fn<1, 27>(__VA_ARGS__);                                \
        else if (qh_ == 9) fn<1, 9>(__VA_ARGS__);                             \
        else fn<1, 15>(__VA_ARGS__);                                          \
        break;                                                                \
      default:                                                                \
        if (qh_ == 27) fn<2, 27>(__VA_ARGS__);                                \
        else if (qh_ == 9) fn<2, 9>(__VA_ARGS__);                             \
        else fn<2, 15>(__VA_ARGS__);                                          \
        break;                                                                \
    }                                                                         \
  } while (0)

// s = fn<PREC, QH>(...)
#define DISPATCH_S(s, c, fn, ...)                                             \
  do {                                                                        \
    const int qh_ = (c)->qh;                                                  \
    switch ((c)->p.precision) {                                               \
      case PFL_FP64: s = qh_ == 27 ? fn<0, 27>(__VA_ARGS__) : qh_ == 9 ? fn<0, 9>(__VA_ARGS__) : fn<0, 15>(__VA_ARGS__); break; \
      case PFL_FP32: s = qh_ == 27 ? fn<1, 27>(__VA_ARGS__) : qh_ == 9 ? fn<1, 9>(__VA_ARGS__) : fn<1, 15>(__VA_ARGS__); break; \
      default: s = qh_ == 27 ? fn<2, 27>(__VA_ARGS__) : qh_ == 9 ? fn<2, 9>(__VA_ARGS__) : fn<2, 15>(__VA_ARGS__); break;       \
    }                                                                         \
  } while (0)

// Copy n doubles from a host or device source into the device at dst.
pfl_status to_device(pfl_ctx* c, double* dst, const double* src, size_t n) {
  CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, c->stream));
  return PFL_OK;
}

// Link words from the device mask, zero populations in solid cells, fresh phi.
template <int PREC, int QH>
pfl_status apply_solid(pfl_ctx* c, const unsigned char* mask_dev) {
  const long long N = c->geo.N;
  unsigned* links = (unsigned*)(c->ws + c->L.links);
  k_links<<<blocks_for(N, 256), 256, 0, c->stream>>>(c->geo, mask_dev, links);
  const size_t offs[4] = {c->L.h, c->L.g, c->L.h2, c->L.g2};
  const int qs[4] = {c->qh, c->qg, c->qh, c->qg};
  for (int k = 0; k < 4; ++k)
    k_zero_solid<PREC><<<blocks_for(N, 256), 256, 0, c->stream>>>(N, qs[k], links,
                                                                  (typename Store<PREC>::S*)(c->ws + offs[k]));
  if constexpr (PREC == 2)
    k_reshift_blocked<QH><<<blocks_for(N, 256), 256, 0, c->stream>>>(
        c->geo, (__half*)hbuf<PREC>(c), (__half*)gbuf<PREC>(c), (const float*)phibuf<PREC>(c, 1), pgbuf(c, 1), links);
  CUDA_TRY(cudaGetLastError());
  c->solid = true;
  return fresh_phi<PREC, QH>(c, false);  // phi = 0 in solid cells; the initial shifts stay
}

// Height of the phi = 1/2 crossing along y in the column (x, z): the first j
// with phi_j >= 1/2 > phi_{j+1} (going up from the heavy side), interpolated
// linearly, j + (phi_j - 1/2) / (phi_j - phi_{j+1}); NaN if there is none.
// One block; the lowest crossing wins.
template <typename PhiT>
__global__ void k_iface(const PhiT* __restrict__ phi, int nx, int ny, int x, int z, double* out) {
  __shared__ int first;
  if (threadIdx.x == 0) first = ny;
  __syncthreads();
  const long long col = (long long)x + (long long)nx * (long long)ny * z;
  for (int j = threadIdx.x; j + 1 < ny; j += blockDim.x) {
    const double a = (double)phi[col + (long long)nx * j], b = (double)phi[col + (long long)nx * (j + 1)];
    if (a >= 0.5 && 0.5 > b) atomicMin(&first, j);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int j = first;
    if (j >= ny) {
      out[0] = __longlong_as_double(0x7ff8000000000000ll);
    } else {
      const double a = (double)phi[col + (long long)nx * j], b = (double)phi[col + (long long)nx * (j + 1)];
      out[0] = (double)j + (a - 0.5) / (a - b);
    }
  }
}

template <int PREC>
void launch_iface(pfl_ctx* c, int x, int z, double* out) {
  k_iface<<<1, 256, 0, c->stream>>>(phicur<PREC>(c), c->p.nx, c->p.ny, x, z, out);
}

void drop_graphs(pfl_ctx* c) {
  for (int k = 0; k < 4; ++k)
    if (c->gx[k]) {
      cudaGraphExecDestroy(c->gx[k]);
      c->gx[k] = nullptr;
    }
}

// One replay of graph_k fused steps (captured on first use for the current
// (ab, cur) state; graph_k is even, so a replay returns the context to it).
// Every launch of the graph reads the step count from the device clock, which
// the graph advances by graph_k at its end: FP16S runs draw the same rounding
// bits as step-by-step launches.
pfl_status graph_steps(pfl_ctx* c) {
  const int slot = c->ab * 2 + c->cur;
  if (!c->gx[slot]) {
    if (!c->cap) CUDA_TRY(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    const long long t = c->t;
    const int ab = c->ab, cur = c->cur;
    const bool stale = c->stale;
    cudaStream_t user = c->stream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      c->stream = c->cap;
      c->capturing = true;
      c->cap_t0 = t;
      DISPATCH(c, launch_steps, c, c->graph_k);
      k_clock<<<1, 1, 0, c->cap>>>(clock_of(c), c->graph_k, 1);
      const cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = e2;
    }
    c->stream = user;
    c->capturing = false;
    c->t = t;
    c->ab = ab;
    c->cur = cur;
    c->stale = stale;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gx[slot], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->gx[slot] = nullptr;
      return cuda_fail(e, "capturing the step graph");
    }
  }
  if (c->clock_t != c->t) {
    k_clock<<<1, 1, 0, c->stream>>>(clock_of(c), c->t, 0);
    c->clock_t = c->t;
  }
  CUDA_TRY(cudaGraphLaunch(c->gx[slot], c->stream));
  c->t += c->graph_k;
  c->clock_t += c->graph_k;
  c->stale = true;
  return PFL_OK;
}

}  // namespace

extern "C" {

int pfl_version(void) { return 3; }

const char* pfl_last_error(void) { return g_err.c_str(); }

size_t pfl_workspace_bytes(const pfl_params* p) {
  if (!check_params(p).empty()) return 0;
  return layout_of(p).total;
}

pfl_status pfl_hydrostatic_pstar(const pfl_params* p, const double* phi0, double* pstar) {
  if (!p || !phi0 || !pstar) return fail(PFL_ERR_ARG, "params, phi0 and pstar must not be NULL");
  pfl_params q = *p;
  q.hydrostatic = 1;  // the checks of the hydrostatic start apply
  const std::string why = check_params(&q);
  if (!why.empty()) return fail(PFL_ERR_ARG, why);
  if (is_device_ptr(phi0) || is_device_ptr(pstar)) return fail(PFL_ERR_ARG, "phi0 and pstar must be host arrays");
  std::vector<double> out;
  hydrostatic_pstar(&q, phi0, out);
  std::copy(out.begin(), out.end(), pstar);
  return PFL_OK;
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
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(device));

  pfl_ctx* c = new pfl_ctx();
  c->p = *p;
  c->device = device;
  c->L = L;
  c->ws = (char*)workspace;
  c->stream = (cudaStream_t)stream;
  c->t = 0;
  c->swapped = 0;
  c->cur = 0;
  c->zm = uses_two_arrays(p);
  c->ab = 0;
  c->stale = false;
  c->qh = qh_of(p);
  c->qg = qg_of(p);
  c->solid = false;
  c->graph_k = 32;
  for (int k = 0; k < 4; ++k) c->gx[k] = nullptr;
  c->cap = nullptr;
  c->capturing = false;
  c->cap_t0 = 0;
  c->clock_t = -1;
  {
    // z planes per block.  Every block marches zc planes and fills two more
    // (the planes below and above its first) before it starts, about half a
    // plane's work; blocks run in waves of `slots` resident blocks.  Take the
    // zc with the least modelled time: waves x (zc + 0.5).
    int sms = 152, per_sm = 2;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const dim3 blk(ZM_TX, ZM_TY);
    if (p->precision == PFL_FP64)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_zm<0, 15, 0>, (int)(blk.x * blk.y), 0);
    else if (p->precision == PFL_FP32)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_zm<1, 15, 0>, (int)(blk.x * blk.y), 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_zm<2, 15, 0>, (int)(blk.x * blk.y), 0);
    if (per_sm < 1) per_sm = 1;
    const long long slots = (long long)sms * per_sm;
    const long long bxy = (long long)((p->nx + ZM_TX - 1) / ZM_TX) * ((p->ny + ZM_TY - 1) / ZM_TY);
    int best = p->nz;
    double best_cost = 1e300;
    for (int zc = p->nz; zc >= 1; --zc) {
      const long long blocks = bxy * ((p->nz + zc - 1) / zc);
      const double cost = (double)((blocks + slots - 1) / slots) * (zc + 0.5);
      if (cost < best_cost * (1 - 1e-9)) {
        best_cost = cost;
        best = zc;
      }
    }
    c->zc = best;
  }
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

  // Hydrostatic start (p0 == NULL, params.hydrostatic): p* from phi0 on the host.
  const long long N = c->geo.N;
  std::vector<double> p_hydro;
  if (!p0 && p->hydrostatic) {
    std::vector<double> phi_host;
    const double* ph0 = phi0;
    if (is_device_ptr(phi0)) {
      phi_host.resize((size_t)N);
      cudaError_t e = cudaMemcpy(phi_host.data(), phi0, (size_t)N * sizeof(double), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "phi0 to the host for the hydrostatic start");
      }
      ph0 = phi_host.data();
    }
    hydrostatic_pstar(p, ph0, p_hydro);
    p0 = p_hydro.data();
  }

  // Initial state, in chunks through the FP64 staging area (5 arrays per
  // chunk).  FP16S takes two passes: every cell's shifts first, then the
  // populations stored against their writers' shifts.
  const long long chunk = N / 5 > 0 ? N / 5 : 1;  // 5 * chunk <= N + 16 staging doubles
  double* st = stage(c);
  const int passes = p->precision == PFL_FP16S ? 2 : 1;
  for (int pass = passes == 2 ? 0 : 1; pass < 2; ++pass)
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
      if (u0 && pass == 1) {
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
      if (pass == 0)
        k_init_shift<<<blocks_for(cnt, 256), 256, 0, c->stream>>>(c0, cnt, a_phi, p0 ? a_p : nullptr,
                                                                   (float*)(c->ws + c->L.phi[1]), pgbuf(c, 1));
      else
        DISPATCH(c, launch_init, c, c0, cnt, a_phi, u0 ? a_ux : nullptr, u0 ? a_uy : nullptr, u0 ? a_uz : nullptr,
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
  DISPATCH_S(s, c, fresh_phi, c, false);
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
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  if (n < 0) return fail(PFL_ERR_ARG, "n_steps must be >= 0");
  if (n == 0) return PFL_OK;
  if (c->zm && c->graph_k > 0 && n >= c->graph_k) {
    // whole graphs of graph_k steps, unless the caller is capturing the stream
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(c->stream, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      for (; n >= c->graph_k; n -= c->graph_k) {
        const pfl_status s = graph_steps(c);
        if (s != PFL_OK) return s;
      }
    }
  }
  if (n > 0) DISPATCH(c, launch_steps, c, n);
  CUDA_TRY(cudaGetLastError());
  return PFL_OK;
}

pfl_status pfl_set_graph_steps(pfl_ctx* c, int k) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  if (k < 0 || k % 2 != 0 || k > 4096) return fail(PFL_ERR_ARG, "graph steps must be 0 or even in [2, 4096]");
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  c->graph_k = k;
  return PFL_OK;
}

pfl_status pfl_fields(pfl_ctx* c, double* phi, double* rho, double* p, double* u) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  const long long N = c->geo.N;
  double* want[6] = {phi, rho, p, u, u ? u + N : nullptr, u ? u + 2 * N : nullptr};
  double* dev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool host[6];
  for (int k = 0; k < 6; ++k) {
    host[k] = want[k] && !is_device_ptr(want[k]);
    if (want[k] && !host[k]) dev[k] = want[k];
  }
  // device outputs in one pass
  DISPATCH(c, ensure_phi, c);
  bool any_dev = false;
  for (int k = 0; k < 6; ++k) any_dev |= dev[k] != nullptr;
  if (any_dev) DISPATCH(c, launch_fields, c, dev);
  // host outputs one at a time through the staging area
  for (int k = 0; k < 6; ++k) {
    if (!host[k]) continue;
    double* o[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    o[k] = stage(c);
    DISPATCH(c, launch_fields, c, o);
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
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  DISPATCH(c, ensure_phi, c);
  const long long N = c->geo.N;
  for (int set = 0; set < 2; ++set) {
    double* dst = set == 0 ? h : g;
    if (!dst) continue;
    const int q = set == 0 ? c->qh : c->qg;
    const bool dev = is_device_ptr(dst);
    for (int i = 0; i < q; ++i) {
      double* o = dev ? dst + (size_t)i * N : stage(c);
      DISPATCH(c, launch_export, c, set, i, o);
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
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  if (!h || !g) return fail(PFL_ERR_ARG, "both population sets are required");
  const long long N = c->geo.N;
  // read the complete current state first when only part would change: not
  // needed, both sets are replaced; the layout becomes the normal one.
  for (int set = 0; set < 2; ++set) {
    const double* src = set == 0 ? h : g;
    const int q = set == 0 ? c->qh : c->qg;
    for (int i = 0; i < q; ++i) {
      CUDA_TRY(cudaMemcpyAsync(stage(c), src + (size_t)i * N, N * sizeof(double), cudaMemcpyDefault, c->stream));
      DISPATCH(c, launch_import, c, set, i, stage(c));
      CUDA_TRY(cudaGetLastError());
      CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
  }
  pfl_status s = PFL_OK;
  DISPATCH_S(s, c, fresh_phi, c, true);
  if (s != PFL_OK) return s;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PFL_OK;
}

// ---- saved states: a header, then the stored arrays as they sit in the
// workspace (current h, current g, both phi buffers, the link words)
constexpr int NSAVED = 7;
struct SavedHeader {
  char magic[8];          // "PFLSTATE"
  int version;            // 2 (7 sections)
  int precision, qh, qg;  // storage and lattices
  int nx, ny, nz, bc[6];  // lattice
  int zm, solid;          // engine (fused two-array step or in-place), solid cells present
  int cur, swapped, stale;
  long long t;
  unsigned long long bytes[NSAVED];  // h, g, phi buffers 0 and 1, links, p* shift buffers 0 and 1
};

// workspace offsets of the saved sections: the current h and g, the phi
// buffers, the links, the FP16S p* shift buffers
static void saved_offsets(const pfl_ctx* c, size_t o[NSAVED]) {
  const bool second = c->zm && c->ab;
  o[0] = second ? c->L.h2 : c->L.h;
  o[1] = second ? c->L.g2 : c->L.g;
  o[2] = c->L.phi[0];
  o[3] = c->L.phi[1];
  o[4] = c->L.links;
  o[5] = c->L.pg[0];
  o[6] = c->L.pg[1];
}

static void saved_sections(const pfl_ctx* c, unsigned long long b[NSAVED]) {
  const unsigned long long N = (unsigned long long)c->geo.N;
  b[0] = (unsigned long long)c->qh * N * pop_bytes(c->p.precision);
  b[1] = (unsigned long long)c->qg * N * pop_bytes(c->p.precision);
  b[2] = b[3] = N * phi_bytes(c->p.precision);
  b[4] = c->solid ? N * sizeof(unsigned) : 0;
  b[5] = b[6] = c->p.precision == PFL_FP16S ? N * sizeof(__half) : 0;
}

size_t pfl_state_bytes(const pfl_ctx* c) {
  if (!c) return 0;
  unsigned long long b[NSAVED];
  saved_sections(c, b);
  size_t total = sizeof(SavedHeader);
  for (int k = 0; k < NSAVED; ++k) total += (size_t)b[k];
  return total;
}

pfl_status pfl_save(pfl_ctx* c, void* buf, size_t bytes) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  if (!buf) return fail(PFL_ERR_ARG, "buffer is NULL");
  if (bytes < pfl_state_bytes(c))
    return fail(PFL_ERR_ARG, "buffer holds " + std::to_string(bytes) + " bytes, a state needs " +
                                 std::to_string(pfl_state_bytes(c)));
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  SavedHeader hd;
  std::memset(&hd, 0, sizeof hd);
  std::memcpy(hd.magic, "PFLSTATE", 8);
  hd.version = 2;
  hd.precision = c->p.precision;
  hd.qh = c->qh;
  hd.qg = c->qg;
  hd.nx = c->p.nx;
  hd.ny = c->p.ny;
  hd.nz = c->p.nz;
  for (int k = 0; k < 6; ++k) hd.bc[k] = c->p.bc[k];
  hd.zm = c->zm;
  hd.solid = c->solid;
  hd.cur = c->cur;
  hd.swapped = c->swapped;
  hd.stale = c->stale;
  hd.t = c->t;
  saved_sections(c, hd.bytes);
  char* dst = (char*)buf;
  CUDA_TRY(cudaMemcpyAsync(dst, &hd, sizeof hd, cudaMemcpyDefault, c->stream));
  size_t off = sizeof hd;
  size_t so[NSAVED];
  saved_offsets(c, so);
  for (int k = 0; k < NSAVED; ++k) {
    if (hd.bytes[k]) CUDA_TRY(cudaMemcpyAsync(dst + off, c->ws + so[k], hd.bytes[k], cudaMemcpyDefault, c->stream));
    off += hd.bytes[k];
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));  // the header lives on this stack
  return PFL_OK;
}

pfl_status pfl_load(pfl_ctx* c, const void* buf, size_t bytes) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  if (!buf) return fail(PFL_ERR_ARG, "buffer is NULL");
  if (bytes < sizeof(SavedHeader)) return fail(PFL_ERR_ARG, "buffer is shorter than a state header");
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  SavedHeader hd;
  CUDA_TRY(cudaMemcpy(&hd, buf, sizeof hd, cudaMemcpyDefault));
  if (std::memcmp(hd.magic, "PFLSTATE", 8) != 0 || hd.version != 2)
    return fail(PFL_ERR_ARG, "not a saved state (magic or version)");
  bool same = hd.precision == c->p.precision && hd.qh == c->qh && hd.qg == c->qg && hd.nx == c->p.nx &&
              hd.ny == c->p.ny && hd.nz == c->p.nz && hd.zm == (int)c->zm;
  for (int k = 0; k < 6; ++k) same = same && hd.bc[k] == c->p.bc[k];
  if (!same)
    return fail(PFL_ERR_ARG, "the saved state's lattice, boundaries, precision or engine differ from the context's");
  if (hd.solid && !c->p.solids) return fail(PFL_ERR_STATE, "the saved state has solid cells; create the context with solids = 1");
  if (!hd.solid && c->solid) return fail(PFL_ERR_STATE, "the context has solid cells and the saved state none");
  unsigned long long want[NSAVED];
  const bool was_solid = c->solid;
  c->solid = hd.solid != 0;
  saved_sections(c, want);
  c->solid = was_solid;
  size_t total = sizeof hd;
  for (int k = 0; k < NSAVED; ++k) {
    if (hd.bytes[k] != want[k]) return fail(PFL_ERR_ARG, "the saved state's section sizes do not match");
    total += (size_t)want[k];
  }
  if (bytes < total) return fail(PFL_ERR_ARG, "buffer is shorter than the saved state");
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  // the saved phi buffers keep their roles: buffer `cur` holds phi^t
  const char* from = (const char*)buf + sizeof hd;
  size_t so[NSAVED];
  saved_offsets(c, so);
  for (int k = 0; k < NSAVED; ++k) {
    if (want[k]) CUDA_TRY(cudaMemcpyAsync(c->ws + so[k], from, want[k], cudaMemcpyDefault, c->stream));
    from += want[k];
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->solid = hd.solid != 0;
  c->cur = hd.cur;
  c->swapped = hd.swapped;
  c->stale = hd.stale != 0;
  c->t = hd.t;
  c->clock_t = -1;  // the device step count of graph replays is set again before the next replay
  return PFL_OK;
}

pfl_status pfl_set_solid(pfl_ctx* c, const unsigned char* mask) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  if (!mask) return fail(PFL_ERR_ARG, "mask is NULL");
  if (!c->p.solids) return fail(PFL_ERR_STATE, "the context was created without solids (pfl_params.solids = 0)");
  if (c->t != 0) return fail(PFL_ERR_STATE, "solid cells are set before the first step");
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  const long long N = c->geo.N;
  unsigned char* st = (unsigned char*)stage(c);  // N bytes fit the N + 16 doubles of the staging area
  CUDA_TRY(cudaMemcpyAsync(st, mask, (size_t)N, cudaMemcpyDefault, c->stream));
  pfl_status s = PFL_OK;
  DISPATCH_S(s, c, apply_solid, c, st);
  if (s != PFL_OK) return s;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PFL_OK;
}

// Largest flow speed of the current state (FP64, on the device into *res).
static pfl_status queue_speed(pfl_ctx* c, double* res) {
  double* part = (double*)(c->ws + c->L.red) + DIAG_BLOCKS * 9 + 16;
  DISPATCH(c, ensure_phi, c);
  DISPATCH(c, launch_umax, c, part, res);
  CUDA_TRY(cudaGetLastError());
  return PFL_OK;
}

pfl_status pfl_diag(pfl_ctx* c, double out[8], long long* nonfinite) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  double* part = (double*)(c->ws + c->L.red);
  double* res = part + DIAG_BLOCKS * 9;
  double* ures = part + DIAG_BLOCKS * 10 + 16;
  DISPATCH(c, ensure_phi, c);
  DISPATCH_PREC(c, launch_diag, c, part, res);
  CUDA_TRY(cudaGetLastError());
  pfl_status st = queue_speed(c, ures);
  if (st != PFL_OK) return st;
  double host[9], umax = 0.0;
  CUDA_TRY(cudaMemcpyAsync(host, res, sizeof(host), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaMemcpyAsync(&umax, ures, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (out)
    for (int k = 0; k < 8; ++k) out[k] = host[k];
  long long nf = (long long)host[8];
  if (nonfinite) *nonfinite = nf;
  if (nf > 0) return fail(PFL_ERR_UNSTABLE, std::to_string(nf) + " cells hold a non-finite phi");
  if (!(umax <= PFL_SPEED_LIMIT))
    return fail(PFL_ERR_UNSTABLE, "flow speed |u| = " + std::to_string(umax) + " exceeds " +
                                      std::to_string(PFL_SPEED_LIMIT) + " (lattice units)");
  return PFL_OK;
}

pfl_status pfl_max_speed(pfl_ctx* c, double* umax) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  if (!umax) return fail(PFL_ERR_ARG, "umax is NULL");
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  double* ures = (double*)(c->ws + c->L.red) + DIAG_BLOCKS * 10 + 16;
  pfl_status st = queue_speed(c, ures);
  if (st != PFL_OK) return st;
  CUDA_TRY(cudaMemcpyAsync(umax, ures, sizeof(double), cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PFL_OK;
}

pfl_status pfl_interface_height(pfl_ctx* c, int x, int z, double* y) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  if (!y) return fail(PFL_ERR_ARG, "y is NULL");
  if (x < 0 || x >= c->p.nx || z < 0 || z >= c->p.nz) return fail(PFL_ERR_ARG, "column (x, z) outside the lattice");
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  DISPATCH(c, ensure_phi, c);
  double* res = (double*)(c->ws + c->L.red) + DIAG_BLOCKS * 9 + 9;  // a spare word after the diag results
  DISPATCH_PREC(c, launch_iface, c, x, z, res);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(y, res, sizeof(double), cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PFL_OK;
}

pfl_status pfl_kernel_times(pfl_ctx* c, int n, double ms[2]) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  if (n <= 0 || !ms) return fail(PFL_ERR_ARG, "n_steps must be > 0 and ms non-NULL");
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  cudaEvent_t ev[3];
  for (int k = 0; k < 3; ++k) CUDA_TRY(cudaEventCreate(&ev[k]));
  double acc[2] = {0, 0};
  pfl_status st = PFL_OK;
  for (int s = 0; s < n && st == PFL_OK; ++s) {
    cudaEventRecord(ev[0], c->stream);
    DISPATCH(c, step_any, c);
    cudaEventRecord(ev[1], c->stream);
    DISPATCH(c, after_step, c);
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

}  // extern "C"

// ----------------------------------------------------------------- adjoint --
namespace {

constexpr int ADJ_MAX_OBS = 1 << 20;  // observations per call (distinct steps in [0, n_steps])
constexpr int ADJ_STAGE = 8;          // device slots through which host weight fields are staged
constexpr int DOT_BLOCKS = 1024;

struct AdjLayout {
  size_t state;      // bytes of one saved state (h, g, phi)
  int K, nck;        // checkpoint interval, number of checkpoints
  size_t ck, seg, fin, lam0, lam1, aux, acc, W, part, res, total;
};

size_t rbytes(int prec) { return prec == PFL_FP64 ? 8 : 4; }

AdjLayout adj_layout(const pfl_ctx* c, int n) {
  AdjLayout A;
  const size_t N = (size_t)c->geo.N;
  const size_t S = pop_bytes(c->p.precision), P = phi_bytes(c->p.precision), R = rbytes(c->p.precision);
  const size_t QH = (size_t)c->qh;
  const size_t QG = (size_t)c->qg;
  A.state = align256(QH * N * S) + align256(QG * N * S) + align256(N * P);
  A.K = 1;
  while ((long long)A.K * A.K < n) ++A.K;
  A.nck = (n + A.K - 1) / A.K;
  if (A.nck < 1) A.nck = 1;
  size_t off = 0;
  A.ck = off;
  off += (size_t)A.nck * A.state;
  A.seg = off;
  off += (size_t)A.K * A.state;
  A.fin = off;
  if (!c->zm) off += A.state;  // the fused engine's reverse sweep leaves the live state alone
  A.lam0 = off;
  off = align256(off + (QH + QG) * N * R);
  A.lam1 = off;
  off = align256(off + (QH + QG) * N * R);
  A.aux = off;
  off = align256(off + 5 * N * R);
  A.acc = off;
  off = align256(off + N * R);
  A.W = off;
  off = align256(off + (size_t)ADJ_STAGE * N * sizeof(double));
  A.part = off;
  const size_t nb = (N + ADJ_THREADS - 1) / ADJ_THREADS;
  off = align256(off + (3 * nb + DOT_BLOCKS) * sizeof(double));
  A.res = off;
  off = align256(off + 8 * sizeof(double));
  A.total = off;
  return A;
}

struct Saved {
  int swapped;
};

// copy the live state (h, g, current phi) into a slot, or back
pfl_status copy_state(pfl_ctx* c, char* slot, bool save) {
  const size_t N = (size_t)c->geo.N;
  const size_t S = pop_bytes(c->p.precision), P = phi_bytes(c->p.precision);
  const size_t hb = (size_t)c->qh * N * S, gb = (size_t)c->qg * N * S, pb = N * P;
  const bool second = c->zm && c->ab;
  char* live[3] = {c->ws + (second ? c->L.h2 : c->L.h), c->ws + (second ? c->L.g2 : c->L.g),
                   c->ws + c->L.phi[c->cur]};
  char* sl[3] = {slot, slot + align256(hb), slot + align256(hb) + align256(gb)};
  const size_t by[3] = {hb, gb, pb};
  for (int k = 0; k < 3; ++k)
    CUDA_TRY(cudaMemcpyAsync(save ? sl[k] : live[k], save ? live[k] : sl[k], by[k], cudaMemcpyDeviceToDevice,
                             c->stream));
  if (!save) c->stale = false;  // the restored phi belongs to the restored populations
  return PFL_OK;
}

template <int PREC>
void launch_dot(pfl_ctx* c, const double* W, double* part, double* out) {
  k_dot<typename Store<PREC>::PhiT><<<DOT_BLOCKS, 256, 0, c->stream>>>((unsigned)c->geo.N, W, phicur<PREC>(c), part);
  k_sum_parts<<<1, 32, 0, c->stream>>>(part, DOT_BLOCKS, 1, out);
}

template <int PREC, int QH>
void launch_adj_step(pfl_ctx* c, const AdjLayout& A, char* aws, char* slot, int swapped, const void* lam_in,
                     void* lam_out, const double* W) {
  typedef typename Store<PREC>::R R;
  const size_t N = (size_t)c->geo.N;
  const size_t S = pop_bytes(c->p.precision);
  const typename Store<PREC>::S* h = (const typename Store<PREC>::S*)slot;
  const typename Store<PREC>::S* g = (const typename Store<PREC>::S*)(slot + align256((size_t)QH * N * S));
  const typename Store<PREC>::PhiT* phi =
      (const typename Store<PREC>::PhiT*)(slot + align256((size_t)QH * N * S) + align256((size_t)qg_of<QH>() * N * S));
  const AdjParR<R> ap = adj_par_r<R>(AdjPar{c->p.mobility, c->p.xi, c->p.sigma});
  const PhysR<R> phr = phys_r<R>(c->ph);
  double* part = (double*)(aws + A.part);
  R* aux = (R*)(aws + A.aux);
  R* acc = (R*)(aws + A.acc);
  const unsigned nb = blocks_for(c->geo.N, ADJ_THREADS);
  if (swapped)
    k_adj_local<PREC, QH, 1><<<nb, ADJ_THREADS, 0, c->stream>>>(c->g32, phr, ap, h, g, phi, (const R*)lam_in,
                                                             acc, (R*)lam_out, aux, part);
  else
    k_adj_local<PREC, QH, 0><<<nb, ADJ_THREADS, 0, c->stream>>>(c->g32, phr, ap, h, g, phi, (const R*)lam_in,
                                                             acc, (R*)lam_out, aux, part);
  const dim3 grid((c->p.nx + ZM_TX - 1) / ZM_TX, (c->p.ny + ZM_TY - 1) / ZM_TY, (c->p.nz + c->zc - 1) / c->zc);
  k_adj_phi<R, qg_of<QH>()><<<grid, dim3(ZM_TX, ZM_TY), 0, c->stream>>>(c->g32, aux, acc, W, c->zc);
}

// lambda at the final time: local part 0, acc = W (the objective's weight on
// phi, which the h entries share)
template <typename R>
__global__ void k_lam_init(unsigned N, int q, R* __restrict__ lam, R* __restrict__ acc, const double* __restrict__ W) {
  const unsigned x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  for (int i = 0; i < q; ++i) lam[(unsigned)i * N + x] = (R)0;
  acc[x] = W ? (R)W[x] : (R)0;
}

// slot layout: h, g, phi (each 256-byte aligned)
template <int PREC>
struct SlotPtr {
  typename Store<PREC>::S* h;
  typename Store<PREC>::S* g;
  typename Store<PREC>::PhiT* phi;
  SlotPtr(const pfl_ctx* c, char* slot) {
    const size_t N = (size_t)c->geo.N, S = pop_bytes(c->p.precision);
    h = (typename Store<PREC>::S*)slot;
    const size_t hb = (size_t)c->qh * N * S;
    g = (typename Store<PREC>::S*)(slot + align256(hb));
    phi = (typename Store<PREC>::PhiT*)(slot + align256(hb) + align256((size_t)c->qg * N * S));
  }
};

// One fused step from slot a into slot b; phi of a (the sum the kernel forms
// in shared memory) goes to a's phi.  FP64 / FP32 only: no shifts.
template <int PREC, int QH>
void zm_step_slots(pfl_ctx* c, const SlotPtr<PREC>& a, const SlotPtr<PREC>& b) {
  const int ty = zm_ty(c->p.nz == 1);
  const dim3 grid((c->p.nx + ZM_TX - 1) / ZM_TX, (c->p.ny + ty - 1) / ty, (c->p.nz + c->zc - 1) / c->zc);
  const dim3 block(ZM_TX, ty);
  if (c->p.nz == 1)
    k_step_zm<PREC, QH, 1><<<grid, block, 0, c->stream>>>(c->g32, c->ph, a.h, a.g, b.h, b.g, nullptr, a.phi, c->zc, 0u);
  else
    k_step_zm<PREC, QH, 0><<<grid, block, 0, c->stream>>>(c->g32, c->ph, a.h, a.g, b.h, b.g, nullptr, a.phi, c->zc, 0u);
}

// Adjoint with the fused two-array engine.  Forward sweep: checkpoints every K
// steps, phi formed only where a checkpoint or an observation needs it.
// Reverse sweep, per segment: the checkpoint is copied into slot 0 and each
// recomputed step writes the next slot directly, so the live state (t_end) is
// never touched and no per-step copy is made.
template <int PREC, int QH, class ObsAt>
pfl_status run_adjoint_zm(pfl_ctx* c, int n, const ObsAt& obs_at, char* aws, const AdjLayout& A, double* J,
                          double grad[3]) {
  typedef typename Store<PREC>::R R;
  double* res = (double*)(aws + A.res);
  double* part = (double*)(aws + A.part);
  double* dot_part = part + 3 * ((c->geo.N + ADJ_THREADS - 1) / ADJ_THREADS);
  for (int k = 0; k < n; ++k) {
    const double* W = obs_at(k);
    if (k % A.K == 0 || W) ensure_phi<PREC, QH>(c);
    if (k % A.K == 0) {
      pfl_status s = copy_state(c, aws + A.ck + (size_t)(k / A.K) * A.state, true);
      if (s != PFL_OK) return s;
    }
    if (W) launch_dot<PREC>(c, W, dot_part, res);
    step_only<PREC, QH, 0>(c);
  }
  ensure_phi<PREC, QH>(c);
  if (const double* W = obs_at(n)) launch_dot<PREC>(c, W, dot_part, res);
  CUDA_TRY(cudaGetLastError());

  void* lam = aws + A.lam0;
  void* lam2 = aws + A.lam1;
  const unsigned nbl = blocks_for(c->geo.N, ADJ_THREADS);  // per-block gradient partials, summed at the end
  CUDA_TRY(cudaMemsetAsync(part, 0, 3 * (size_t)nbl * sizeof(double), c->stream));
  k_lam_init<R><<<blocks_for(c->geo.N, 256), 256, 0, c->stream>>>((unsigned)c->geo.N, c->qh + c->qg, (R*)lam,
                                                                   (R*)(aws + A.acc), obs_at(n));
  for (int sgm = A.nck - 1; sgm >= 0; --sgm) {
    const int k0 = sgm * A.K, k1 = (k0 + A.K < n) ? k0 + A.K : n;
    char* seg = aws + A.seg;
    CUDA_TRY(cudaMemcpyAsync(seg, aws + A.ck + (size_t)sgm * A.state, A.state, cudaMemcpyDeviceToDevice, c->stream));
    for (int k = k0; k + 1 < k1; ++k)
      zm_step_slots<PREC, QH>(c, SlotPtr<PREC>(c, seg + (size_t)(k - k0) * A.state),
                          SlotPtr<PREC>(c, seg + (size_t)(k + 1 - k0) * A.state));
    if (k1 - 1 > k0) {  // phi of the last slot (the others were formed by the steps out of them)
      const SlotPtr<PREC> last(c, seg + (size_t)(k1 - 1 - k0) * A.state);
      k_phi32<PREC, QH, 0><<<blocks_for(c->geo.N, 256), 256, 0, c->stream>>>(c->g32, last.h, nullptr, last.phi);
    }
    for (int k = k1 - 1; k >= k0; --k) {
      launch_adj_step<PREC, QH>(c, A, aws, seg + (size_t)(k - k0) * A.state, 0, lam, lam2, obs_at(k));
      std::swap(lam, lam2);
    }
    CUDA_TRY(cudaGetLastError());
  }
  k_sum_parts<<<3, 32, 0, c->stream>>>(part, (int)nbl, 3, res + 1);
  double hres[4];
  CUDA_TRY(cudaMemcpyAsync(hres, res, sizeof(hres), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (J) *J = hres[0];
  if (grad)
    for (int k = 0; k < 3; ++k) grad[k] = hres[1 + k];
  return PFL_OK;
}

// The weight field of the observation at step k (relative to the adjoint's
// first step), as device memory, or NULL: a device field as given; a host
// field copied, when asked for, into the next of ADJ_STAGE staging slots of
// the adjoint workspace (the copy is ordered on the stream before the kernel
// that reads the slot, and after the kernels that read its previous content).
struct ObsTable {
  std::vector<int> at;                 // step -> observation index, or -1
  const double* const* w;
  std::vector<char> dev;               // the field is device memory
  double* stage;                       // ADJ_STAGE slots of N doubles
  size_t N;
  cudaStream_t stream;
  mutable int next = 0;
  mutable cudaError_t err = cudaSuccess;
  const double* operator()(int k) const {
    if (k < 0 || k >= (int)at.size() || at[(size_t)k] < 0) return nullptr;
    const int o = at[(size_t)k];
    if (dev[(size_t)o]) return w[o];
    double* slot = stage + (size_t)(next++ % ADJ_STAGE) * N;
    cudaError_t e = cudaMemcpyAsync(slot, w[o], N * sizeof(double), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) err = e;
    return slot;
  }
};

template <int PREC, int QH>
pfl_status run_adjoint(pfl_ctx* c, int n, const ObsTable& obs_at, char* aws, const AdjLayout& A, double* J,
                       double grad[3]) {
  typedef typename Store<PREC>::R R;
  double* res = (double*)(aws + A.res);  // [0] J, [1..3] dJ/d(M, xi, sigma)
  double* part = (double*)(aws + A.part);
  CUDA_TRY(cudaMemsetAsync(res, 0, 8 * sizeof(double), c->stream));
  if (c->zm) return run_adjoint_zm<PREC, QH>(c, n, obs_at, aws, A, J, grad);
  // several weights at one step are summed into the first by the caller side; here one per step
  const long long t0 = c->t;
  std::vector<int> ck_swapped(A.nck, 0), seg_swapped(A.K, 0);
  // forward sweep with checkpoints
  ensure_phi<PREC, QH>(c);
  for (int k = 0; k < n; ++k) {
    if (k % A.K == 0) {
      ck_swapped[k / A.K] = c->swapped;
      pfl_status s = copy_state(c, aws + A.ck + (size_t)(k / A.K) * A.state, true);
      if (s != PFL_OK) return s;
    }
    if (const double* W = obs_at(k)) launch_dot<PREC>(c, W, part + 3 * ((c->geo.N + ADJ_THREADS - 1) / ADJ_THREADS), res);
    const bool bgk = false;
    (void)bgk;
    step_only<PREC, QH, 0>(c);
    after_step<PREC, QH>(c);
    ensure_phi<PREC, QH>(c);
  }
  if (const double* W = obs_at(n)) launch_dot<PREC>(c, W, part + 3 * ((c->geo.N + ADJ_THREADS - 1) / ADJ_THREADS), res);
  const int fin_swapped = c->swapped;
  const long long t_end = c->t;
  pfl_status st = copy_state(c, aws + A.fin, true);
  if (st != PFL_OK) return st;
  CUDA_TRY(cudaGetLastError());

  // reverse sweep, one checkpoint segment at a time
  void* lam = aws + A.lam0;
  void* lam2 = aws + A.lam1;
  const unsigned nbl = blocks_for(c->geo.N, ADJ_THREADS);  // per-block gradient partials, summed at the end
  CUDA_TRY(cudaMemsetAsync(part, 0, 3 * (size_t)nbl * sizeof(double), c->stream));
  k_lam_init<R><<<blocks_for(c->geo.N, 256), 256, 0, c->stream>>>((unsigned)c->geo.N, c->qh + c->qg, (R*)lam,
                                                                   (R*)(aws + A.acc), obs_at(n));
  for (int sgm = A.nck - 1; sgm >= 0; --sgm) {
    const int k0 = sgm * A.K, k1 = (k0 + A.K < n) ? k0 + A.K : n;
    st = copy_state(c, aws + A.ck + (size_t)sgm * A.state, false);
    if (st != PFL_OK) return st;
    c->swapped = ck_swapped[sgm];
    for (int k = k0; k < k1; ++k) {
      seg_swapped[k - k0] = c->swapped;
      st = copy_state(c, aws + A.seg + (size_t)(k - k0) * A.state, true);
      if (st != PFL_OK) return st;
      if (k + 1 < k1) {  // the last state of the segment is never stepped from here
        step_only<PREC, QH, 0>(c);
        after_step<PREC, QH>(c);
        ensure_phi<PREC, QH>(c);
      }
    }
    for (int k = k1 - 1; k >= k0; --k) {
      launch_adj_step<PREC, QH>(c, A, aws, aws + A.seg + (size_t)(k - k0) * A.state, seg_swapped[k - k0], lam, lam2,
                            obs_at(k));
      std::swap(lam, lam2);
    }
    CUDA_TRY(cudaGetLastError());
  }
  k_sum_parts<<<3, 32, 0, c->stream>>>(part, (int)nbl, 3, res + 1);
  // back to the end of the forward run
  st = copy_state(c, aws + A.fin, false);
  if (st != PFL_OK) return st;
  c->swapped = fin_swapped;
  c->t = t_end;
  (void)t0;
  double hres[4];
  CUDA_TRY(cudaMemcpyAsync(hres, res, sizeof(hres), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (J) *J = hres[0];
  if (grad)
    for (int k = 0; k < 3; ++k) grad[k] = hres[1 + k];
  return PFL_OK;
}

}  // namespace

extern "C" {

size_t pfl_adjoint_workspace_bytes(const pfl_ctx* c, int n_steps) {
  if (!c || n_steps < 1) return 0;
  return adj_layout(c, n_steps).total;
}

pfl_status pfl_adjoint(pfl_ctx* c, int n_steps, int n_obs, const int* obs_steps, const double* const* obs_weights,
                       void* adj_workspace, size_t adj_bytes, double* J, double grad[3]) {
  if (!c) return fail(PFL_ERR_ARG, "context is NULL");
  if (n_steps < 1) return fail(PFL_ERR_ARG, "n_steps must be >= 1");
  if (c->p.precision == PFL_FP16S) return fail(PFL_ERR_STATE, "the adjoint runs on FP64 or FP32 storage");
  if (c->solid) return fail(PFL_ERR_STATE, "the adjoint covers lattices without solid cells");
  if (c->p.collision != PFL_MRT) return fail(PFL_ERR_STATE, "the adjoint covers the MRT collision");
  if (!c->idx32) return fail(PFL_ERR_STATE, "lattice too large for the adjoint kernels (27 N >= 2^32)");
  if (n_obs < 1 || n_obs > ADJ_MAX_OBS || !obs_steps || !obs_weights)
    return fail(PFL_ERR_ARG, "need 1.." + std::to_string(ADJ_MAX_OBS) + " observations");
  for (int o = 0; o < n_obs; ++o) {
    if (obs_steps[o] < 0 || obs_steps[o] > n_steps || !obs_weights[o])
      return fail(PFL_ERR_ARG, "observation step outside [0, n_steps] or NULL weights");
    for (int q = 0; q < o; ++q)
      if (obs_steps[q] == obs_steps[o]) return fail(PFL_ERR_ARG, "observation steps must be distinct");
  }
  if (!adj_workspace || !is_device_ptr(adj_workspace)) return fail(PFL_ERR_ARG, "adjoint workspace must be device memory");
  if (((uintptr_t)adj_workspace & 255) != 0) return fail(PFL_ERR_ARG, "adjoint workspace must be 256-byte aligned");
  const AdjLayout A = adj_layout(c, n_steps);
  if (adj_bytes < A.total)
    return fail(PFL_ERR_OOM, "adjoint workspace holds " + std::to_string(adj_bytes) + " bytes, needs " +
                                 std::to_string(A.total));
  DeviceScope on_device;
  CUDA_TRY(on_device.enter(c->device));
  char* aws = (char*)adj_workspace;
  const size_t N = (size_t)c->geo.N;
  ObsTable obs;
  obs.at.assign((size_t)n_steps + 1, -1);
  obs.dev.resize((size_t)n_obs);
  for (int o = 0; o < n_obs; ++o) {
    obs.at[(size_t)obs_steps[o]] = o;
    obs.dev[(size_t)o] = is_device_ptr(obs_weights[o]) ? 1 : 0;
  }
  obs.w = obs_weights;
  obs.stage = (double*)(aws + A.W);
  obs.N = N;
  obs.stream = c->stream;
  pfl_status st;
  if (c->p.precision == PFL_FP64)
    st = c->qh == 27 ? run_adjoint<0, 27>(c, n_steps, obs, aws, A, J, grad)
         : c->qh == 9 ? run_adjoint<0, 9>(c, n_steps, obs, aws, A, J, grad)
                      : run_adjoint<0, 15>(c, n_steps, obs, aws, A, J, grad);
  else
    st = c->qh == 27 ? run_adjoint<1, 27>(c, n_steps, obs, aws, A, J, grad)
         : c->qh == 9 ? run_adjoint<1, 9>(c, n_steps, obs, aws, A, J, grad)
                      : run_adjoint<1, 15>(c, n_steps, obs, aws, A, J, grad);
  if (st == PFL_OK && obs.err != cudaSuccess) return cuda_fail(obs.err, "observation weights to the device");
  return st;
}

void pfl_destroy(pfl_ctx* c) {
  if (!c) return;
  DeviceScope on_device;  // the stream (NULL: the legacy stream) is the context's device's
  on_device.enter(c->device);
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

}  // extern "C"
