// Batched PFLBM: many independent lattices of uneven size and their own
// parameters (M, xi, sigma, ...) advanced together.
//
// Every lattice time step is one persistent launch of the stream-collide over
// all instances and one of the phi pass: a grid of (SMs x resident blocks)
// blocks walks a device work list of tiles (instance, first cell), each tile
// one cell per thread, and reads the instance's geometry, parameters and
// buffers from a device table.  Instances fall into two size classes (below
// and above 64 K cells); each class has its own work list and launch shape.
// The shapes -- threads per block and grid size -- are chosen at init by
// timing the candidates on the initial state (which is then rebuilt).  The
// step loop is captured once into a CUDA graph of 2 G lattice steps (an even
// count, so parity and phi buffers return to their starting roles) and
// replayed.
//
// The per-cell arithmetic is step_cell / phi_cell, the same code as the
// single-lattice kernels, so an instance of the batch evolves exactly like the
// same lattice run alone.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pflbm.h"
#include "errors.h"
#include "host_common.h"
#include "step.cuh"

using namespace pfl;
using namespace pfl_host;

namespace {

pfl_status bfail(pfl_status s, const std::string& m) {
  pfl_internal::set_error(m);
  return s;
}

#define BTRY(call)                                                                                         \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess) return bfail(PFL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct BInst {
  Geo32 geo;
  Phys ph;
  void* h;
  void* g;
  void* phi[2];
  int active;
  int frozen_cur, frozen_swapped;  // host bookkeeping: roles of the buffers when the instance stopped
};

struct BTile {
  int inst;
  unsigned c0;
};

constexpr int NCLASS = 2;
constexpr unsigned SMALL_CELLS = 65536;
constexpr int GRAPH_PAIRS = 8;  // a graph holds 2 * GRAPH_PAIRS lattice steps

template <int PREC, int ODD, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS == 128 ? 4 : 2)
    k_batch_step(const BInst* __restrict__ inst, const BTile* __restrict__ tiles, int ntiles, int cur,
                 const unsigned* __restrict__ tstep) {
  typedef typename Store<PREC>::S S;
  typedef typename Store<PREC>::PhiT PhiT;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const BTile tile = tiles[t];
    const BInst* I = inst + tile.inst;
    if (!I->active) continue;
    const unsigned cell = tile.c0 + threadIdx.x;
    if (cell < I->geo.N)
      step_cell<PREC, 15, ODD>(I->geo, I->ph, (S*)I->h, (S*)I->g, (const PhiT*)I->phi[cur], (const PhiT*)I->phi[1 - cur],
                           cell, *tstep * 0x9E3779B9u + (unsigned)tile.inst * 0x85EBCA6Bu);
  }
}

// The phi pass of the last class also advances the device step counter that
// seeds the stochastic rounding (the graph replays fixed kernel arguments).
template <int PREC, int READ_ODD, int THREADS>
__global__ void __launch_bounds__(THREADS) k_batch_phi(const BInst* __restrict__ inst, const BTile* __restrict__ tiles,
                                                       int ntiles, int cur, unsigned* __restrict__ tick) {
  typedef typename Store<PREC>::S S;
  typedef typename Store<PREC>::PhiT PhiT;
  if (tick && blockIdx.x == 0 && threadIdx.x == 0) *tick += 1u;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const BTile tile = tiles[t];
    const BInst* I = inst + tile.inst;
    if (!I->active) continue;
    const unsigned cell = tile.c0 + threadIdx.x;
    if (cell < I->geo.N)
      ((PhiT*)I->phi[1 - cur])[cell] = phi_cell<PREC, 15, READ_ODD>(I->geo, (const S*)I->h, (const PhiT*)I->phi[cur], cell);
  }
}

struct Shape {
  int threads;  // 128 or 256 (one cell per thread per tile)
  int grid;     // blocks of the persistent launch
};

struct ClassPlan {
  std::vector<int> members;
  Shape shape{128, 0};
  BTile* tiles = nullptr;  // device, for shape.threads
  int ntiles = 0;
};

Phys phys_of(const pfl_params* p) {
  Phys ph;
  ph.rho_h = p->rho_h;
  ph.rho_l = p->rho_l;
  ph.tau_h = 3.0 * p->nu_h + 0.5;
  ph.tau_l = 3.0 * p->nu_l + 0.5;
  ph.beta = 12.0 * p->sigma / p->xi;
  ph.kappa = 1.5 * p->sigma * p->xi;
  ph.inv_xi = 1.0 / p->xi;
  ph.omega_phi = 1.0 / (3.0 * p->mobility + 0.5);
  ph.gx = p->gravity[0];
  ph.gy = p->gravity[1];
  ph.gz = p->gravity[2];
  return ph;
}

}  // namespace

struct pfl_batch {
  int count;
  int prec;
  int device;
  cudaStream_t stream;
  char* ws;
  std::vector<pfl_params> p;
  std::vector<BInst> inst;     // host copy of the table
  std::vector<size_t> off;     // workspace offset of each instance's buffers
  size_t table_off, tiles_off, stage_off, red_off;
  BInst* d_inst;
  unsigned* d_tick;  // device step counter (seed of the FP16 stochastic rounding)
  ClassPlan cls[NCLASS];
  int cur, swapped;
  long long t;
  cudaGraphExec_t graph;
  int sms, tuned;
};

namespace {

struct BLayout {
  std::vector<size_t> off;
  size_t table, tiles, stage, red, total;
};

size_t inst_bytes(const pfl_params& p) {
  const size_t N = (size_t)p.nx * p.ny * p.nz;
  return align256(15 * N * pop_bytes(p.precision)) + align256(27 * N * pop_bytes(p.precision)) +
         2 * align256(N * phi_bytes(p.precision));
}

BLayout blayout(const pfl_params* p, int count) {
  BLayout L;
  size_t off = 0, maxN = 0, tiles = 0;
  for (int i = 0; i < count; ++i) {
    L.off.push_back(off);
    off += inst_bytes(p[i]);
    const size_t N = (size_t)p[i].nx * p[i].ny * p[i].nz;
    maxN = std::max(maxN, N);
    tiles += (N + 127) / 128;  // the largest tile count over the shapes (128 threads)
  }
  L.table = off;
  off = align256(off + (size_t)count * sizeof(BInst) + 256);
  L.tiles = off;
  off = align256(off + tiles * sizeof(BTile));
  L.stage = off;
  off = align256(off + (maxN + 16) * sizeof(double));
  L.red = off;
  off = align256(off + (DIAG_BLOCKS * 9 + 16) * sizeof(double));
  L.total = off;
  return L;
}

template <int PREC>
void launch_class_step(pfl_batch* b, const ClassPlan& c) {
  if (c.ntiles == 0) return;
  const int g = c.shape.grid;
  if (c.shape.threads == 128) {
    if (b->swapped)
      k_batch_step<PREC, 1, 128><<<g, 128, 0, b->stream>>>(b->d_inst, c.tiles, c.ntiles, b->cur, b->d_tick);
    else
      k_batch_step<PREC, 0, 128><<<g, 128, 0, b->stream>>>(b->d_inst, c.tiles, c.ntiles, b->cur, b->d_tick);
  } else {
    if (b->swapped)
      k_batch_step<PREC, 1, 256><<<g, 256, 0, b->stream>>>(b->d_inst, c.tiles, c.ntiles, b->cur, b->d_tick);
    else
      k_batch_step<PREC, 0, 256><<<g, 256, 0, b->stream>>>(b->d_inst, c.tiles, c.ntiles, b->cur, b->d_tick);
  }
}

template <int PREC>
void launch_class_phi(pfl_batch* b, const ClassPlan& c, unsigned* tick) {
  if (c.ntiles == 0) return;
  const int g = c.shape.grid;
  // after the step kernel flipped `swapped`: READ_ODD = swapped
  if (c.shape.threads == 128) {
    if (b->swapped)
      k_batch_phi<PREC, 1, 128><<<g, 128, 0, b->stream>>>(b->d_inst, c.tiles, c.ntiles, b->cur, tick);
    else
      k_batch_phi<PREC, 0, 128><<<g, 128, 0, b->stream>>>(b->d_inst, c.tiles, c.ntiles, b->cur, tick);
  } else {
    if (b->swapped)
      k_batch_phi<PREC, 1, 256><<<g, 256, 0, b->stream>>>(b->d_inst, c.tiles, c.ntiles, b->cur, tick);
    else
      k_batch_phi<PREC, 0, 256><<<g, 256, 0, b->stream>>>(b->d_inst, c.tiles, c.ntiles, b->cur, tick);
  }
}

// one lattice step of every instance: stream-collide of all classes, then phi
template <int PREC>
void batch_step_once(pfl_batch* b) {
  for (int k = 0; k < NCLASS; ++k) launch_class_step<PREC>(b, b->cls[k]);
  b->swapped ^= 1;
  int last = -1;
  for (int k = 0; k < NCLASS; ++k)
    if (b->cls[k].ntiles) last = k;
  for (int k = 0; k < NCLASS; ++k) launch_class_phi<PREC>(b, b->cls[k], k == last ? b->d_tick : nullptr);
  b->cur = 1 - b->cur;
  b->t += 1;
}

void batch_step_dispatch(pfl_batch* b) {
  switch (b->prec) {
    case PFL_FP64: batch_step_once<0>(b); break;
    case PFL_FP32: batch_step_once<1>(b); break;
    default: batch_step_once<2>(b); break;
  }
}

// Work list of one class for a given tile size (threads per block).
pfl_status build_tiles(pfl_batch* b, ClassPlan& c, int threads, BTile* dst) {
  std::vector<BTile> v;
  // larger instances first: their tiles start early in the grid-stride walk
  std::vector<int> order = c.members;
  std::sort(order.begin(), order.end(), [&](int a, int q) { return b->inst[a].geo.N > b->inst[q].geo.N; });
  for (int i : order)
    for (unsigned c0 = 0; c0 < b->inst[i].geo.N; c0 += threads) v.push_back(BTile{i, c0});
  c.tiles = dst;
  c.ntiles = (int)v.size();
  if (!v.empty())
    BTRY(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(BTile), cudaMemcpyHostToDevice, b->stream));
  BTRY(cudaStreamSynchronize(b->stream));
  return PFL_OK;
}

template <int PREC>
void launch_init_one(pfl_batch* b, int i, long long c0, long long cnt, const double* phi0, const double* ux,
                     const double* uy, const double* uz, const double* p0) {
  Geo geo;
  geo.nx = b->p[i].nx;
  geo.ny = b->p[i].ny;
  geo.nz = b->p[i].nz;
  for (int a = 0; a < 3; ++a) geo.wall[a] = b->p[i].bc[2 * a] == PFL_NOSLIP;
  geo.N = b->inst[i].geo.N;
  k_init<PREC, 15><<<blocks_for(cnt, 256), 256, 0, b->stream>>>(geo, (typename Store<PREC>::S*)b->inst[i].h,
                                                            (typename Store<PREC>::S*)b->inst[i].g, c0, cnt, phi0, ux,
                                                            uy, uz, p0);
}

template <int PREC>
void launch_phi_one(pfl_batch* b, int i) {
  const BInst& I = b->inst[i];
  k_phi32<PREC, 15, 0><<<blocks_for(I.geo.N, 256), 256, 0, b->stream>>>(
      I.geo, (const typename Store<PREC>::S*)I.h, (const typename Store<PREC>::PhiT*)I.phi[1],
      (typename Store<PREC>::PhiT*)I.phi[0]);
}

// Equilibrium start of every instance (zero shifts in phi[1], phi into phi[0]).
pfl_status initial_state(pfl_batch* b, const double* const* phi0, const double* const* u0, const double* const* p0) {
  double* st = (double*)(b->ws + b->stage_off);
  for (int i = 0; i < b->count; ++i) {
    const long long N = b->inst[i].geo.N;
    const long long chunk = N / 5 > 0 ? N / 5 : 1;
    for (long long c0 = 0; c0 < N; c0 += chunk) {
      const long long cnt = (N - c0 < chunk) ? N - c0 : chunk;
      const double* u = u0 ? u0[i] : nullptr;
      const double* pp = p0 ? p0[i] : nullptr;
      BTRY(cudaMemcpyAsync(st, phi0[i] + c0, cnt * 8, cudaMemcpyDefault, b->stream));
      if (u) {
        BTRY(cudaMemcpyAsync(st + cnt, u + c0, cnt * 8, cudaMemcpyDefault, b->stream));
        BTRY(cudaMemcpyAsync(st + 2 * cnt, u + N + c0, cnt * 8, cudaMemcpyDefault, b->stream));
        BTRY(cudaMemcpyAsync(st + 3 * cnt, u + 2 * N + c0, cnt * 8, cudaMemcpyDefault, b->stream));
      }
      if (pp) BTRY(cudaMemcpyAsync(st + 4 * cnt, pp + c0, cnt * 8, cudaMemcpyDefault, b->stream));
      switch (b->prec) {
        case PFL_FP64:
          launch_init_one<0>(b, i, c0, cnt, st, u ? st + cnt : nullptr, u ? st + 2 * cnt : nullptr,
                             u ? st + 3 * cnt : nullptr, pp ? st + 4 * cnt : nullptr);
          break;
        case PFL_FP32:
          launch_init_one<1>(b, i, c0, cnt, st, u ? st + cnt : nullptr, u ? st + 2 * cnt : nullptr,
                             u ? st + 3 * cnt : nullptr, pp ? st + 4 * cnt : nullptr);
          break;
        default:
          launch_init_one<2>(b, i, c0, cnt, st, u ? st + cnt : nullptr, u ? st + 2 * cnt : nullptr,
                             u ? st + 3 * cnt : nullptr, pp ? st + 4 * cnt : nullptr);
          break;
      }
      BTRY(cudaGetLastError());
      BTRY(cudaStreamSynchronize(b->stream));
    }
    BTRY(cudaMemsetAsync(b->inst[i].phi[1], 0, (size_t)N * phi_bytes(b->prec), b->stream));
    switch (b->prec) {
      case PFL_FP64: launch_phi_one<0>(b, i); break;
      case PFL_FP32: launch_phi_one<1>(b, i); break;
      default: launch_phi_one<2>(b, i); break;
    }
    BTRY(cudaGetLastError());
  }
  b->cur = 0;
  b->swapped = 0;
  b->t = 0;
  BTRY(cudaMemsetAsync(b->d_tick, 0, sizeof(unsigned), b->stream));
  BTRY(cudaStreamSynchronize(b->stream));
  return PFL_OK;
}

int resident_blocks(int prec, int threads) {
  int nb = 0;
  const void* fn = nullptr;
  if (prec == PFL_FP64)
    fn = threads == 128 ? (const void*)k_batch_step<0, 1, 128> : (const void*)k_batch_step<0, 1, 256>;
  else if (prec == PFL_FP32)
    fn = threads == 128 ? (const void*)k_batch_step<1, 1, 128> : (const void*)k_batch_step<1, 1, 256>;
  else
    fn = threads == 128 ? (const void*)k_batch_step<2, 1, 128> : (const void*)k_batch_step<2, 1, 256>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  return nb < 1 ? 1 : nb;
}

// Autotuner: for each class, time every (threads, grid) candidate over two
// lattice steps of the whole batch (other classes at their current shape) and
// keep the fastest.  Grids are multiples of the SM count times the resident
// blocks per SM, capped by the tile count.
pfl_status tune(pfl_batch* b) {
  BTile* tiles_base = (BTile*)(b->ws + b->tiles_off);
  size_t tile_cursor = 0;
  cudaEvent_t e0, e1;
  BTRY(cudaEventCreate(&e0));
  BTRY(cudaEventCreate(&e1));
  // default shapes first (so every class can run while another is tuned)
  BTile* dst[NCLASS];
  for (int k = 0; k < NCLASS; ++k) {
    dst[k] = tiles_base + tile_cursor;
    size_t worst = 0;
    for (int i : b->cls[k].members) worst += (b->inst[i].geo.N + 127) / 128;
    tile_cursor += worst;
    pfl_status s = build_tiles(b, b->cls[k], 128, dst[k]);
    if (s != PFL_OK) return s;
    b->cls[k].shape = Shape{128, std::min(b->cls[k].ntiles, b->sms * resident_blocks(b->prec, 128))};
  }
  for (int k = 0; k < NCLASS; ++k) {
    ClassPlan& c = b->cls[k];
    if (c.members.empty()) continue;
    float best = 1e30f;
    Shape best_shape = c.shape;
    for (int threads : {128, 256}) {
      pfl_status s = build_tiles(b, c, threads, dst[k]);
      if (s != PFL_OK) return s;
      const int res = resident_blocks(b->prec, threads);
      for (int mult : {1, 2, 4}) {
        Shape sh{threads, std::max(1, std::min(c.ntiles, mult * b->sms * res))};
        c.shape = sh;
        batch_step_dispatch(b);  // warm-up
        batch_step_dispatch(b);
        BTRY(cudaEventRecord(e0, b->stream));
        batch_step_dispatch(b);
        batch_step_dispatch(b);
        BTRY(cudaEventRecord(e1, b->stream));
        BTRY(cudaEventSynchronize(e1));
        BTRY(cudaGetLastError());
        float ms = 0;
        BTRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
          best = ms;
          best_shape = sh;
        }
        if (sh.grid == c.ntiles) break;  // larger grids are the same launch
      }
    }
    pfl_status s = build_tiles(b, c, best_shape.threads, dst[k]);
    if (s != PFL_OK) return s;
    c.shape = best_shape;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tuned = 1;
  return PFL_OK;
}

pfl_status capture_graph(pfl_batch* b) {
  // 2 * GRAPH_PAIRS steps starting at parity 0 / buffer 0 return there.  The
  // caller's stream may be the legacy default stream, which cannot be
  // captured: capture on a private stream, replay on the caller's.
  cudaGraph_t g;
  const int cur0 = b->cur, sw0 = b->swapped;
  const long long t0 = b->t;
  cudaStream_t user = b->stream, cap;
  BTRY(cudaStreamSynchronize(user));
  BTRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  b->stream = cap;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int s = 0; s < 2 * GRAPH_PAIRS; ++s) batch_step_dispatch(b);
    e = cudaStreamEndCapture(cap, &g);
  }
  b->stream = user;
  cudaStreamDestroy(cap);
  b->cur = cur0;
  b->swapped = sw0;
  b->t = t0;
  if (e != cudaSuccess) return bfail(PFL_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(PFL_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return PFL_OK;
}

}  // namespace

extern "C" {

size_t pfl_batch_workspace_bytes(const pfl_params* params, int count) {
  if (!params || count < 1) return 0;
  for (int i = 0; i < count; ++i) {
    if (!check_params(&params[i]).empty()) return 0;
    if (params[i].precision != params[0].precision || params[i].collision != PFL_MRT) return 0;
    if (qh_of(&params[i]) != 15 || params[i].solids) return 0;
    if (27ull * params[i].nx * params[i].ny * params[i].nz >= (1ull << 32)) return 0;
  }
  return blayout(params, count).total;
}

pfl_status pfl_batch_init(const pfl_params* params, int count, const double* const* phi0, const double* const* u0,
                          const double* const* p0, void* workspace, size_t workspace_bytes, void* stream, int tune_shapes,
                          pfl_batch** out) {
  if (!out) return bfail(PFL_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!params || count < 1 || !phi0) return bfail(PFL_ERR_ARG, "need count >= 1 parameter sets and phi0 arrays");
  for (int i = 0; i < count; ++i) {
    std::string why = check_params(&params[i]);
    if (!why.empty()) return bfail(PFL_ERR_ARG, "instance " + std::to_string(i) + ": " + why);
    if (params[i].precision != params[0].precision)
      return bfail(PFL_ERR_ARG, "all instances of a batch share one precision");
    if (params[i].collision != PFL_MRT) return bfail(PFL_ERR_ARG, "the batch runs the MRT collision");
    if (qh_of(&params[i]) != 15) return bfail(PFL_ERR_ARG, "the batch steps D3Q15 phase fields only");
    if (params[i].solids) return bfail(PFL_ERR_ARG, "the batch takes no solid cells");
    if (27ull * params[i].nx * params[i].ny * params[i].nz >= (1ull << 32))
      return bfail(PFL_ERR_ARG, "instance " + std::to_string(i) + " too large for 32-bit indices");
    if (!phi0[i]) return bfail(PFL_ERR_ARG, "phi0 of instance " + std::to_string(i) + " is NULL");
  }
  if (!workspace || ((uintptr_t)workspace & 255)) return bfail(PFL_ERR_ARG, "workspace must be 256-byte aligned device memory");
  const BLayout L = blayout(params, count);
  if (workspace_bytes < L.total)
    return bfail(PFL_ERR_OOM, "workspace holds " + std::to_string(workspace_bytes) + " bytes, needs " +
                                  std::to_string(L.total));
  int device = 0;
  if (!is_device_ptr(workspace, &device)) return bfail(PFL_ERR_ARG, "workspace is not device memory");
  BTRY(cudaSetDevice(device));

  pfl_batch* b = new pfl_batch();
  b->count = count;
  b->prec = params[0].precision;
  b->device = device;
  b->stream = (cudaStream_t)stream;
  b->ws = (char*)workspace;
  b->p.assign(params, params + count);
  b->off = L.off;
  b->table_off = L.table;
  b->tiles_off = L.tiles;
  b->stage_off = L.stage;
  b->red_off = L.red;
  b->d_inst = (BInst*)(b->ws + L.table);
  b->d_tick = (unsigned*)(b->ws + L.table + align256((size_t)count * sizeof(BInst)));
  b->graph = nullptr;
  b->tuned = 0;
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, device);
  const size_t S = pop_bytes(b->prec), P = phi_bytes(b->prec);
  for (int i = 0; i < count; ++i) {
    const pfl_params& q = params[i];
    BInst I;
    const unsigned N = (unsigned)((size_t)q.nx * q.ny * q.nz);
    I.geo.nx = q.nx;
    I.geo.ny = q.ny;
    I.geo.nz = q.nz;
    I.geo.N = N;
    I.geo.dx = make_fastdiv((unsigned)q.nx);
    I.geo.dy = make_fastdiv((unsigned)q.ny);
    for (int a = 0; a < 3; ++a) I.geo.wall[a] = q.bc[2 * a] == PFL_NOSLIP;
    if (!fastdiv_ok((unsigned)q.nx, N) || !fastdiv_ok((unsigned)q.ny, N / q.nx)) {
      delete b;
      return bfail(PFL_ERR_STATE, "integer divider self-check failed");
    }
    I.ph = phys_of(&q);
    char* base = b->ws + L.off[i];
    I.h = base;
    I.g = base + align256(15 * (size_t)N * S);
    I.phi[0] = base + align256(15 * (size_t)N * S) + align256(27 * (size_t)N * S);
    I.phi[1] = (char*)I.phi[0] + align256((size_t)N * P);
    I.active = 1;
    I.frozen_cur = 0;
    I.frozen_swapped = 0;
    b->inst.push_back(I);
    b->cls[N < SMALL_CELLS ? 0 : 1].members.push_back(i);
  }
  pfl_status s = PFL_OK;
  cudaError_t e = cudaMemcpyAsync(b->d_inst, b->inst.data(), count * sizeof(BInst), cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) s = bfail(PFL_ERR_CUDA, cudaGetErrorString(e));
  if (s == PFL_OK) s = initial_state(b, phi0, u0, p0);
  if (s == PFL_OK) {
    if (tune_shapes) {
      s = tune(b);
      if (s == PFL_OK) s = initial_state(b, phi0, u0, p0);  // the timing steps moved the state
    } else {
      // default shapes without timing: 128 threads, grid = SMs x resident blocks
      BTile* base = (BTile*)(b->ws + b->tiles_off);
      size_t cursor = 0;
      for (int k = 0; k < NCLASS && s == PFL_OK; ++k) {
        s = build_tiles(b, b->cls[k], 128, base + cursor);
        for (int i : b->cls[k].members) cursor += (b->inst[i].geo.N + 127) / 128;
        b->cls[k].shape = Shape{128, std::max(1, std::min(b->cls[k].ntiles, b->sms * resident_blocks(b->prec, 128)))};
      }
    }
  }
  if (s == PFL_OK) s = capture_graph(b);
  if (s != PFL_OK) {
    delete b;
    return s;
  }
  *out = b;
  return PFL_OK;
}

pfl_status pfl_batch_step(pfl_batch* b, int n) {
  if (!b) return bfail(PFL_ERR_ARG, "batch is NULL");
  if (n < 0) return bfail(PFL_ERR_ARG, "n_steps must be >= 0");
  BTRY(cudaSetDevice(b->device));
  int done = 0;
  // whole graphs only from the graph's starting roles (even parity, buffer 0)
  while (n - done >= 2 * GRAPH_PAIRS && b->swapped == 0 && b->cur == 0) {
    BTRY(cudaGraphLaunch(b->graph, b->stream));
    b->t += 2 * GRAPH_PAIRS;
    done += 2 * GRAPH_PAIRS;
  }
  for (; done < n; ++done) batch_step_dispatch(b);
  BTRY(cudaGetLastError());
  return PFL_OK;
}

pfl_status pfl_batch_fields(pfl_batch* b, int i, double* phi, double* rho, double* p, double* u) {
  if (!b) return bfail(PFL_ERR_ARG, "batch is NULL");
  if (i < 0 || i >= b->count) return bfail(PFL_ERR_ARG, "instance index out of range");
  BTRY(cudaSetDevice(b->device));
  const BInst& I = b->inst[i];
  const int cur = I.active ? b->cur : I.frozen_cur;
  const int swapped = I.active ? b->swapped : I.frozen_swapped;
  Geo geo;
  geo.nx = (int)I.geo.nx;
  geo.ny = (int)I.geo.ny;
  geo.nz = (int)I.geo.nz;
  for (int a = 0; a < 3; ++a) geo.wall[a] = I.geo.wall[a];
  geo.N = I.geo.N;
  const long long N = geo.N;
  double* want[6] = {phi, rho, p, u, u ? u + N : nullptr, u ? u + 2 * N : nullptr};
  double* st = (double*)(b->ws + b->stage_off);
  for (int k = 0; k < 6; ++k) {
    if (!want[k]) continue;
    const bool dev = is_device_ptr(want[k]);
    double* o[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    o[k] = dev ? want[k] : st;
    const unsigned nb = blocks_for(N, 256);
#define BF(PREC)                                                                                                  \
  if (swapped)                                                                                                    \
    k_fields<PREC, 15, 1><<<nb, 256, 0, b->stream>>>(geo, I.ph, (const Store<PREC>::S*)I.g,                           \
                                                 (const Store<PREC>::PhiT*)I.phi[cur], o[0], o[1],                 \
                                                 o[2], o[3], o[4], o[5]);                                         \
  else                                                                                                            \
    k_fields<PREC, 15, 0><<<nb, 256, 0, b->stream>>>(geo, I.ph, (const Store<PREC>::S*)I.g,                           \
                                                 (const Store<PREC>::PhiT*)I.phi[cur], o[0], o[1],                 \
                                                 o[2], o[3], o[4], o[5]);
    switch (b->prec) {
      case PFL_FP64: BF(0) break;
      case PFL_FP32: BF(1) break;
      default: BF(2) break;
    }
#undef BF
    BTRY(cudaGetLastError());
    if (!dev) BTRY(cudaMemcpyAsync(want[k], st, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BTRY(cudaStreamSynchronize(b->stream));
  }
  return PFL_OK;
}

pfl_status pfl_batch_diag(pfl_batch* b, double* out, long long* nonfinite) {
  if (!b) return bfail(PFL_ERR_ARG, "batch is NULL");
  BTRY(cudaSetDevice(b->device));
  double* part = (double*)(b->ws + b->red_off);
  double* res = part + DIAG_BLOCKS * 9;
  int bad = 0;
  bool table_dirty = false;
  for (int i = 0; i < b->count; ++i) {
    BInst& I = b->inst[i];
    Geo geo;
    geo.nx = (int)I.geo.nx;
    geo.ny = (int)I.geo.ny;
    geo.nz = (int)I.geo.nz;
    geo.wall[0] = geo.wall[1] = geo.wall[2] = 0;
    geo.N = I.geo.N;
    const int cur = I.active ? b->cur : I.frozen_cur;
    if (b->prec == PFL_FP64)
      k_diag<double><<<DIAG_BLOCKS, DIAG_THREADS, 0, b->stream>>>(geo, (const double*)I.phi[cur], part);
    else
      k_diag<float><<<DIAG_BLOCKS, DIAG_THREADS, 0, b->stream>>>(geo, (const float*)I.phi[cur], part);
    k_diag_final<<<9, 32, 0, b->stream>>>(part, DIAG_BLOCKS, res);
    BTRY(cudaGetLastError());
    double h[9];
    BTRY(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    BTRY(cudaStreamSynchronize(b->stream));
    if (out)
      for (int k = 0; k < 8; ++k) out[8 * i + k] = h[k];
    const long long nf = (long long)h[8];
    if (nonfinite) nonfinite[i] = nf;
    if (nf > 0) {
      ++bad;
      if (I.active) {  // an unstable instance stops; the others go on
        I.active = 0;
        I.frozen_cur = b->cur;
        I.frozen_swapped = b->swapped;
        table_dirty = true;
      }
    }
  }
  if (table_dirty) {
    BTRY(cudaMemcpyAsync(b->d_inst, b->inst.data(), b->count * sizeof(BInst), cudaMemcpyHostToDevice, b->stream));
    BTRY(cudaStreamSynchronize(b->stream));
  }
  if (bad) return bfail(PFL_ERR_UNSTABLE, std::to_string(bad) + " instances hold non-finite phi and were stopped");
  return PFL_OK;
}

pfl_status pfl_batch_shapes(const pfl_batch* b, int* threads, int* grid, int* ntiles) {
  if (!b) return bfail(PFL_ERR_ARG, "batch is NULL");
  for (int k = 0; k < NCLASS; ++k) {
    if (threads) threads[k] = b->cls[k].shape.threads;
    if (grid) grid[k] = b->cls[k].shape.grid;
    if (ntiles) ntiles[k] = b->cls[k].ntiles;
  }
  return PFL_OK;
}

long long pfl_batch_time(const pfl_batch* b) { return b ? b->t : -1; }

void pfl_batch_destroy(pfl_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  delete b;
}

}  // extern "C"
