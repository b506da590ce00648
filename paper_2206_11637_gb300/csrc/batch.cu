// Batched PFLBM: many independent lattices of uneven size and their own
// parameters (M, xi, sigma, ...) advanced together.
//
// Every lattice time step is one persistent launch of the fused two-array
// step per class of instances (quasi-2-D lattices with one z plane, and 3-D
// lattices): a grid of (SMs x resident blocks x m) blocks walks a device work
// list of tiles (instance, xy tile, z chunk), and each block runs the same
// tile code as the single-lattice step (zm_tile: the phi stencil from a
// shared-memory ring marched along z, both collisions, push streaming into the
// instance's other array pair) with the instance's geometry and parameters,
// read from a device table into shared memory.  phi of the stored state is
// formed in the step itself, so there is no separate phi pass.  The launch
// shapes -- the tile height of the quasi-2-D class, the z chunk of the 3-D
// class, the grid size of both -- are chosen at init by timing the candidates
// on the initial state (which is then rebuilt).  The step loop is captured
// once into a CUDA graph of 2 G lattice steps (an even count, so the array
// pairs return to their starting roles) and replayed.
//
// An instance of the batch evolves exactly like the same lattice run alone by
// the fused single-lattice step: the per-cell arithmetic is the same code.
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
  void* h[2];   // the two array pairs of the fused step
  void* g[2];
  void* phi;    // phi written by the steps (phi of the state each step started from)
  void* phic;   // phi of the current state, formed on demand (fields, diagnostics)
  int zc;       // z planes per tile of the work list
  int active;
  int frozen_ab;  // host bookkeeping: the pair holding the state when the instance stopped
};

struct BTile {
  int inst;
  unsigned short bx, by, bz, pad;
};

constexpr int NCLASS = 2;     // class 0: one z plane (quasi-2-D), class 1: 3-D
constexpr int GRAPH_PAIRS = 8;  // a graph holds 2 * GRAPH_PAIRS lattice steps

// Tiles are handed out by a counter (PFL_BATCH_DYNAMIC = 1): a block takes the
// next tile of the list when it finishes one, so the large-first list ends
// with small tiles on every SM; 0 walks the list with a fixed stride.
#ifndef PFL_BATCH_DYNAMIC
#define PFL_BATCH_DYNAMIC 1
#endif

// One lattice step of the instances of one class: a persistent walk over the
// class's work list (ab: the array pair holding the current state), by blocks
// of TX x TY threads, resident like the single-lattice step's (the same
// threads per SM).  ctr: the class's two counters (next tile, blocks done),
// zero at launch; the last block to finish zeroes them for the next launch,
// which stream order puts after this one.
template <int PREC, int TX, int TY, int FLAT>
__global__ void __launch_bounds__(TX * TY, (PREC == 0 ? PFL_ZM_MINB_FP64 : PFL_ZM_MINB) * ZM_TX * ZM_TY / (TX * TY))
    k_batch_zm(const BInst* __restrict__ inst, const BTile* __restrict__ tiles, int ntiles, int ab,
               unsigned* __restrict__ ctr) {
  typedef typename Store<PREC>::S S;
  typedef typename Store<PREC>::PhiT PhiT;
  __shared__ Geo32 sgeo;
  __shared__ Phys sph;
  __shared__ int sact;
  __shared__ void* sptr[5];
  __shared__ int szc;
  __shared__ int snext;
  if (PFL_ZM_PDL) asm volatile("griddepcontrol.wait;" ::: "memory");
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int t = blockIdx.x;; t += gridDim.x) {
    if (PFL_BATCH_DYNAMIC) {
      if (tid == 0) snext = (int)atomicAdd(ctr, 1u);
      __syncthreads();
      t = snext;
    }
    if (t >= ntiles) break;
    const BTile tile = tiles[t];
    if (tid == 0) {
      const BInst* I = inst + tile.inst;
      sgeo = I->geo;
      sph = I->ph;
      sact = I->active;
      sptr[0] = I->h[ab];
      sptr[1] = I->g[ab];
      sptr[2] = I->h[1 - ab];
      sptr[3] = I->g[1 - ab];
      sptr[4] = I->phi;
      szc = I->zc;
    }
    __syncthreads();
    if (sact)
      zm_tile<PREC, 15, TY, FLAT, 0, TX>(sgeo, sph, (const S*)sptr[0], (const S*)sptr[1], (S*)sptr[2], (S*)sptr[3], nullptr,
                                     (PhiT*)sptr[4], szc, 0u, nullptr, nullptr, nullptr, tile.bx, tile.by, tile.bz);
    __syncthreads();  // the next tile refills the shared rings, the instance slot and snext
  }
  if (PFL_BATCH_DYNAMIC && tid == 0 && atomicAdd(ctr + 1, 1u) == gridDim.x - 1) {
    ctr[0] = 0;  // every block has taken its last ticket
    ctr[1] = 0;
  }
}

struct Shape {
  int tx;    // tile width: 32, or 16 (FP32) for instances a few tiles wide
  int ty;    // tile height (threads per block = tx * ty): 4 or 8 for one z plane, 8 or 16 in 3-D
  int zc;    // z planes per tile (3-D class; 0 = the whole lattice)
  int grid;  // blocks of the persistent launch
};

// Tile shapes (tx, ty) of each class: every precision takes the first two, FP32
// also the third.  A 16-wide tile leaves fewer threads idle on lattices that
// are not a multiple of 32 wide (a 40-wide drop fills 40 of 64 columns in
// 32-wide tiles, 40 of 48 in 16-wide ones) for a larger share of ring cells.
constexpr int NSHAPE = 3;
constexpr int SHAPES[NCLASS][NSHAPE][2] = {{{32, 4}, {32, 8}, {16, 8}}, {{32, 8}, {16, 8}, {16, 16}}};
constexpr int shapes_for(int prec) { return prec == PFL_FP32 ? 3 : 2; }

struct ClassPlan {
  std::vector<int> members;
  Shape shape{32, 8, 0, 0};
  BTile* tiles = nullptr;  // device
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
  size_t table_off, tiles_off, stage_off, red_off, ctr_off;
  BInst* d_inst;
  ClassPlan cls[NCLASS];
  int ab;                      // the array pair holding the current state
  long long t;
  cudaGraphExec_t graph;
  int sms, tuned;
};

namespace {

struct BLayout {
  std::vector<size_t> off;
  size_t table, tiles, stage, red, ctr, total;
};

size_t inst_bytes(const pfl_params& p) {
  const size_t N = (size_t)p.nx * p.ny * p.nz;
  return 2 * (align256(15 * N * pop_bytes(p.precision)) + align256(27 * N * pop_bytes(p.precision))) +
         2 * align256(N * phi_bytes(p.precision));
}

// tiles of one instance for a tile shape and z chunk
size_t tiles_of(const pfl_params& p, int tx, int ty, int zc) {
  const size_t zc_ = zc > 0 && zc < p.nz ? (size_t)zc : (size_t)p.nz;
  return (size_t)((p.nx + tx - 1) / tx) * ((p.ny + ty - 1) / ty) * ((p.nz + zc_ - 1) / zc_);
}

BLayout blayout(const pfl_params* p, int count) {
  BLayout L;
  size_t off = 0, maxN = 0, tiles = 0;
  for (int i = 0; i < count; ++i) {
    L.off.push_back(off);
    off += inst_bytes(p[i]);
    const size_t N = (size_t)p[i].nx * p[i].ny * p[i].nz;
    maxN = std::max(maxN, N);
    tiles += tiles_of(p[i], 16, 4, 1);  // at least as many as any shape takes
  }
  L.table = off;
  off = align256(off + (size_t)count * sizeof(BInst) + 256);
  L.tiles = off;
  off = align256(off + tiles * sizeof(BTile));
  L.stage = off;
  off = align256(off + (maxN + 16) * sizeof(double));
  L.red = off;
  off = align256(off + (DIAG_BLOCKS * 10 + 32) * sizeof(double));
  L.ctr = off;  // tile counters of the two classes
  off = align256(off + 2 * NCLASS * sizeof(unsigned));
  L.total = off;
  return L;
}

int shape_index(int cls, const Shape& sh) {
  for (int j = 0; j < NSHAPE; ++j)
    if (SHAPES[cls][j][0] == sh.tx && SHAPES[cls][j][1] == sh.ty) return j;
  return -1;
}

// kernel function of (precision, class, shape); FP64 has the first two shapes only
template <int PREC, int CLS>
const void* batch_fn(int j) {
  if (j == 0) return (const void*)k_batch_zm<PREC, SHAPES[CLS][0][0], SHAPES[CLS][0][1], CLS == 0>;
  if (j == 1) return (const void*)k_batch_zm<PREC, SHAPES[CLS][1][0], SHAPES[CLS][1][1], CLS == 0>;
  if constexpr (PREC == 1) {
    if (j == 2) return (const void*)k_batch_zm<PREC, SHAPES[CLS][2][0], SHAPES[CLS][2][1], CLS == 0>;
  }
  return nullptr;
}

template <int PREC, int CLS, int J>
void launch_shape(pfl_batch* b, const ClassPlan& c) {
  k_batch_zm<PREC, SHAPES[CLS][J][0], SHAPES[CLS][J][1], CLS == 0>
      <<<c.shape.grid, dim3(SHAPES[CLS][J][0], SHAPES[CLS][J][1]), 0, b->stream>>>(
          b->d_inst, c.tiles, c.ntiles, b->ab, (unsigned*)(b->ws + b->ctr_off) + 2 * CLS);
}

template <int PREC, int CLS>
void launch_class(pfl_batch* b, const ClassPlan& c) {
  const int j = shape_index(CLS, c.shape);
  if (j == 0) launch_shape<PREC, CLS, 0>(b, c);
  if (j == 1) launch_shape<PREC, CLS, 1>(b, c);
  if constexpr (PREC == 1) {
    if (j == 2) launch_shape<PREC, CLS, 2>(b, c);
  }
}

template <int PREC>
void launch_class_step(pfl_batch* b, const ClassPlan& c, int cls) {
  if (c.ntiles == 0) return;
  if (cls == 0)
    launch_class<PREC, 0>(b, c);
  else
    launch_class<PREC, 1>(b, c);
}

// one lattice step of every instance: the fused step of both classes
template <int PREC>
void batch_step_once(pfl_batch* b) {
  for (int k = 0; k < NCLASS; ++k) launch_class_step<PREC>(b, b->cls[k], k);
  b->ab ^= 1;
  b->t += 1;
}

void batch_step_dispatch(pfl_batch* b) {
  if (b->prec == PFL_FP64)
    batch_step_once<0>(b);
  else
    batch_step_once<1>(b);
}

// Work list of one class for a shape: every instance's (xy tile, z chunk)
// tiles, larger instances first (their tiles start early in the walk).
pfl_status build_tiles(pfl_batch* b, ClassPlan& c, const Shape& sh, BTile* dst) {
  std::vector<BTile> v;
  std::vector<int> order = c.members;
  std::sort(order.begin(), order.end(), [&](int a, int q) { return b->inst[a].geo.N > b->inst[q].geo.N; });
  for (int i : order) {
    const Geo32& g = b->inst[i].geo;
    const int zc = sh.zc > 0 && sh.zc < (int)g.nz ? sh.zc : (int)g.nz;
    b->inst[i].zc = zc;
    const int nbx = (g.nx + sh.tx - 1) / sh.tx, nby = (g.ny + sh.ty - 1) / sh.ty, nbz = (g.nz + zc - 1) / zc;
    for (int bz = 0; bz < nbz; ++bz)
      for (int by = 0; by < nby; ++by)
        for (int bx = 0; bx < nbx; ++bx)
          v.push_back(BTile{i, (unsigned short)bx, (unsigned short)by, (unsigned short)bz, 0});
  }
  c.tiles = dst;
  c.ntiles = (int)v.size();
  if (!v.empty())
    BTRY(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(BTile), cudaMemcpyHostToDevice, b->stream));
  BTRY(cudaMemcpyAsync(b->d_inst, b->inst.data(), b->count * sizeof(BInst), cudaMemcpyHostToDevice, b->stream));
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
  k_init<PREC, 15><<<blocks_for(cnt, 256), 256, 0, b->stream>>>(geo, (typename Store<PREC>::S*)b->inst[i].h[0],
                                                            (typename Store<PREC>::S*)b->inst[i].g[0], c0, cnt, phi0, ux,
                                                            uy, uz, p0);
}

// phi of the current state of instance i (pair `ab`) into its phic buffer
template <int PREC>
void launch_phi_one(pfl_batch* b, int i, int ab) {
  const BInst& I = b->inst[i];
  k_phi32<PREC, 15, 0><<<blocks_for(I.geo.N, 256), 256, 0, b->stream>>>(
      I.geo, (const typename Store<PREC>::S*)I.h[ab], nullptr, (typename Store<PREC>::PhiT*)I.phic);
}

void phi_one(pfl_batch* b, int i, int ab) {
  if (b->prec == PFL_FP64)
    launch_phi_one<0>(b, i, ab);
  else
    launch_phi_one<1>(b, i, ab);
}

// Equilibrium start of every instance in pair 0.
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
      if (b->prec == PFL_FP64)
        launch_init_one<0>(b, i, c0, cnt, st, u ? st + cnt : nullptr, u ? st + 2 * cnt : nullptr,
                           u ? st + 3 * cnt : nullptr, pp ? st + 4 * cnt : nullptr);
      else
        launch_init_one<1>(b, i, c0, cnt, st, u ? st + cnt : nullptr, u ? st + 2 * cnt : nullptr,
                           u ? st + 3 * cnt : nullptr, pp ? st + 4 * cnt : nullptr);
      BTRY(cudaGetLastError());
      BTRY(cudaStreamSynchronize(b->stream));
    }
  }
  b->ab = 0;
  b->t = 0;
  BTRY(cudaStreamSynchronize(b->stream));
  return PFL_OK;
}

int resident_blocks(int prec, int cls, const Shape& sh) {
  int nb = 0;
  const int j = shape_index(cls, sh);
  const void* fn = prec == PFL_FP64 ? (cls == 0 ? batch_fn<0, 0>(j) : batch_fn<0, 1>(j))
                                    : (cls == 0 ? batch_fn<1, 0>(j) : batch_fn<1, 1>(j));
  if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, sh.tx * sh.ty, 0) != cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  return nb < 1 ? 1 : nb;
}

// Default shape of a class: 32 x 4 tiles (one z plane) or 32 x 8, the z chunk by
// the cost model of the single-lattice step (waves of resident blocks times
// zc + 1/2, over the class's largest instance), grid = SMs x resident blocks.
Shape default_shape(pfl_batch* b, int k) {
  Shape sh{32, k == 0 ? 4 : 8, 0, 0};
  if (k == 1) {
    int big = -1;
    for (int i : b->cls[k].members)
      if (big < 0 || b->inst[i].geo.N > b->inst[big].geo.N) big = i;
    if (big >= 0) {
      const Geo32& g = b->inst[big].geo;
      const long long slots = (long long)b->sms * resident_blocks(b->prec, 1, sh);
      const long long bxy = (long long)((g.nx + sh.tx - 1) / sh.tx) * ((g.ny + sh.ty - 1) / sh.ty);
      double best = 1e300;
      for (int zc = (int)g.nz; zc >= 1; --zc) {
        const long long blocks = bxy * ((g.nz + zc - 1) / zc);
        const double cost = (double)((blocks + slots - 1) / slots) * (zc + 0.5);
        if (cost < best * (1 - 1e-9)) {
          best = cost;
          sh.zc = zc;
        }
      }
    }
  }
  sh.grid = b->sms * resident_blocks(b->prec, k, sh);
  return sh;
}

// Autotuner: for each class, time every candidate shape over two lattice
// steps of the whole batch (the other class at its current shape) and keep
// the fastest.  Candidates: the class's tile shapes (SHAPES; FP64 the 32-wide
// ones), in 3-D each with the z chunks of the cost model, 8, 16, 32 and the
// whole lattice, and each with grids of 1, 2 and 4 x SMs x resident blocks,
// capped by the tile count.
pfl_status tune(pfl_batch* b) {
  BTile* dst[NCLASS];
  BTile* base = (BTile*)(b->ws + b->tiles_off);
  size_t cursor = 0;
  for (int k = 0; k < NCLASS; ++k) {
    dst[k] = base + cursor;
    for (int i : b->cls[k].members) cursor += tiles_of(b->p[i], 16, 4, 1);
  }
  cudaEvent_t e0, e1;
  BTRY(cudaEventCreate(&e0));
  BTRY(cudaEventCreate(&e1));
  for (int k = 0; k < NCLASS; ++k) {
    b->cls[k].shape = default_shape(b, k);
    pfl_status s = build_tiles(b, b->cls[k], b->cls[k].shape, dst[k]);
    if (s != PFL_OK) return s;
  }
  for (int k = 0; k < NCLASS; ++k) {
    ClassPlan& c = b->cls[k];
    if (c.members.empty()) continue;
    std::vector<Shape> cand;
    const Shape d = c.shape;
    for (int j = 0; j < shapes_for(b->prec); ++j) {
      const int tx = SHAPES[k][j][0], ty = SHAPES[k][j][1];
      if (k == 0) {
        cand.push_back(Shape{tx, ty, 0, 0});
      } else {
        for (int zc : {d.zc, 8, 16, 32, 0}) {
          bool dup = false;
          for (const Shape& q : cand) dup |= q.tx == tx && q.ty == ty && q.zc == zc;
          if (!dup) cand.push_back(Shape{tx, ty, zc, 0});
        }
      }
    }
    float best = 1e30f;
    Shape best_shape = d;
    for (Shape sh : cand) {
      pfl_status s = build_tiles(b, c, sh, dst[k]);
      if (s != PFL_OK) return s;
      const int res = resident_blocks(b->prec, k, sh);
      for (int mult : {1, 2, 4}) {
        sh.grid = std::max(1, std::min(c.ntiles, mult * b->sms * res));
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
    pfl_status s = build_tiles(b, c, best_shape, dst[k]);
    if (s != PFL_OK) return s;
    c.shape = best_shape;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tuned = 1;
  return PFL_OK;
}

pfl_status capture_graph(pfl_batch* b) {
  // 2 * GRAPH_PAIRS steps starting at pair 0 return there.  The caller's
  // stream may be the legacy default stream, which cannot be captured:
  // capture on a private stream, replay on the caller's.
  cudaGraph_t g;
  const int ab0 = b->ab;
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
  b->ab = ab0;
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
    if (qh_of(&params[i]) != 15 || params[i].solids || params[i].precision == PFL_FP16S) return 0;
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
    if (params[i].precision == PFL_FP16S) return bfail(PFL_ERR_ARG, "the batch runs FP64 or FP32 storage");
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
  DeviceScope on_device;
  BTRY(on_device.enter(device));

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
  b->ctr_off = L.ctr;
  b->d_inst = (BInst*)(b->ws + L.table);
  b->graph = nullptr;
  b->tuned = 0;
  b->ab = 0;
  b->t = 0;
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
    char* at = b->ws + L.off[i];
    for (int pr = 0; pr < 2; ++pr) {
      I.h[pr] = at;
      at += align256(15 * (size_t)N * S);
      I.g[pr] = at;
      at += align256(27 * (size_t)N * S);
    }
    I.phi = at;
    I.phic = at + align256((size_t)N * P);
    I.zc = q.nz;
    I.active = 1;
    I.frozen_ab = 0;
    b->inst.push_back(I);
    b->cls[q.nz == 1 ? 0 : 1].members.push_back(i);
  }
  pfl_status s = PFL_OK;
  cudaError_t e = cudaMemcpyAsync(b->d_inst, b->inst.data(), count * sizeof(BInst), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->ctr_off, 0, 2 * NCLASS * sizeof(unsigned), b->stream);
  if (e != cudaSuccess) s = bfail(PFL_ERR_CUDA, cudaGetErrorString(e));
  if (s == PFL_OK) s = initial_state(b, phi0, u0, p0);
  if (s == PFL_OK) {
    if (tune_shapes) {
      s = tune(b);
      if (s == PFL_OK) s = initial_state(b, phi0, u0, p0);  // the timing steps moved the state
    } else {
      BTile* base = (BTile*)(b->ws + b->tiles_off);
      size_t cursor = 0;
      for (int k = 0; k < NCLASS && s == PFL_OK; ++k) {
        b->cls[k].shape = default_shape(b, k);
        s = build_tiles(b, b->cls[k], b->cls[k].shape, base + cursor);
        for (int i : b->cls[k].members) cursor += tiles_of(b->p[i], 16, 4, 1);
        b->cls[k].shape.grid = std::max(1, std::min(b->cls[k].ntiles, b->cls[k].shape.grid));
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
  DeviceScope on_device;
  BTRY(on_device.enter(b->device));
  int done = 0;
  // whole graphs only from the graph's starting roles (pair 0 current)
  while (n - done >= 2 * GRAPH_PAIRS && b->ab == 0) {
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
  DeviceScope on_device;
  BTRY(on_device.enter(b->device));
  const BInst& I = b->inst[i];
  const int ab = I.active ? b->ab : I.frozen_ab;
  Geo geo;
  geo.nx = (int)I.geo.nx;
  geo.ny = (int)I.geo.ny;
  geo.nz = (int)I.geo.nz;
  for (int a = 0; a < 3; ++a) geo.wall[a] = I.geo.wall[a];
  geo.N = I.geo.N;
  const long long N = geo.N;
  phi_one(b, i, ab);
  BTRY(cudaGetLastError());
  double* want[6] = {phi, rho, p, u, u ? u + N : nullptr, u ? u + 2 * N : nullptr};
  double* st = (double*)(b->ws + b->stage_off);
  for (int k = 0; k < 6; ++k) {
    if (!want[k]) continue;
    const bool dev = is_device_ptr(want[k]);
    double* o[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    o[k] = dev ? want[k] : st;
    const unsigned nb = blocks_for(N, 256);
    if (b->prec == PFL_FP64)
      k_fields<0, 15, 0><<<nb, 256, 0, b->stream>>>(geo, I.ph, (const Store<0>::S*)I.g[ab], (const Store<0>::PhiT*)I.phic,
                                                    o[0], o[1], o[2], o[3], o[4], o[5]);
    else
      k_fields<1, 15, 0><<<nb, 256, 0, b->stream>>>(geo, I.ph, (const Store<1>::S*)I.g[ab], (const Store<1>::PhiT*)I.phic,
                                                    o[0], o[1], o[2], o[3], o[4], o[5]);
    BTRY(cudaGetLastError());
    if (!dev) BTRY(cudaMemcpyAsync(want[k], st, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BTRY(cudaStreamSynchronize(b->stream));
  }
  return PFL_OK;
}

pfl_status pfl_batch_diag(pfl_batch* b, double* out, long long* nonfinite) {
  if (!b) return bfail(PFL_ERR_ARG, "batch is NULL");
  DeviceScope on_device;
  BTRY(on_device.enter(b->device));
  double* part = (double*)(b->ws + b->red_off);
  double* res = part + DIAG_BLOCKS * 9;
  double* upart = part + DIAG_BLOCKS * 9 + 16;
  double* ures = part + DIAG_BLOCKS * 10 + 16;
  int bad = 0;
  bool table_dirty = false;
  for (int i = 0; i < b->count; ++i) {
    BInst& I = b->inst[i];
    Geo geo;
    geo.nx = (int)I.geo.nx;
    geo.ny = (int)I.geo.ny;
    geo.nz = (int)I.geo.nz;
    for (int a = 0; a < 3; ++a) geo.wall[a] = I.geo.wall[a];
    geo.N = I.geo.N;
    const int ab = I.active ? b->ab : I.frozen_ab;
    phi_one(b, i, ab);
    if (b->prec == PFL_FP64) {
      k_diag<double><<<DIAG_BLOCKS, DIAG_THREADS, 0, b->stream>>>(geo, (const double*)I.phic, part);
      k_umax<0, 15, 0><<<DIAG_BLOCKS, DIAG_THREADS, 0, b->stream>>>(geo, I.ph, (const Store<0>::S*)I.g[ab],
                                                                    (const Store<0>::PhiT*)I.phic, upart);
    } else {
      k_diag<float><<<DIAG_BLOCKS, DIAG_THREADS, 0, b->stream>>>(geo, (const float*)I.phic, part);
      k_umax<1, 15, 0><<<DIAG_BLOCKS, DIAG_THREADS, 0, b->stream>>>(geo, I.ph, (const Store<1>::S*)I.g[ab],
                                                                    (const Store<1>::PhiT*)I.phic, upart);
    }
    k_diag_final<<<9, 32, 0, b->stream>>>(part, DIAG_BLOCKS, res);
    k_max_final<<<1, 32, 0, b->stream>>>(upart, DIAG_BLOCKS, ures);
    BTRY(cudaGetLastError());
    double h[9], umax = 0.0;
    BTRY(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    BTRY(cudaMemcpyAsync(&umax, ures, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BTRY(cudaStreamSynchronize(b->stream));
    if (out)
      for (int k = 0; k < 8; ++k) out[8 * i + k] = h[k];
    const long long nf = (long long)h[8];
    if (nonfinite) nonfinite[i] = nf;
    if (nf > 0 || !(umax <= PFL_SPEED_LIMIT)) {
      ++bad;
      if (I.active) {  // an unstable instance stops; the others go on
        I.active = 0;
        I.frozen_ab = b->ab;
        table_dirty = true;
      }
    }
  }
  if (table_dirty) {
    BTRY(cudaMemcpyAsync(b->d_inst, b->inst.data(), b->count * sizeof(BInst), cudaMemcpyHostToDevice, b->stream));
    BTRY(cudaStreamSynchronize(b->stream));
  }
  if (bad)
    return bfail(PFL_ERR_UNSTABLE, std::to_string(bad) +
                                       " instances hold non-finite phi or a flow speed above the limit and were stopped");
  return PFL_OK;
}

pfl_status pfl_batch_set_shape(pfl_batch* b, int cls, int tile_x, int tile_y, int z_chunk, int grid) {
  if (!b) return bfail(PFL_ERR_ARG, "batch is NULL");
  if (cls < 0 || cls >= NCLASS) return bfail(PFL_ERR_ARG, "class must be 0 (one z plane) or 1 (3-D)");
  if (z_chunk < 0 || grid < 0) return bfail(PFL_ERR_ARG, "z_chunk and grid must be >= 0");
  Shape sh{tile_x, tile_y, cls == 1 ? z_chunk : 0, 0};
  const int j = shape_index(cls, sh);
  if (j < 0 || j >= shapes_for(b->prec))
    return bfail(PFL_ERR_ARG, "tile " + std::to_string(tile_x) + " x " + std::to_string(tile_y) +
                                  " is not a shape of this class and precision");
  DeviceScope on_device;
  BTRY(on_device.enter(b->device));
  BTRY(cudaStreamSynchronize(b->stream));
  ClassPlan& c = b->cls[cls];
  if (!c.tiles) return PFL_OK;  // no instance of this class
  pfl_status s = build_tiles(b, c, sh, c.tiles);
  if (s != PFL_OK) return s;
  sh.grid = grid > 0 ? grid : b->sms * resident_blocks(b->prec, cls, sh);
  sh.grid = std::max(1, std::min(c.ntiles, sh.grid));
  c.shape = sh;
  // the graph holds the old launches; capture it again from pair 0
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  const int ab = b->ab;
  b->ab = 0;
  s = capture_graph(b);
  b->ab = ab;
  return s;
}

pfl_status pfl_batch_shapes(const pfl_batch* b, int* threads, int* grid, int* ntiles) {
  if (!b) return bfail(PFL_ERR_ARG, "batch is NULL");
  for (int k = 0; k < NCLASS; ++k) {
    if (threads) threads[k] = b->cls[k].shape.tx * b->cls[k].shape.ty;
    if (grid) grid[k] = b->cls[k].shape.grid;
    if (ntiles) ntiles[k] = b->cls[k].ntiles;
  }
  return PFL_OK;
}

long long pfl_batch_time(const pfl_batch* b) { return b ? b->t : -1; }

void pfl_batch_destroy(pfl_batch* b) {
  if (!b) return;
  DeviceScope on_device;  // the stream (NULL: the legacy stream) is the batch's device's
  on_device.enter(b->device);
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  delete b;
}

}  // extern "C"
