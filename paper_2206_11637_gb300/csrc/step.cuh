// Fused stream-collide kernel of the MRT path, written around opposite-velocity
// pairs.
//
// The collisions reduce to moments (see kernels.cuh): with degree-2 moments
// relaxed at omega and all higher ones at 1 (g), or degrees 1 and 2 at
// omega_phi and higher at 1 (h), every post-collision population is a
// quadratic polynomial of its velocity,
//   f+_i / w_i = alpha + beta . c_i + c_i . Gamma . c_i,
// so a pair (c, -c) shares E = alpha + c.Gamma.c and differs only in the sign
// of L = beta . c.  Moments are gathered the same way: S = f_c + f_-c feeds the
// even moments (p*, phi, second moments), D = f_c - f_-c the odd ones.
//   g:  alpha = p* - 3/2 u.u - a2 tr(Pi^d)/3,  beta = 3 u + 3/2 F / rho,
//       Gamma = 9/2 u u^T + a2 Pi^d,           a2 = 9/2 (1 - omega)
//   h:  alpha = phi - a2 tr(Pi^dh)/3,           beta = 3 phi u + a1 J^d + (1 - omega_phi/2) theta n,
//       Gamma = a2 Pi^dh,                       a1 = 3 (1 - omega_phi), a2 = 9/2 (1 - omega_phi)
// For the shifted FP16 format the coefficients are pre-scaled by the format's
// power-of-two factor and alpha_h carries the shift, so a stored value is
// E +- L without a per-population multiply by 1 / w.
//
// Neighbour addressing: per cell, the cell-index offsets of the -1 / +1
// neighbours along each axis (periodic wrap folded in) and whether the link
// crosses a no-slip face; offsets of a direction are sums of these, fixed at
// compile time inside the unrolled loops.
#pragma once
#include <type_traits>

#include "kernels.cuh"

#ifndef PFL_STEP_THREADS
#define PFL_STEP_THREADS 128
#endif
#ifndef PFL_STEP_MINB
#define PFL_STEP_MINB 4
#endif
// Resident blocks per SM the fused step is compiled for.  Three (80 registers,
// a few bytes of spill) beat two (128 registers) by 13-20 % for FP16S: the
// kernel is latency-bound and gains from the extra warps.  FP64, bound by the
// FP64 units, keeps two (three would spill ~200 bytes per thread).
#ifndef PFL_ZM_MINB
#define PFL_ZM_MINB 3
#endif
#ifndef PFL_ZM_MINB_FP64
#define PFL_ZM_MINB_FP64 2
#endif
// L1 prefetch of the g populations of the plane the fused FP32 step collides
// next, issued one plane ahead right after the plane barrier (1; 0 = none).
// Measured on the 128x384x128 bubble: FP32 14.0 -> 14.9 GLUPS.  FP16S (issue
// bound) lost 5 %, single-plane lattices 8-10 % and the D3Q27 phase field 1 %
// (10.94 -> 10.82), so they take none.
#ifndef PFL_ZM_PREFETCH
#define PFL_ZM_PREFETCH 1
#endif
// Programmatic dependent launch of the fused step (1; 0 = plain launches):
// the host launches each step with programmatic stream serialisation, so the
// next step's blocks are scheduled while the last blocks of the previous one
// finish; every block waits (griddepcontrol.wait, a no-op without the launch
// attribute) for the previous grid's completion before its first global access.
// 200x400 wave: FP16S 11.3 -> 12.0 GLUPS, FP32 11.6 -> 12.3; the 3-D bubble is
// unchanged.  Releasing the dependents early (launch_dependents right after
// the wait) lost 6-13 %: waiting blocks then hold the SMs' block slots.
#ifndef PFL_ZM_PDL
#define PFL_ZM_PDL 1
#endif
// Interior form of the fused step (1; 0 = the general form everywhere): blocks
// clear of the lattice's faces by two cells take neighbour offsets without
// wall, wrap or solid tests.  Measured on the 512x384x512 impact (events, 128
// steps): FP16S 13.5 GLUPS with it against 16.1 without, FP32 14.5 against
// 14.8 -- the second copy of the unrolled body costs more than the tests it
// saves -- so it is off.
#ifndef PFL_ZM_INTERIOR
#define PFL_ZM_INTERIOR 0
#endif

namespace pfl {

// Exact q = n / d for 32-bit unsigned n and a divisor fixed for the launch
// (division by an invariant integer using multiplication, Granlund and
// Montgomery 1994, round-up multiplier form): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n), q = (t + ((n - t) >> s1)) >> s2,
// s1 = min(l, 1), s2 = max(l - 1, 0).
struct FastDiv {
  unsigned d, m;
  int s1, s2;
};

inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  f.d = d;
  int l = 0;
  while ((1ull << l) < d) ++l;
  f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l - 1 > 0 ? l - 1 : 0;
  return f;
}

__host__ __device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  const unsigned t = __umulhi(n, f.m);
#else
  const unsigned t = (unsigned)(((unsigned long long)n * f.m) >> 32);
#endif
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

// Host check of the divider on the boundary cases and a spread of numerators.
inline bool fastdiv_ok(unsigned d, unsigned nmax) {
  const FastDiv f = make_fastdiv(d);
  const unsigned probe[] = {0u, 1u, d - 1, d, d + 1, 2 * d - 1, 2 * d, nmax - 1, nmax};
  for (unsigned n : probe)
    if (n <= nmax && fdiv(n, f) != n / d) return false;
  unsigned long long x = 0x9e3779b97f4a7c15ull;
  for (int k = 0; k < 4096; ++k) {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    const unsigned n = (unsigned)(x % ((unsigned long long)nmax + 1));
    if (fdiv(n, f) != n / d) return false;
  }
  return true;
}

// Launch geometry of the 32-bit-indexed kernels (27 N < 2^32).
struct Geo32 {
  unsigned nx, ny, nz, N;
  FastDiv dx, dy;   // division by nx and by ny
  int wall[3];
};

struct AxisOff {
  int om, op;    // population neighbour offsets of x-1, x+1
  bool vm, vp;   // the link to x-1 / x+1 stays inside (false behind a wall)
  int sm, sp;    // phi-stencil offsets (mirror at walls)
};

__device__ __forceinline__ AxisOff axis_off(unsigned x, unsigned n, int stride, int wall) {
  AxisOff a;
  if (wall) {
    a.vm = x > 0;
    a.vp = x + 1 < n;
    a.om = -stride;
    a.op = stride;
    a.sm = a.vm ? a.om : 0;
    a.sp = a.vp ? a.op : 0;
  } else {
    a.vm = a.vp = true;
    a.om = x > 0 ? -stride : (int)(n - 1) * stride;
    a.op = x + 1 < n ? stride : -(int)(n - 1) * stride;
    a.sm = a.om;
    a.sp = a.op;
  }
  return a;
}


// Blocked links of a cell next to solid cells: bit (cx+1) + 3(cy+1) + 9(cz+1)
// is set when the neighbour in direction c is solid; bit 13 (the rest
// direction) marks the cell itself solid.  Zero away from solids, and a
// compile-time zero in kernels built without solids.
__host__ __device__ constexpr unsigned link_bit(int cx, int cy, int cz) {
  return 1u << ((cx + 1) + 3 * (cy + 1) + 9 * (cz + 1));
}
constexpr unsigned SOLID_SELF = 1u << 13;

// seed of the FP16 stochastic rounding of step t (Fibonacci hashing of t)
__host__ __device__ __forceinline__ unsigned step_seed_of(unsigned long long t) {
  return (unsigned)(t * 0x9E3779B97F4A7C15ull >> 32);
}

struct CellOff {
  AxisOff X, Y, Z;
  unsigned blk = 0;  // blocked links (solid neighbours)
  // population offset and validity of direction (cx, cy, cz): a link leaving
  // through a no-slip face or into a solid cell is bounced back half-way
  __device__ __forceinline__ int off(int cx, int cy, int cz) const {
    return (cx < 0 ? X.om : cx > 0 ? X.op : 0) + (cy < 0 ? Y.om : cy > 0 ? Y.op : 0) +
           (cz < 0 ? Z.om : cz > 0 ? Z.op : 0);
  }
  __device__ __forceinline__ bool valid(int cx, int cy, int cz) const {
    return (cx < 0 ? X.vm : cx > 0 ? X.vp : true) && (cy < 0 ? Y.vm : cy > 0 ? Y.vp : true) &&
           (cz < 0 ? Z.vm : cz > 0 ? Z.vp : true) && !(blk & link_bit(cx, cy, cz));
  }
  __device__ __forceinline__ int soff(int cx, int cy, int cz) const {
    return (cx < 0 ? X.sm : cx > 0 ? X.sp : 0) + (cy < 0 ? Y.sm : cy > 0 ? Y.sp : 0) +
           (cz < 0 ? Z.sm : cz > 0 ? Z.sp : 0);
  }
};

// Offsets of a cell whose neighbours two cells deep all lie inside the lattice
// (no face, no wrap, no solid): every link is valid and the offset of
// direction c is cx + cy sy + cz sz.  The fused step takes this form for blocks
// whose tile, ring and z range stay clear of the lattice's faces.
struct CellOffI {
  int sy, sz;
  static constexpr unsigned blk = 0;
  __device__ __forceinline__ int off(int cx, int cy, int cz) const { return cx + cy * sy + cz * sz; }
  __device__ __forceinline__ constexpr bool valid(int, int, int) const { return true; }
  __device__ __forceinline__ int soff(int cx, int cy, int cz) const { return off(cx, cy, cz); }
};

// Raw stored value as the arithmetic type (FP16: the stored number, unscaled).
template <int PREC>
__device__ __forceinline__ typename Store<PREC>::R raw(typename Store<PREC>::S v) {
  if constexpr (PREC == 2)
    return __half2float(v);
  else
    return v;
}
template <int PREC>
__device__ __forceinline__ typename Store<PREC>::S pack(typename Store<PREC>::R v) {
  if constexpr (PREC == 2)
    return __float2half_rn(v);
  else
    return v;
}

// Stochastic rounding for the FP16 stores of the step.  Round-to-nearest
// repeats the same error every step where a field changes slowly, and those
// errors add up linearly in time (mass drift of phi); rounding up with the
// probability given by the discarded bits makes every store unbiased.  The
// random bits come from a per-cell stream: the 32-bit hash of (cell, step)
// (lowbias32 by C. Wellons) seeds a linear congruential sequence (Numerical
// Recipes constants), whose top 13 bits are added below the FP16 mantissa of
// the FP32 value before truncation toward zero.
__device__ __forceinline__ unsigned hash32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

struct Dither {
  unsigned r;
  __device__ __forceinline__ unsigned next() {
    r = r * 1664525u + 1013904223u;
    return r >> 19;
  }
  // 32 bits for a pair: the state's high half, and the low half xor-ed with
  // the high one (the low bits of a power-of-two LCG have short periods)
  __device__ __forceinline__ unsigned next32() {
    r = r * 1664525u + 1013904223u;
    return r ^ (r >> 16);
  }
};

// Stochastic rounding of a pair in one conversion (sm_100-family
// cvt.rs.f16x2.f32): A lands in the high half and is rounded with the high 16
// random bits, B in the low half with the low 16; each rounds away from zero
// with the probability of its discarded fraction (an unbiased rounding, like
// pack_sr).  PFL_FP16S_HWSR = 0 keeps pack_sr for every store.
#ifndef PFL_FP16S_HWSR
#define PFL_FP16S_HWSR 1
#endif
__device__ __forceinline__ void pack2_sr(float A, float B, unsigned bits, __half& a, __half& b) {
  unsigned d;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(A), "f"(B), "r"(bits));
  a = __ushort_as_half((unsigned short)(d >> 16));
  b = __ushort_as_half((unsigned short)(d & 0xffffu));
}

template <int PREC>
__device__ __forceinline__ typename Store<PREC>::S pack_sr(typename Store<PREC>::R v, Dither& d) {
  if constexpr (PREC == 2) {
    const unsigned b = __float_as_uint(v) + d.next();
    return __float2half_rz(__uint_as_float(b));
  } else {
    return v;
  }
}

// w (s + r) for a lattice weight w, s the large part of a stored population
// (phi or p*) and r the small rest.  FP32 carries w as hi + lo: the FP32
// roundings of the D3Q15 weights alone sum to 1 + 7.5e-9 (D3Q27 likewise),
// a bias of the zeroth and second moments that repeats every step and, over
// 1000 steps, was the largest FP32 error of phi and u.  FP64 uses w as is.
template <typename R>
__device__ __forceinline__ R wsum(double w, R s, R r) {
  if constexpr (sizeof(R) == 4) {
    const float hi = (float)w, lo = (float)(w - (double)hi);
    return fmaf(hi, s, fmaf(lo, s, hi * r));
  } else {
    return fma(w, s, w * r);
  }
}

__device__ __forceinline__ void cell_off(const Geo32& geo, unsigned c, CellOff& o) {
  const unsigned yz = fdiv(c, geo.dx);
  const unsigned x = c - yz * geo.nx;
  const unsigned z = fdiv(yz, geo.dy);
  const unsigned y = yz - z * geo.ny;
  o.X = axis_off(x, geo.nx, 1, geo.wall[0]);
  o.Y = axis_off(y, geo.ny, (int)geo.nx, geo.wall[1]);
  o.Z = axis_off(z, geo.nz, (int)(geo.nx * geo.ny), geo.wall[2]);
}

// Load the pair (i: direction c, oi: direction -c) arriving at `cell`.
// a, b: raw stored values; fa, fb: the cells that wrote them.  Indices are
// 32-bit (unsigned wrap-around arithmetic; the final index is in range).
template <int PREC, int READ_ODD, class Off>
__device__ __forceinline__ void load_pair(const typename Store<PREC>::S* __restrict__ f, unsigned N, unsigned cell,
                                          const Off& o, int i, int oi, int cx, int cy, int cz,
                                          typename Store<PREC>::R& a, typename Store<PREC>::R& b, unsigned& fa,
                                          unsigned& fb) {
  const bool vmc = o.valid(-cx, -cy, -cz), vc = o.valid(cx, cy, cz);
  const unsigned nm = cell + (unsigned)o.off(-cx, -cy, -cz), np = cell + (unsigned)o.off(cx, cy, cz);
  fa = vmc ? nm : cell;
  fb = vc ? np : cell;
  if (!READ_ODD) {
    a = raw<PREC>(f[(unsigned)i * N + cell]);
    b = raw<PREC>(f[(unsigned)oi * N + cell]);
  } else {
    a = raw<PREC>(f[vmc ? (unsigned)oi * N + nm : (unsigned)i * N + cell]);
    b = raw<PREC>(f[vc ? (unsigned)i * N + np : (unsigned)oi * N + cell]);
  }
}

// Store the post-collision pair (A: direction c, B: direction -c) of `cell`.
template <int PREC, int ODD, class Off>
__device__ __forceinline__ void store_pair(typename Store<PREC>::S* __restrict__ f, unsigned N, unsigned cell,
                                           const Off& o, int i, int oi, int cx, int cy, int cz,
                                           typename Store<PREC>::R A, typename Store<PREC>::R B, Dither& d) {
  typename Store<PREC>::S a, b;
  if constexpr (PREC == 2 && PFL_FP16S_HWSR) {
    pack2_sr(A, B, d.next32(), a, b);
  } else {
    a = pack_sr<PREC>(A, d);
    b = pack_sr<PREC>(B, d);
  }
  if (!ODD) {
    f[(unsigned)oi * N + cell] = a;
    f[(unsigned)i * N + cell] = b;
  } else {
    const bool vc = o.valid(cx, cy, cz), vmc = o.valid(-cx, -cy, -cz);
    f[vc ? (unsigned)i * N + cell + (unsigned)o.off(cx, cy, cz) : (unsigned)oi * N + cell] = a;
    f[vmc ? (unsigned)oi * N + cell + (unsigned)o.off(-cx, -cy, -cz) : (unsigned)i * N + cell] = b;
  }
}

// phi^t around a cell read from the current phi buffer (stencil offsets, so
// mirrored across walls).
template <int PREC>
struct GlobalPhi {
  const typename Store<PREC>::PhiT* __restrict__ phi;
  const CellOff* o;
  unsigned cell;
  __device__ __forceinline__ typename Store<PREC>::R operator()(int cx, int cy, int cz) const {
    return (typename Store<PREC>::R)__ldg(phi + cell + o->soff(cx, cy, cz));
  }
};

// p* shift of the cell that wrote a g population (FP16S): the population
// arriving from offset (dx, dy, dz) -- the opposite of its velocity -- was
// written by `writer` (the neighbour, or the cell itself after a bounce-back,
// valid = false).  GlobalShift reads the writer's shift from the per-cell
// array; the fused step reads it from a shared-memory ring (SmemShift).
struct GlobalShift {
  const __half* __restrict__ p;
  __device__ __forceinline__ float operator()(unsigned writer, int dx, int dy, int dz, bool valid) const {
    return __half2float(__ldg(p + writer));
  }
};
struct NoShift {
  __device__ __forceinline__ float operator()(unsigned, int, int, int, bool) const { return 0.0f; }
};

// The collide-stream update of one cell, shared by every stream-collide
// kernel: populations are read from (hin, gin) in the layout READ_ODD and
// written to (hout, gout) in the layout WRITE_ODD (the same arrays and parity
// for the in-place AA step; a second array pair and push streaming for the
// two-array step).  phi_at(c) returns phi^t at the stencil neighbour c.
template <int PREC, int QH, int READ_ODD, int WRITE_ODD, class PhiAt, int HM = 0, class PShift = NoShift,
          class Off = CellOff>
__device__ __forceinline__ void collide_cell(const Geo32& geo, const Phys& ph, const Off& o,
                                             const typename Store<PREC>::S* hin,
                                             const typename Store<PREC>::S* gin, typename Store<PREC>::S* hout,
                                             typename Store<PREC>::S* gout, const PhiAt& phi_at,
                                             const typename Store<PREC>::PhiT* __restrict__ shift,
                                             unsigned cell, unsigned seed,
                                             const typename Store<PREC>::R* hmom = nullptr, int hstride = 0,
                                             const PShift& pshift = PShift(), __half* __restrict__ pg_out = nullptr) {
  typedef typename Store<PREC>::R R;
  constexpr bool F16 = PREC == 2;
  constexpr int QG = qg_of<QH>();  // D2Q9 with the 2-D phase field, else D3Q27
  constexpr int GR = (QG - 1) / 2;  // rest index of g
  const unsigned N = geo.N;
  Dither dith{F16 ? hash32(cell * 0x9E3779B1u + seed) : 0u};

  // ---- phi stencil over D3Q27 weights, by pairs
  const R pc = phi_at(0, 0, 0);
  R gx = 0, gy = 0, gz = 0, lap = 0;
#pragma unroll
  for (int i = 0; i < GR; ++i) {
    const int cx = q27_cx(lq_to27<QG>(i)), cy = q27_cy(lq_to27<QG>(i)), cz = q27_cz(lq_to27<QG>(i));
    const R a = phi_at(cx, cy, cz);
    const R b = phi_at(-cx, -cy, -cz);
    const R w = (R)lq_w<QG>(i);
    const R d = w * (a - b);
    if (cx) gx += cx > 0 ? d : -d;
    if (cy) gy += cy > 0 ? d : -d;
    if (cz) gz += cz > 0 ? d : -d;
    lap += w * ((a - pc) + (b - pc));  // differences first: exact for nearby values
  }
  gx *= (R)3;
  gy *= (R)3;
  gz *= (R)3;
  lap *= (R)6;

  // ---- g moments (FP16: g_i = w_i (s / KG + P_writer))
  R pst, jx = 0, jy = 0, jz = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pyz = 0, pxz = 0;
  {
    const R rest = raw<PREC>(gin[(unsigned)GR * N + cell]);
    pst = F16 ? (rest * (R)(1.0 / KG16) + (R)pshift(cell, 0, 0, 0, false)) * (R)lq_w<QG>(GR) : rest;
  }
#pragma unroll
  for (int i = 0; i < GR; ++i) {
    const int cx = q27_cx(lq_to27<QG>(i)), cy = q27_cy(lq_to27<QG>(i)), cz = q27_cz(lq_to27<QG>(i));
    R a, b;
    unsigned fa, fb;
    load_pair<PREC, READ_ODD>(gin, N, cell, o, i, QG - 1 - i, cx, cy, cz, a, b, fa, fb);
    R S = a + b, D = a - b;
    if (F16) {
      // a arrives from x - c, b from x + c
      const R pa = (R)pshift(fa, -cx, -cy, -cz, o.valid(-cx, -cy, -cz));
      const R pb = (R)pshift(fb, cx, cy, cz, o.valid(cx, cy, cz));
      const R w = (R)lq_w<QG>(i);
      S = w * (S * (R)(1.0 / KG16) + (pa + pb));
      D = w * (D * (R)(1.0 / KG16) + (pa - pb));
    }
    pst += S;
    if (cx) jx += cx > 0 ? D : -D;
    if (cy) jy += cy > 0 ? D : -D;
    if (cz) jz += cz > 0 ? D : -D;
    if (cx) pxx += S;
    if (cy) pyy += S;
    if (cz) pzz += S;
    if (cx && cy) pxy += (cx * cy > 0) ? S : -S;
    if (cy && cz) pyz += (cy * cz > 0) ? S : -S;
    if (cx && cz) pxz += (cx * cz > 0) ? S : -S;
  }

  // ---- forces and velocity (same expressions as hydro_macro)
  const R drho = (R)(ph.rho_h - ph.rho_l);
  const R rho = (R)ph.rho_l + pc * drho;
  const R tau = (R)ph.tau_l + pc * (R)(ph.tau_h - ph.tau_l);
  const R omega = (R)1 / tau;
  const R nu = (tau - (R)0.5) * (R)(1.0 / 3.0);
  const R mu = (R)4 * (R)ph.beta * pc * (pc - (R)1) * (pc - (R)0.5) - (R)ph.kappa * lap;
  const R inv2rho = (R)0.5 / rho;
  const R cp = -pst * (R)(1.0 / 3.0) * drho;
  R Fx = (mu + cp) * gx + rho * (R)ph.gx;
  R Fy = (mu + cp) * gy + rho * (R)ph.gy;
  R Fz = (mu + cp) * gz + rho * (R)ph.gz;
  const R p3 = pst * (R)(1.0 / 3.0);
  {
    const R u0x = jx + Fx * inv2rho, u0y = jy + Fy * inv2rho, u0z = jz + Fz * inv2rho;
    const R nxx = pxx - p3 - u0x * u0x, nyy = pyy - p3 - u0y * u0y, nzz = pzz - p3 - u0z * u0z;
    const R nxy = pxy - u0x * u0y, nyz = pyz - u0y * u0z, nxz = pxz - u0x * u0z;
    const R cm = (R)-3 * nu * omega * drho;
    Fx += cm * (nxx * gx + nxy * gy + nxz * gz);
    Fy += cm * (nxy * gx + nyy * gy + nyz * gz);
    Fz += cm * (nxz * gx + nyz * gy + nzz * gz);
  }
  const R ux = jx + Fx * inv2rho, uy = jy + Fy * inv2rho, uz = jz + Fz * inv2rho;
  // FP16S: every g this cell writes is stored against P = fp16(p*) of the cell
  R pw = 0;
  if constexpr (F16) {
    const __half q = __float2half_rn(pst);
    pg_out[cell] = q;
    pw = __half2float(q);
  }

  // ---- g post-collision coefficients and pair stores
  {
    const R uu = ux * ux + uy * uy + uz * uz;
    const R a2 = ((R)1 - omega) * (R)4.5;
    // deviatoric second moments.  FP32 / FP64 form (3 P_aa - p*) / 3 with one
    // rounding: p* (1/3) would carry the rounded constant 1/3, a bias of
    // 3e-8 p* that repeats every step (FP16S keeps its form)
    const R third = (R)(1.0 / 3.0);
    const R dxx = F16 ? pxx - p3 - ux * ux : fma((R)3, pxx, -pst) * third - ux * ux;
    const R dyy = F16 ? pyy - p3 - uy * uy : fma((R)3, pyy, -pst) * third - uy * uy;
    const R dzz = QG == 9 ? (R)0 : (F16 ? pzz - p3 - uz * uz : fma((R)3, pzz, -pst) * third - uz * uz);  // 2-D: the trace runs over x and y
    const R K = F16 ? (R)KG16 : (R)1;
    // alpha = p* + als with als small: FP32 and FP64 round p* once per stored
    // value (FP16S stores K (alpha - P) + ... directly)
    const R als = -(R)1.5 * uu - a2 * (dxx + dyy + dzz) * (R)(1.0 / 3.0);
    const R al = K * (pst - pw - (R)1.5 * uu - a2 * (dxx + dyy + dzz) * (R)(1.0 / 3.0));
    const R fr = (R)1.5 / rho;
    const R bx = K * ((R)3 * ux + fr * Fx), by = K * ((R)3 * uy + fr * Fy), bz = K * ((R)3 * uz + fr * Fz);
    const R Gxx = K * ((R)4.5 * ux * ux + a2 * dxx), Gyy = K * ((R)4.5 * uy * uy + a2 * dyy),
            Gzz = K * ((R)4.5 * uz * uz + a2 * dzz);
    const R Gxy = K * (R)2 * ((R)4.5 * ux * uy + a2 * (pxy - ux * uy));
    const R Gyz = K * (R)2 * ((R)4.5 * uy * uz + a2 * (pyz - uy * uz));
    const R Gxz = K * (R)2 * ((R)4.5 * ux * uz + a2 * (pxz - ux * uz));
    gout[(unsigned)GR * N + cell] =
        pack_sr<PREC>(F16 ? al : wsum<R>(lq_w<QG>(GR), pst, als), dith);
#pragma unroll
    for (int i = 0; i < GR; ++i) {
      const int cx = q27_cx(lq_to27<QG>(i)), cy = q27_cy(lq_to27<QG>(i)), cz = q27_cz(lq_to27<QG>(i));
      // FP32 / FP64: the small terms first, the equilibrium part once (one
      // rounding at its size); FP16S as E = al + ..., A = E + L
      R E = F16 ? al : (R)0;
      if (cx) E += Gxx;
      if (cy) E += Gyy;
      if (cz) E += Gzz;
      if (cx && cy) E += (cx * cy > 0) ? Gxy : -Gxy;
      if (cy && cz) E += (cy * cz > 0) ? Gyz : -Gyz;
      if (cx && cz) E += (cx * cz > 0) ? Gxz : -Gxz;
      R L = 0;
      if (cx) L += cx > 0 ? bx : -bx;
      if (cy) L += cy > 0 ? by : -by;
      if (cz) L += cz > 0 ? bz : -bz;
      R A, B;
      if (F16) {
        A = E + L;
        B = E - L;
      } else {
        A = wsum<R>(lq_w<QG>(i), pst, als + (E + L));
        B = wsum<R>(lq_w<QG>(i), pst, als + (E - L));
      }
      store_pair<PREC, WRITE_ODD>(gout, N, cell, o, i, QG - 1 - i, cx, cy, cz, A, B, dith);
    }
  }

  // ---- h moments (shifted FP16: h = w (s / KH + phi_writer)), or given by the caller
  R phl, hjx = 0, hjy = 0, hjz = 0, hxx = 0, hyy = 0, hzz = 0, hxy = 0, hyz = 0, hxz = 0;
  if (HM) {
    phl = hmom[0];
    hjx = hmom[hstride];
    hjy = hmom[2 * hstride];
    hjz = hmom[3 * hstride];
    hxx = hmom[4 * hstride];
    hyy = hmom[5 * hstride];
    hzz = hmom[6 * hstride];
    hxy = hmom[7 * hstride];
    hyz = hmom[8 * hstride];
    hxz = hmom[9 * hstride];
  } else {
    const R rest = raw<PREC>(hin[(unsigned)hq_rest<QH>() * N + cell]);
    phl = F16 ? (rest * (R)(1.0 / KH16) + (R)__ldg(shift + cell)) * (R)hq_w<QH>(hq_rest<QH>()) : rest;
  }
#pragma unroll
  for (int k = 0; k < (HM ? 0 : hq_rest<QH>()); ++k) {
    const int cx = hq_cx<QH>(k), cy = hq_cy<QH>(k), cz = hq_cz<QH>(k);
    R a, b;
    unsigned fa, fb;
    load_pair<PREC, READ_ODD>(hin, N, cell, o, k, QH - 1 - k, cx, cy, cz, a, b, fa, fb);
    R S, D;
    if (F16) {
      const R sa = (R)__ldg(shift + fa), sb = (R)__ldg(shift + fb);
      const R w = (R)hq_w<QH>(k);
      S = w * ((a + b) * (R)(1.0 / KH16) + (sa + sb));
      D = w * ((a - b) * (R)(1.0 / KH16) + (sa - sb));
    } else {
      S = a + b;
      D = a - b;
    }
    phl += S;
    if (cx) hjx += cx > 0 ? D : -D;
    if (cy) hjy += cy > 0 ? D : -D;
    if (cz) hjz += cz > 0 ? D : -D;
    if (cx) hxx += S;
    if (cy) hyy += S;
    if (cz) hzz += S;
    if (cx && cy) hxy += (cx * cy > 0) ? S : -S;
    if (cy && cz) hyz += (cy * cz > 0) ? S : -S;
    if (cx && cz) hxz += (cx * cz > 0) ? S : -S;
  }

  // ---- h post-collision coefficients and pair stores
  {
    const R omp = (R)ph.omega_phi;
    const R gn = sqrt(gx * gx + gy * gy + gz * gz);
    const R theta = (R)4 * pc * ((R)1 - pc) * (R)ph.inv_xi;
    const R tn = theta / (gn + (R)1e-6) * ((R)1 - (R)0.5 * omp);  // (1 - omega_phi/2) theta / |grad phi|
    const R a1 = ((R)1 - omp) * (R)3, a2 = ((R)1 - omp) * (R)4.5;
    // deviatoric second moments and the non-equilibrium flux.  FP32 / FP64
    // form (3 H_aa - phi) / 3 and J - phi u with one rounding each: phi (1/3)
    // would carry the rounded constant 1/3, a bias of 3e-8 phi that repeats
    // every step (FP16S keeps its form)
    const R ph3 = phl * (R)(1.0 / 3.0);
    const R third = (R)(1.0 / 3.0);
    const R dxx = F16 ? hxx - ph3 : fma((R)3, hxx, -phl) * third;
    const R dyy = F16 ? hyy - ph3 : fma((R)3, hyy, -phl) * third;
    const R dzz = QG == 9 ? (R)0 : (F16 ? hzz - ph3 : fma((R)3, hzz, -phl) * third);
    const R K = F16 ? (R)KH16 : (R)1;
    const R sh = F16 ? pc : (R)0;   // this cell's phi: the shift of everything it writes
    // alpha = phi + als with als small: FP32 and FP64 round phi once per stored
    // value (FP16S stores K (alpha - phi_x) + ... directly)
    const R als = -a2 * (dxx + dyy + dzz) * (R)(1.0 / 3.0);
    const R al = K * ((phl - sh) - a2 * (dxx + dyy + dzz) * (R)(1.0 / 3.0));
    const R jdx = F16 ? hjx - phl * ux : fma(-phl, ux, hjx);
    const R jdy = F16 ? hjy - phl * uy : fma(-phl, uy, hjy);
    const R jdz = F16 ? hjz - phl * uz : fma(-phl, uz, hjz);
    const R bx = K * ((R)3 * phl * ux + a1 * jdx + tn * gx);
    const R by = K * ((R)3 * phl * uy + a1 * jdy + tn * gy);
    const R bz = K * ((R)3 * phl * uz + a1 * jdz + tn * gz);
    const R Gxx = K * a2 * dxx, Gyy = K * a2 * dyy, Gzz = K * a2 * dzz;
    const R Gxy = K * (R)2 * a2 * hxy, Gyz = K * (R)2 * a2 * hyz, Gxz = K * (R)2 * a2 * hxz;
    hout[(unsigned)hq_rest<QH>() * N + cell] =
        pack_sr<PREC>(F16 ? al : wsum<R>(hq_w<QH>(hq_rest<QH>()), phl, als), dith);
#pragma unroll
    for (int k = 0; k < hq_rest<QH>(); ++k) {
      const int cx = hq_cx<QH>(k), cy = hq_cy<QH>(k), cz = hq_cz<QH>(k);
      R E = F16 ? al : (R)0;
      if (cx) E += Gxx;
      if (cy) E += Gyy;
      if (cz) E += Gzz;
      if (cx && cy) E += (cx * cy > 0) ? Gxy : -Gxy;
      if (cy && cz) E += (cy * cz > 0) ? Gyz : -Gyz;
      if (cx && cz) E += (cx * cz > 0) ? Gxz : -Gxz;
      R L = 0;
      if (cx) L += cx > 0 ? bx : -bx;
      if (cy) L += cy > 0 ? by : -by;
      if (cz) L += cz > 0 ? bz : -bz;
      R A, B;
      if (F16) {
        A = E + L;
        B = E - L;
      } else {
        A = wsum<R>(hq_w<QH>(k), phl, als + (E + L));
        B = wsum<R>(hq_w<QH>(k), phl, als + (E - L));
      }
      store_pair<PREC, WRITE_ODD>(hout, N, cell, o, k, QH - 1 - k, cx, cy, cz, A, B, dith);
    }
  }
}

// In-place AA update of one cell with the stencil read from the phi buffer.
// pg_in / pg_out: the p* shifts of the stored g (FP16S; NULL otherwise),
// read for the populations loaded and written for those stored.
template <int PREC, int QH, int ODD>
__device__ __forceinline__ void step_cell(const Geo32& geo, const Phys& ph, typename Store<PREC>::S* __restrict__ h,
                                          typename Store<PREC>::S* __restrict__ g,
                                          const typename Store<PREC>::PhiT* __restrict__ phi,
                                          const typename Store<PREC>::PhiT* __restrict__ shift, unsigned cell,
                                          unsigned seed, const __half* __restrict__ pg_in = nullptr,
                                          __half* __restrict__ pg_out = nullptr) {
  CellOff o;
  cell_off(geo, cell, o);
  GlobalPhi<PREC> at{phi, &o, cell};
  collide_cell<PREC, QH, ODD, ODD, GlobalPhi<PREC>, 0, GlobalShift>(geo, ph, o, h, g, h, g, at, shift, cell, seed,
                                                                    nullptr, 0, GlobalShift{pg_in}, pg_out);
}

template <int PREC, int QH, int ODD>
__global__ void __launch_bounds__(PFL_STEP_THREADS, PFL_STEP_MINB)
    k_step_mrt(Geo32 geo, Phys ph, typename Store<PREC>::S* __restrict__ h, typename Store<PREC>::S* __restrict__ g,
               const typename Store<PREC>::PhiT* __restrict__ phi,
               const typename Store<PREC>::PhiT* __restrict__ shift, unsigned seed,
               const __half* __restrict__ pg_in = nullptr, __half* __restrict__ pg_out = nullptr) {
  const unsigned cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= geo.N) return;
  step_cell<PREC, QH, ODD>(geo, ph, h, g, phi, shift, cell, seed, pg_in, pg_out);
}

// phi of one cell from the stored h (READ_ODD after an even step).
template <int PREC, int QH, int READ_ODD>
__device__ __forceinline__ typename Store<PREC>::R phi_cell(const Geo32& geo,
                                                            const typename Store<PREC>::S* __restrict__ h,
                                                            const typename Store<PREC>::PhiT* __restrict__ shift,
                                                            unsigned cell, unsigned blk = 0) {
  typedef typename Store<PREC>::R R;
  constexpr bool F16 = PREC == 2;
  CellOff o;
  cell_off(geo, cell, o);
  o.blk = blk;  // a bounced population was written by this cell
  R s = F16 ? (raw<PREC>(h[(unsigned)hq_rest<QH>() * geo.N + cell]) * (R)(1.0 / KH16) + (R)__ldg(shift + cell)) * (R)hq_w<QH>(hq_rest<QH>())
            : raw<PREC>(h[(unsigned)hq_rest<QH>() * geo.N + cell]);
#pragma unroll
  for (int k = 0; k < hq_rest<QH>(); ++k) {
    R a, b;
    unsigned fa, fb;
    load_pair<PREC, READ_ODD>(h, geo.N, cell, o, k, QH - 1 - k, hq_cx<QH>(k), hq_cy<QH>(k), hq_cz<QH>(k), a, b, fa, fb);
    if (F16)
      s += (R)hq_w<QH>(k) * ((a + b) * (R)(1.0 / KH16) + ((R)__ldg(shift + fa) + (R)__ldg(shift + fb)));
    else
      s += a + b;
  }
  return s;
}

// phi = sum_i h_i of the state left by the last step (READ_ODD after an even
// step); `shift` holds the shifts of the stored populations (FP16S).  With
// `links` (a lattice with solid cells) blocked links bounce and solid cells
// hold phi = 0.
template <int PREC, int QH, int READ_ODD>
__global__ void __launch_bounds__(256) k_phi32(Geo32 geo, const typename Store<PREC>::S* __restrict__ h,
                                               const typename Store<PREC>::PhiT* __restrict__ shift,
                                               typename Store<PREC>::PhiT* __restrict__ phi,
                                               const unsigned* __restrict__ links = nullptr) {
  const unsigned cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= geo.N) return;
  const unsigned blk = links ? __ldg(links + cell) : 0u;
  phi[cell] = (blk & SOLID_SELF) ? (typename Store<PREC>::PhiT)0 : phi_cell<PREC, QH, READ_ODD>(geo, h, shift, cell, blk);
}

}  // namespace pfl

namespace pfl {

// ---------------------------------------------------------------------------
// Fused two-array step: stream-collide and the phi stencil in one launch.
//
// The populations live in two array pairs; a step reads the current pair in
// its own cell (every slot local, coalesced) and pushes the post-collision
// populations to the other pair (x + c, or the opposite slot of x behind a
// wall).  Nothing a step reads is overwritten during that step, so a block may
// read its neighbours' populations: each block owns an xy tile of ZM_TX x
// ZM_TY columns and marches through a chunk of z planes, computing phi^t =
// sum_i h_i for its tile plus a one-cell ring into a three-plane shared-memory
// ring before colliding a plane.  phi^t of every cell is written once (the
// FP16S shift of the populations written this step and the phi output), so
// the separate phi pass and its re-read of h disappear.  Ring and z-halo
// planes repeat the phi sum of neighbouring tiles (from L2).
// A single-plane lattice (FLAT) has no z march to hide latency behind; its
// tiles are 32 x 4, so that a small lattice spreads over more blocks (and the
// SMs' loads even out) for a slightly larger share of ring cells.
constexpr int ZM_TX = 32;
constexpr int ZM_TY = 8;
constexpr int ZM_TY_FLAT = 4;
__host__ __device__ constexpr int zm_ty(int flat) { return flat ? ZM_TY_FLAT : ZM_TY; }

// FLAT: a single plane, its own z neighbour (periodic) -- every cz reads the
// plane itself, so the compiler loads each in-plane value once.
template <int PREC, int FLAT = 0, int PW = ZM_TX + 2>
struct SmemPhi {
  const typename Store<PREC>::PhiT* plane[3];  // planes z - 1, z, z + 1 of (tile height + 2) x PW values
  int i0;                 // index of this thread's column in a plane
  unsigned blk = 0;       // blocked links: a solid neighbour reads as this cell (neutral wetting)
  __device__ __forceinline__ typename Store<PREC>::R operator()(int cx, int cy, int cz) const {
    if (blk & link_bit(cx, cy, cz)) return (typename Store<PREC>::R)plane[1][i0];
    return (typename Store<PREC>::R)plane[FLAT ? 1 : 1 + cz][i0 + cy * PW + cx];
  }
};

// p* shift of the writer of a g population from the ring of P planes z - 1,
// z, z + 1 of the fused step (tile plus a one-cell ring, like SmemPhi): the
// neighbour at (dx, dy, dz), or the cell itself after a bounce-back.
template <int FLAT = 0, int PW = ZM_TX + 2>
struct SmemShift {
  const float* plane[3];
  int i0;
  __device__ __forceinline__ float operator()(unsigned, int dx, int dy, int dz, bool valid) const {
    return valid ? plane[FLAT ? 1 : 1 + dz][i0 + dy * PW + dx] : plane[1][i0];
  }
};

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %0;\n\tprefetch.global.L1 [ga];\n\t}" ::"l"(p));
}

__device__ __forceinline__ int wrap_or_clamp(int v, int n, int wall) {
  if (wall) return v < 0 ? 0 : (v >= n ? n - 1 : v);
  return v < 0 ? v + n : (v >= n ? v - n : v);
}

// The 10 h moments (phi, sum c h, sum c c h) of `cell` of the current pair
// (normal layout, neighbour offsets o), accumulated by pairs in the same order
// as the collision does, so moms[0] equals its phi bitwise.
template <int PREC, int QH, class Off>
__device__ __forceinline__ void h_moments_at(const Geo32& geo, const typename Store<PREC>::S* __restrict__ h,
                                             const typename Store<PREC>::PhiT* __restrict__ shift, unsigned cell,
                                             const Off& o, typename Store<PREC>::R m[10]) {
  typedef typename Store<PREC>::R R;
  constexpr bool F16 = PREC == 2;
  const unsigned N = geo.N;
  R phl, hjx = 0, hjy = 0, hjz = 0, hxx = 0, hyy = 0, hzz = 0, hxy = 0, hyz = 0, hxz = 0;
  {
    const R rest = raw<PREC>(h[(unsigned)hq_rest<QH>() * N + cell]);
    phl = F16 ? (rest * (R)(1.0 / KH16) + (R)__ldg(shift + cell)) * (R)hq_w<QH>(hq_rest<QH>()) : rest;
  }
#pragma unroll
  for (int k = 0; k < hq_rest<QH>(); ++k) {
    const int cx = hq_cx<QH>(k), cy = hq_cy<QH>(k), cz = hq_cz<QH>(k);
    R a, b;
    unsigned fa, fb;
    load_pair<PREC, 0>(h, N, cell, o, k, QH - 1 - k, cx, cy, cz, a, b, fa, fb);
    R S, D;
    if (F16) {
      const R sa = (R)__ldg(shift + fa), sb = (R)__ldg(shift + fb);
      const R w = (R)hq_w<QH>(k);
      S = w * ((a + b) * (R)(1.0 / KH16) + (sa + sb));
      D = w * ((a - b) * (R)(1.0 / KH16) + (sa - sb));
    } else {
      S = a + b;
      D = a - b;
    }
    phl += S;
    if (cx) hjx += cx > 0 ? D : -D;
    if (cy) hjy += cy > 0 ? D : -D;
    if (cz) hjz += cz > 0 ? D : -D;
    if (cx) hxx += S;
    if (cy) hyy += S;
    if (cz) hzz += S;
    if (cx && cy) hxy += (cx * cy > 0) ? S : -S;
    if (cy && cz) hyz += (cy * cz > 0) ? S : -S;
    if (cx && cz) hxz += (cx * cz > 0) ? S : -S;
  }
  m[0] = phl;
  m[1] = hjx;
  m[2] = hjy;
  m[3] = hjz;
  m[4] = hxx;
  m[5] = hyy;
  m[6] = hzz;
  m[7] = hxy;
  m[8] = hyz;
  m[9] = hxz;
}

// phi of `cell` of the current pair (normal layout), same sum as the phi pass.
template <int PREC, int QH, class Off>
__device__ __forceinline__ typename Store<PREC>::R phi_at(const Geo32& geo, const typename Store<PREC>::S* __restrict__ h,
                                                          const typename Store<PREC>::PhiT* __restrict__ shift,
                                                          unsigned cell, const Off& o) {
  typedef typename Store<PREC>::R R;
  constexpr bool F16 = PREC == 2;
  R s = F16 ? (raw<PREC>(h[(unsigned)hq_rest<QH>() * geo.N + cell]) * (R)(1.0 / KH16) + (R)__ldg(shift + cell)) * (R)hq_w<QH>(hq_rest<QH>())
            : raw<PREC>(h[(unsigned)hq_rest<QH>() * geo.N + cell]);
#pragma unroll
  for (int k = 0; k < hq_rest<QH>(); ++k) {
    R a, b;
    unsigned fa, fb;
    load_pair<PREC, 0>(h, geo.N, cell, o, k, QH - 1 - k, hq_cx<QH>(k), hq_cy<QH>(k), hq_cz<QH>(k), a, b, fa, fb);
    if (F16)
      s += (R)hq_w<QH>(k) * ((a + b) * (R)(1.0 / KH16) + ((R)__ldg(shift + fa) + (R)__ldg(shift + fb)));
    else
      s += a + b;
  }
  return s;
}

// Offsets of cell (x, y, z): the general form, or (INT) the interior one.
template <int INT>
struct OffOf;
template <>
struct OffOf<0> {
  typedef CellOff T;
  static __device__ __forceinline__ CellOff at(const Geo32& geo, unsigned x, unsigned y, unsigned z, unsigned blk) {
    CellOff o;
    o.X = axis_off(x, geo.nx, 1, geo.wall[0]);
    o.Y = axis_off(y, geo.ny, (int)geo.nx, geo.wall[1]);
    o.Z = axis_off(z, geo.nz, (int)(geo.nx * geo.ny), geo.wall[2]);
    o.blk = blk;  // a bounced population was written by this cell
    return o;
  }
};
template <>
struct OffOf<1> {
  typedef CellOffI T;
  static __device__ __forceinline__ CellOffI at(const Geo32& geo, unsigned, unsigned, unsigned, unsigned) {
    return CellOffI{(int)geo.nx, geo.nz == 1 ? 0 : (int)(geo.nx * geo.ny)};
  }
};

template <int PREC, int QH, int INT = 0>
__device__ __forceinline__ void h_moments_xyz(const Geo32& geo, const typename Store<PREC>::S* __restrict__ h,
                                              const typename Store<PREC>::PhiT* __restrict__ shift, unsigned x,
                                              unsigned y, unsigned z, typename Store<PREC>::R m[10],
                                              unsigned blk = 0) {
  const unsigned cell = x + geo.nx * (y + geo.ny * z);
  h_moments_at<PREC, QH>(geo, h, shift, cell, OffOf<INT>::at(geo, x, y, z, blk), m);
}

template <int PREC, int QH, int INT = 0>
__device__ __forceinline__ typename Store<PREC>::R phi_at_xyz(const Geo32& geo,
                                                              const typename Store<PREC>::S* __restrict__ h,
                                                              const typename Store<PREC>::PhiT* __restrict__ shift,
                                                              unsigned x, unsigned y, unsigned z,
                                                              unsigned blk = 0) {
  const unsigned cell = x + geo.nx * (y + geo.ny * z);
  return phi_at<PREC, QH>(geo, h, shift, cell, OffOf<INT>::at(geo, x, y, z, blk));
}

// position r in [0, 2 (W + H) - 4) of the frame of a W x H plane -> (i, j)
__device__ __forceinline__ void frame_pos(int r, int W, int H, int& i, int& j) {
  if (r < W) {
    i = r;
    j = 0;
  } else if (r < 2 * W) {
    i = r - W;
    j = H - 1;
  } else if (r < 2 * W + (H - 2)) {
    i = 0;
    j = 1 + (r - 2 * W);
  } else {
    i = W - 1;
    j = 1 + (r - 2 * W - (H - 2));
  }
}

// grid: (ceil(nx / ZM_TX), ceil(ny / TY), ceil(nz / zc)), block ZM_TX x TY with
// TY = zm_ty(FLAT).
// SOLID: the lattice holds solid cells, given by `links` (one word per cell).
// tclock (launches replayed from a CUDA graph): the FP16 rounding seed comes
// from the step count *tclock + tofs in device memory instead of `seed`, the
// same function of the step count as the host's.
// One tile of the fused step: the xy tile (bx, by) of TX x TY columns and
// the z chunk bz of zc planes (the grid of k_step_zm, or an entry of the
// batched engine's work list), run by a block of TX x TY threads.  The caller
// has waited for the previous step.
template <int PREC, int QH, int TY, int FLAT, int SOLID, int TX = ZM_TX>
__device__ __forceinline__ void zm_tile(const Geo32& geo, const Phys& ph, const typename Store<PREC>::S* __restrict__ hA,
                                        const typename Store<PREC>::S* __restrict__ gA,
                                        typename Store<PREC>::S* __restrict__ hB, typename Store<PREC>::S* __restrict__ gB,
                                        const typename Store<PREC>::PhiT* __restrict__ phi_shift,
                                        typename Store<PREC>::PhiT* __restrict__ phi_out, int zc, unsigned seed,
                                        const unsigned* __restrict__ links, const __half* __restrict__ pg_in,
                                        __half* __restrict__ pg_out, int bx, int by, int bz) {
  typedef typename Store<PREC>::PhiT PhiT;
  typedef typename Store<PREC>::R R;
  constexpr int NT = TX * TY;
  constexpr int PW = TX + 2, PH = TY + 2, PS = PW * PH;
  constexpr int NRING = 2 * (PW + PH) - 4;
  static_assert(NRING <= NT, "one thread per ring position");
  // phi planes z - 1, z, z + 1 and the one being filled: with four slots the
  // fill of plane z + 1 overwrites plane z - 3, which every thread finished
  // reading before the barrier of the previous plane, so one barrier per plane
  // suffices.  The h moments are per thread and need none.  FP64 keeps three
  // slots (static shared memory stays under 48 KB) and a second barrier.
  constexpr int NS = FLAT ? 1 : (sizeof(R) == 8 ? 3 : 4);
  __shared__ PhiT ring[NS][PS];
  __shared__ R hmom[FLAT ? 1 : 2][10 * NT];  // h moments of the tile's own cells
  constexpr bool F16 = PREC == 2;
  __shared__ float pring[F16 ? NS : 1][F16 ? PS : 1];  // FP16S: p* shifts of the stored g, ring like phi
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int x0 = bx * TX, y0 = by * TY;
  const int z0 = bz * zc;
  const int z1 = min(z0 + zc, (int)geo.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < (int)geo.nx && y < (int)geo.ny;
  const unsigned xq = (unsigned)wrap_or_clamp(x, (int)geo.nx, geo.wall[0]);
  const unsigned yq = (unsigned)wrap_or_clamp(y, (int)geo.ny, geo.wall[1]);
  int ri = 0, rj = 0;
  if (tid < NRING) frame_pos(tid, PW, PH, ri, rj);
  const unsigned rxq = (unsigned)wrap_or_clamp(x0 - 1 + ri, (int)geo.nx, geo.wall[0]);
  const unsigned ryq = (unsigned)wrap_or_clamp(y0 - 1 + rj, (int)geo.ny, geo.wall[1]);

  // L1 prefetch of the g populations plane zp's collision will read
  auto prefetch_plane = [&](int zp) {
    if (!(PFL_ZM_PREFETCH && PREC == 1 && QH == 15 && !FLAT) || !active || zp >= z1) return;
    constexpr int QG = qg_of<QH>();
    const unsigned c = (unsigned)x + geo.nx * ((unsigned)y + geo.ny * (unsigned)zp);
#pragma unroll
    for (int i = 0; i < QG; ++i) prefetch_l1(gA + (unsigned)i * geo.N + c);
  };

  // The march over the block's z planes, in the general form (INT = 0) or, for
  // blocks whose tile, ring and planes z0 - 2 .. z1 + 1 lie clear of the
  // lattice's faces, the interior one (INT = 1: every link valid, neighbour
  // offsets without wall or wrap tests).
  auto march = [&](auto int_tag) {
  constexpr int INT = decltype(int_tag)::value;
  // phi of plane zp over the tile (with the h moments of the own cells) and its ring
  auto fill = [&](int zp, int slot, int mslot) {
    const unsigned zq = (unsigned)wrap_or_clamp(zp, (int)geo.nz, geo.wall[2]);
    R m[10];
    const unsigned bt = SOLID ? __ldg(links + xq + geo.nx * (yq + geo.ny * zq)) : 0u;
    h_moments_xyz<PREC, QH, INT>(geo, hA, phi_shift, xq, yq, zq, m, bt);
    ring[slot][(ty + 1) * PW + tx + 1] = (PhiT)m[0];
    if constexpr (F16) pring[slot][(ty + 1) * PW + tx + 1] = ld_pshift(pg_in, xq + geo.nx * (yq + geo.ny * zq));
#pragma unroll
    for (int k = 0; k < 10; ++k) hmom[mslot][k * NT + tid] = m[k];
    if (tid < NRING) {
      const unsigned br = SOLID ? __ldg(links + rxq + geo.nx * (ryq + geo.ny * zq)) : 0u;
      ring[slot][rj * PW + ri] = (PhiT)phi_at_xyz<PREC, QH, INT>(geo, hA, phi_shift, rxq, ryq, zq, br);
      if constexpr (F16) pring[slot][rj * PW + ri] = ld_pshift(pg_in, rxq + geo.nx * (ryq + geo.ny * zq));
    }
  };

  prefetch_plane(z0);
  if (FLAT) {
    fill(0, 0, 0);
  } else {
    fill(z0 - 1, 0, 1);  // moments of plane z0 - 1 are never used (written to the spare slot)
    fill(z0, 1, 0);
  }
  for (int z = z0; z < z1; ++z) {
    const int b = z - (z0 - 1);
    if (!FLAT) fill(z + 1, (b + 1) % NS, (z + 1 - z0) & 1);
    __syncthreads();
    if (!FLAT) prefetch_plane(z + 1);
    const unsigned cell = (unsigned)x + geo.nx * ((unsigned)y + geo.ny * (unsigned)z);
    const unsigned blk = (SOLID && active) ? __ldg(links + cell) : 0u;
    if (SOLID && active && (blk & SOLID_SELF)) {
      phi_out[cell] = (PhiT)0;  // solid cells are not updated; their populations stay zero
    } else if (active) {
      const typename OffOf<INT>::T o = OffOf<INT>::at(geo, (unsigned)x, (unsigned)y, (unsigned)z, blk);
      SmemPhi<PREC, FLAT, PW> at;
      if (FLAT) {
        at.plane[0] = at.plane[1] = at.plane[2] = ring[0];
      } else {
        at.plane[0] = ring[(b - 1) % NS];
        at.plane[1] = ring[b % NS];
        at.plane[2] = ring[(b + 1) % NS];
      }
      // with one z plane the z neighbours are the plane itself (periodic or mirrored)
      at.i0 = (ty + 1) * PW + (tx + 1);
      at.blk = blk;
      SmemShift<FLAT, PW> psh;
      if constexpr (F16) {
        if (FLAT) {
          psh.plane[0] = psh.plane[1] = psh.plane[2] = pring[0];
        } else {
          psh.plane[0] = pring[(b - 1) % NS];
          psh.plane[1] = pring[b % NS];
          psh.plane[2] = pring[(b + 1) % NS];
        }
        psh.i0 = at.i0;
      }
      phi_out[cell] = (PhiT)at(0, 0, 0);
      collide_cell<PREC, QH, 0, 1, SmemPhi<PREC, FLAT, PW>, 1, SmemShift<FLAT, PW>, typename OffOf<INT>::T>(
          geo, ph, o, hA, gA, hB, gB, at, phi_shift, cell, seed, &hmom[FLAT ? 0 : ((z - z0) & 1)][tid], NT, psh,
          pg_out);
    }
    if (NS == 3) __syncthreads();
  }
  };
  const bool interior = !SOLID && PFL_ZM_INTERIOR && x0 >= 2 && x0 + TX + 1 < (int)geo.nx && y0 >= 2 &&
                        y0 + TY + 1 < (int)geo.ny && (FLAT || (z0 >= 2 && z1 + 1 < (int)geo.nz));
  if (interior)
    march(std::integral_constant<int, 1>());
  else
    march(std::integral_constant<int, 0>());
}

template <int PREC, int QH, int FLAT, int SOLID = 0>
__global__ void __launch_bounds__(ZM_TX * zm_ty(FLAT), (PREC == 0 ? PFL_ZM_MINB_FP64 : PFL_ZM_MINB) * ZM_TY / zm_ty(FLAT))
    k_step_zm(Geo32 geo, Phys ph, const typename Store<PREC>::S* __restrict__ hA,
              const typename Store<PREC>::S* __restrict__ gA, typename Store<PREC>::S* __restrict__ hB,
              typename Store<PREC>::S* __restrict__ gB, const typename Store<PREC>::PhiT* __restrict__ phi_shift,
              typename Store<PREC>::PhiT* __restrict__ phi_out, int zc, unsigned seed,
              const unsigned* __restrict__ links = nullptr, const unsigned long long* tclock = nullptr,
              int tofs = 0, const __half* __restrict__ pg_in = nullptr, __half* __restrict__ pg_out = nullptr) {
  // global memory only after the previous step has completed
  if (PFL_ZM_PDL) asm volatile("griddepcontrol.wait;" ::: "memory");
  if (PREC == 2 && tclock) seed = step_seed_of(*tclock + (unsigned long long)tofs);
  zm_tile<PREC, QH, zm_ty(FLAT), FLAT, SOLID>(geo, ph, hA, gA, hB, gB, phi_shift, phi_out, zc, seed, links, pg_in,
                                              pg_out, blockIdx.x, blockIdx.y, blockIdx.z);
}

}  // namespace pfl
