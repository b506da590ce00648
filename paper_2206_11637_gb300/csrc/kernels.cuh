// PFLBM device kernels: fused stream-collide of h (D3Q15 / D3Q27, or D2Q9 in
// 2-D) and g (D3Q27, or D2Q9 in 2-D) with
// in-place AA streaming, the phi = sum h pass, initialisation, field output
// and FP64 reductions.
//
// Time step t (section "Conservative Allen-Cahn model"; schedule: both
// collisions at t use phi^t and its stencil, u^t from g in the same cell;
// then both sets stream; then phi^{t+1} = sum_i h_i):
//   stencil   grad phi = 3 sum w_i c_i phi(x + c_i), lap phi = 6 sum w_i (phi(x + c_i) - phi(x))
//             over D3Q27 weights; phi mirrored across no-slip faces.
//   forces    mu = 4 beta phi (phi - 1)(phi - 1/2) - kappa lap phi, F_s = mu grad phi,
//             F_b = rho g, F_p = -p* c_s^2 (rho_H - rho_L) grad phi,
//             F_mu = nu (rho_H - rho_L)[grad u + grad u^T] grad phi with the strain
//             rate -(omega / c_s^2) Pi^neq from the non-equilibrium second
//             moment of g taken against g^eq(p*, u0), u0 = j + (F_s+F_b+F_p)/(2 rho).
//   velocity  u = sum c_i g_i + F / (2 rho).
//   g         weighted-orthogonal MRT with degree 2 at omega(phi) and degree >= 3
//             at 1.  With moments graded by degree and w-orthogonal, M^-1 S M
//             acts as a projector sum, and the post-collision state reduces to
//               g+_i = g^eq_i + (1 - omega) w_i 9/2 (c_i c_i - I/3) : Pi^d + 1/2 G_i,
//             Pi^d = sum c c (g - g^eq(p*, u)), G_i = 3 w_i c_i . F / rho (Guo
//             source; its (I - S/2) factor is 1/2 on the conserved degree 1).
//   h         degrees 1 and 2 at omega_phi, degree >= 3 at 1:
//               h+_i = h^eq_i + (1 - omega_phi)[3 w_i c_i . J^d + w_i 9/2 (c_i c_i - I/3) : Pi^dh]
//                      + (1 - omega_phi / 2) w_i c_i . (theta n),
//             h^eq_i = w_i phi (1 + 3 c_i . u), theta = 4 phi (1 - phi) / xi,
//             n = grad phi / (|grad phi| + 1e-6).
//
// AA pattern (one array per set, updated in place):
//   even step: read f_i at x from slot i, write f+_i to slot opp(i) at x;
//   odd step:  read f_i at x from slot opp(i) of x - c_i (slot i of x itself when
//              x - c_i lies behind a no-slip face: halfway bounce-back), write
//              f+_i to slot i of x + c_i (slot opp(i) of x behind a wall).
//   Every location is read and then written by the same thread, so the update
//   is race-free without a second array.  In both parities the population read
//   at x for direction i was written by x - c_i (by x itself after a bounce).
//
// phi is double-buffered: a step reads phi^t from `phi` (stencil) and, for the
// FP16S format, phi^{t-1} -- from which the shifts of the populations it loads
// follow -- from `shift`; it writes populations shifted by phi^t values.  The
// phi pass then writes phi^{t+1} into the buffer that held phi^{t-1}.
#pragma once
#include "lattice.cuh"

namespace pfl {

struct Geo {
  int nx, ny, nz;
  int wall[3];  // per axis: 1 = no-slip faces, 0 = periodic
  long long N;
};

struct Phys {
  double rho_h, rho_l, tau_h, tau_l, beta, kappa, inv_xi, omega_phi, gx, gy, gz;
};

// Coordinates of x-1, x, x+1 along one axis.  pop[]: -1 behind a wall.
// sten[]: clamped at walls (mirror of phi), wrapped when periodic.
__device__ __forceinline__ void axis_nb(int x, int n, int wall, int pop[3], int sten[3]) {
  int xm = x - 1, xp = x + 1;
  if (wall) {
    pop[0] = xm;
    pop[2] = (xp < n) ? xp : -1;
    sten[0] = xm < 0 ? 0 : xm;
    sten[2] = xp >= n ? n - 1 : xp;
  } else {
    xm = xm < 0 ? xm + n : xm;
    xp = xp >= n ? xp - n : xp;
    pop[0] = xm;
    pop[2] = xp;
    sten[0] = xm;
    sten[2] = xp;
  }
  pop[1] = x;
  sten[1] = x;
}

struct Nb {
  int px[3], py[3], pz[3];
  int sx[3], sy[3], sz[3];
};

__device__ __forceinline__ void cell_coords(const Geo& geo, long long cell, int& x, int& y, int& z) {
  long long yz = cell / geo.nx;
  x = (int)(cell - yz * geo.nx);
  z = (int)(yz / geo.ny);
  y = (int)(yz - (long long)z * geo.ny);
}

__device__ __forceinline__ void make_nb(const Geo& geo, int x, int y, int z, Nb& nb) {
  axis_nb(x, geo.nx, geo.wall[0], nb.px, nb.sx);
  axis_nb(y, geo.ny, geo.wall[1], nb.py, nb.sy);
  axis_nb(z, geo.nz, geo.wall[2], nb.pz, nb.sz);
}

__device__ __forceinline__ long long lin(const Geo& geo, int x, int y, int z) {
  return (long long)x + (long long)geo.nx * ((long long)y + (long long)geo.ny * (long long)z);
}

// Location of population i (opposite oi) arriving at `cell` for the next
// collision, and the cell that wrote it.  READ_ODD = state left by an even
// step (gather from x - c with bounce-back); otherwise the normal state.
template <int READ_ODD>
__device__ __forceinline__ size_t src_index(const Geo& geo, const Nb& nb, long long cell, int i, int oi, int cx,
                                            int cy, int cz, long long& from) {
  int ax = nb.px[1 - cx], ay = nb.py[1 - cy], az = nb.pz[1 - cz];
  const bool inside = ax >= 0 && ay >= 0 && az >= 0;
  from = inside ? lin(geo, ax, ay, az) : cell;
  if (!READ_ODD) return (size_t)i * geo.N + cell;
  if (inside) return (size_t)oi * geo.N + from;
  return (size_t)i * geo.N + cell;
}

// Destination of the post-collision population i of `cell`.
template <int ODD>
__device__ __forceinline__ size_t dst_index(const Geo& geo, const Nb& nb, long long cell, int i, int oi, int cx,
                                            int cy, int cz) {
  if (!ODD) return (size_t)oi * geo.N + cell;
  int ax = nb.px[1 + cx], ay = nb.py[1 + cy], az = nb.pz[1 + cz];
  if (ax >= 0 && ay >= 0 && az >= 0) return (size_t)i * geo.N + lin(geo, ax, ay, az);
  return (size_t)oi * geo.N + cell;
}

// Everything a cell needs before its collisions.
template <typename R>
struct Macro {
  R phi, gx, gy, gz, lap;
  R rho, omega, nu;
  R pst, jx, jy, jz;                  // p*, sum c g
  R pxx, pyy, pzz, pxy, pyz, pxz;     // sum c c g
  R Fx, Fy, Fz, ux, uy, uz;
};

template <int PREC, int QG>
__device__ __forceinline__ void stencil(const Geo& geo, const Nb& nb, long long cell,
                                        const typename Store<PREC>::PhiT* __restrict__ phi,
                                        Macro<typename Store<PREC>::R>& m, unsigned blk = 0) {
  typedef typename Store<PREC>::R R;
  R pc = (R)__ldg(phi + cell);
  R gx = 0, gy = 0, gz = 0, lap = 0;
#pragma unroll
  for (int i = 0; i < QG; ++i) {
    if (i == (QG - 1) / 2) continue;
    const int cx = q27_cx(lq_to27<QG>(i)), cy = q27_cy(lq_to27<QG>(i)), cz = q27_cz(lq_to27<QG>(i));
    // a solid neighbour (bit (cx+1) + 3(cy+1) + 9(cz+1) of blk) reads as this cell
    R v = (blk >> ((cx + 1) + 3 * (cy + 1) + 9 * (cz + 1))) & 1u
              ? pc
              : (R)__ldg(phi + lin(geo, nb.sx[1 + cx], nb.sy[1 + cy], nb.sz[1 + cz]));
    const R w = (R)lq_w<QG>(i);
    if (cx) gx += (cx > 0 ? w : -w) * v;
    if (cy) gy += (cy > 0 ? w : -w) * v;
    if (cz) gz += (cz > 0 ? w : -w) * v;
    lap += w * (v - pc);
  }
  m.phi = pc;
  m.gx = (R)3 * gx;
  m.gy = (R)3 * gy;
  m.gz = (R)3 * gz;
  m.lap = (R)6 * lap;
}

// Hydrodynamic moments, forces and velocity.  gv receives the 27 values (used
// by the BGK mode; dead code otherwise).
template <int PREC, int QG, int READ_ODD>
__device__ __forceinline__ void hydro_macro(const Geo& geo, const Phys& ph, const Nb& nb, long long cell,
                                            const typename Store<PREC>::S* __restrict__ g, Macro<typename Store<PREC>::R>& m,
                                            typename Store<PREC>::R gv[QG], const __half* __restrict__ pg = nullptr) {
  typedef typename Store<PREC>::R R;
  R pst = 0, jx = 0, jy = 0, jz = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pyz = 0, pxz = 0;
#pragma unroll
  for (int i = 0; i < QG; ++i) {
    const int cx = q27_cx(lq_to27<QG>(i)), cy = q27_cy(lq_to27<QG>(i)), cz = q27_cz(lq_to27<QG>(i));
    long long from;
    const size_t idx = src_index<READ_ODD>(geo, nb, cell, i, QG - 1 - i, cx, cy, cz, from);
    R psh = 0;
    if constexpr (PREC == 2) psh = ld_pshift(pg, from);
    R v = ld_g<PREC, QG>(g, idx, i, psh);
    gv[i] = v;
    pst += v;
    if (cx) jx += cx > 0 ? v : -v;
    if (cy) jy += cy > 0 ? v : -v;
    if (cz) jz += cz > 0 ? v : -v;
    if (cx) pxx += v;
    if (cy) pyy += v;
    if (cz) pzz += v;
    if (cx && cy) pxy += (cx * cy > 0) ? v : -v;
    if (cy && cz) pyz += (cy * cz > 0) ? v : -v;
    if (cx && cz) pxz += (cx * cz > 0) ? v : -v;
  }
  m.pst = pst;
  m.jx = jx;
  m.jy = jy;
  m.jz = jz;
  m.pxx = pxx;
  m.pyy = pyy;
  m.pzz = pzz;
  m.pxy = pxy;
  m.pyz = pyz;
  m.pxz = pxz;

  const R phi = m.phi;
  const R drho = (R)(ph.rho_h - ph.rho_l);
  m.rho = (R)ph.rho_l + phi * drho;
  const R tau = (R)ph.tau_l + phi * (R)(ph.tau_h - ph.tau_l);
  m.omega = (R)1 / tau;
  m.nu = (tau - (R)0.5) * (R)(1.0 / 3.0);
  const R mu = (R)4 * (R)ph.beta * phi * (phi - (R)1) * (phi - (R)0.5) - (R)ph.kappa * m.lap;
  const R inv2rho = (R)0.5 / m.rho;
  const R cp = -pst * (R)(1.0 / 3.0) * drho;
  // F_s + F_b + F_p
  R Fx = mu * m.gx + m.rho * (R)ph.gx + cp * m.gx;
  R Fy = mu * m.gy + m.rho * (R)ph.gy + cp * m.gy;
  R Fz = mu * m.gz + m.rho * (R)ph.gz + cp * m.gz;
  const R u0x = jx + Fx * inv2rho, u0y = jy + Fy * inv2rho, u0z = jz + Fz * inv2rho;
  const R p3 = pst * (R)(1.0 / 3.0);
  const R nxx = pxx - p3 - u0x * u0x, nyy = pyy - p3 - u0y * u0y, nzz = pzz - p3 - u0z * u0z;
  const R nxy = pxy - u0x * u0y, nyz = pyz - u0y * u0z, nxz = pxz - u0x * u0z;
  const R cm = (R)-3 * m.nu * m.omega * drho;
  Fx += cm * (nxx * m.gx + nxy * m.gy + nxz * m.gz);
  Fy += cm * (nxy * m.gx + nyy * m.gy + nyz * m.gz);
  Fz += cm * (nxz * m.gx + nyz * m.gy + nzz * m.gz);
  m.Fx = Fx;
  m.Fy = Fy;
  m.Fz = Fz;
  m.ux = jx + Fx * inv2rho;
  m.uy = jy + Fy * inv2rho;
  m.uz = jz + Fz * inv2rho;
}

// h population k arriving at `cell` (FP16S: shifted by phi of the writing cell,
// read from `shift`).
template <int PREC, int QH, int READ_ODD>
__device__ __forceinline__ typename Store<PREC>::R load_h(const Geo& geo, const Nb& nb, long long cell, int k,
                                                          const typename Store<PREC>::S* __restrict__ h,
                                                          const typename Store<PREC>::PhiT* __restrict__ shift) {
  typedef typename Store<PREC>::R R;
  long long from;
  const size_t idx = src_index<READ_ODD>(geo, nb, cell, k, QH - 1 - k, hq_cx<QH>(k), hq_cy<QH>(k), hq_cz<QH>(k), from);
  R sh = 0;
  if constexpr (PREC == 2) sh = __ldg(shift + from);
  return ld_h<PREC, QH>(h, idx, k, sh);
}

// One time step: collide both sets at every cell and stream them in place.
template <int PREC, int QH, int ODD, int BGK>
__global__ void __launch_bounds__(256) k_step(Geo geo, Phys ph, typename Store<PREC>::S* __restrict__ h,
                                              typename Store<PREC>::S* __restrict__ g,
                                              const typename Store<PREC>::PhiT* __restrict__ phi,
                                              const typename Store<PREC>::PhiT* __restrict__ shift,
                                              const __half* __restrict__ pg_in = nullptr,
                                              __half* __restrict__ pg_out = nullptr) {
  typedef typename Store<PREC>::R R;
  constexpr int QG = qg_of<QH>();
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= geo.N) return;
  int x, y, z;
  cell_coords(geo, cell, x, y, z);
  Nb nb;
  make_nb(geo, x, y, z, nb);
  Macro<R> m;
  stencil<PREC, QG>(geo, nb, cell, phi, m);
  R gv[QG];
  hydro_macro<PREC, QG, ODD>(geo, ph, nb, cell, g, m, gv, pg_in);
  // FP16S: the p* shift of everything this cell writes
  R pw = 0;
  if constexpr (PREC == 2) {
    const __half ps = __float2half_rn(m.pst);
    pg_out[cell] = ps;
    pw = __half2float(ps);
  }

  // ---- g collision and streaming
  {
    const R ux = m.ux, uy = m.uy, uz = m.uz;
    const R uu = ux * ux + uy * uy + uz * uz;
    const R p3 = m.pst * (R)(1.0 / 3.0);
    const R dxx = m.pxx - p3 - ux * ux, dyy = m.pyy - p3 - uy * uy;
    const R dzz = QG == 9 ? (R)0 : m.pzz - p3 - uz * uz;  // 2-D: the trace runs over x and y
    const R dxy = m.pxy - ux * uy, dyz = m.pyz - uy * uz, dxz = m.pxz - ux * uz;
    const R tr3 = (dxx + dyy + dzz) * (R)(1.0 / 3.0);
    const R a2 = ((R)1 - m.omega) * (R)4.5;
    const R inv_rho = (R)1 / m.rho;
    const R fx = (R)1.5 * m.Fx * inv_rho, fy = (R)1.5 * m.Fy * inv_rho, fz = (R)1.5 * m.Fz * inv_rho;
    // BGK: (1 - omega/2) G_i with G_i = 2 w_i (1.5 c.F / rho)
    const R om = m.omega, fbgk = ((R)1 - (R)0.5 * om) * (R)2;
#pragma unroll
    for (int i = 0; i < QG; ++i) {
      const int cx = q27_cx(lq_to27<QG>(i)), cy = q27_cy(lq_to27<QG>(i)), cz = q27_cz(lq_to27<QG>(i));
      const R w = (R)lq_w<QG>(i);
      const R cu = (R)cx * ux + (R)cy * uy + (R)cz * uz;
      const R geq = w * (m.pst + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * uu);
      const R cf = (R)cx * fx + (R)cy * fy + (R)cz * fz;  // 1.5 c.F / rho
      R post;
      if (BGK) {
        post = gv[i] - om * (gv[i] - geq) + fbgk * w * cf;
      } else {
        const R hd = (R)(cx * cx) * dxx + (R)(cy * cy) * dyy + (R)(cz * cz) * dzz +
                     (R)2 * ((R)(cx * cy) * dxy + (R)(cy * cz) * dyz + (R)(cx * cz) * dxz) - tr3;
        post = geq + w * (a2 * hd + cf);
      }
      st_g<PREC, QG>(g, dst_index<ODD>(geo, nb, cell, i, QG - 1 - i, cx, cy, cz), i, post, pw);
    }
  }

  // ---- h collision and streaming
  {
    R hv[QH];
    R phl = 0, jx = 0, jy = 0, jz = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pyz = 0, pxz = 0;
#pragma unroll
    for (int k = 0; k < QH; ++k) {
      const int cx = hq_cx<QH>(k), cy = hq_cy<QH>(k), cz = hq_cz<QH>(k);
      const R v = load_h<PREC, QH, ODD>(geo, nb, cell, k, h, shift);
      hv[k] = v;
      phl += v;
      if (cx) jx += cx > 0 ? v : -v;
      if (cy) jy += cy > 0 ? v : -v;
      if (cz) jz += cz > 0 ? v : -v;
      if (cx) pxx += v;
      if (cy) pyy += v;
      if (cz) pzz += v;
      if (cx && cy) pxy += (cx * cy > 0) ? v : -v;
      if (cy && cz) pyz += (cy * cz > 0) ? v : -v;
      if (cx && cz) pxz += (cx * cz > 0) ? v : -v;
    }
    const R ux = m.ux, uy = m.uy, uz = m.uz;
    const R omp = (R)ph.omega_phi;
    const R gn = sqrt(m.gx * m.gx + m.gy * m.gy + m.gz * m.gz);
    const R theta = (R)4 * m.phi * ((R)1 - m.phi) * (R)ph.inv_xi;
    const R tn = theta / (gn + (R)1e-6);
    const R tx = tn * m.gx, ty = tn * m.gy, tz = tn * m.gz;  // theta * n
    const R src = (R)1 - (R)0.5 * omp;
    const R a1 = ((R)1 - omp) * (R)3, a2 = ((R)1 - omp) * (R)4.5;
    const R Jx = jx - phl * ux, Jy = jy - phl * uy, Jz = jz - phl * uz;
    const R p3 = phl * (R)(1.0 / 3.0);
    const R dxx = pxx - p3, dyy = pyy - p3, dzz = QG == 9 ? (R)0 : pzz - p3;
    const R tr3 = (dxx + dyy + dzz) * (R)(1.0 / 3.0);
    // populations are written as q = h+ / w - shift; the shift is this cell's phi
    const R sh = (PREC == 2) ? m.phi : (R)0;
#pragma unroll
    for (int k = 0; k < QH; ++k) {
      const int cx = hq_cx<QH>(k), cy = hq_cy<QH>(k), cz = hq_cz<QH>(k);
      const R cu = (R)cx * ux + (R)cy * uy + (R)cz * uz;
      const R ct = (R)cx * tx + (R)cy * ty + (R)cz * tz;
      R q;
      if (BGK) {
        const R w = (R)hq_w<QH>(k);
        const R heq = w * phl * ((R)1 + (R)3 * cu);
        q = (hv[k] - omp * (hv[k] - heq)) * (R)(1.0 / hq_w<QH>(k)) + src * ct - sh;
      } else {
        const R cJ = (R)cx * Jx + (R)cy * Jy + (R)cz * Jz;
        const R hd = (R)(cx * cx) * dxx + (R)(cy * cy) * dyy + (R)(cz * cz) * dzz +
                     (R)2 * ((R)(cx * cy) * pxy + (R)(cy * cz) * pyz + (R)(cx * cz) * pxz) - tr3;
        q = (phl - sh) + phl * (R)3 * cu + a1 * cJ + a2 * hd + src * ct;
      }
      st_h_q<PREC, QH>(h, dst_index<ODD>(geo, nb, cell, k, QH - 1 - k, cx, cy, cz), k, q);
    }
  }
}

// phi = sum_i h_i of the state left by the last step (READ_ODD after an even
// step); `shift` holds the shifts of the stored populations.
template <int PREC, int QH, int READ_ODD>
__global__ void __launch_bounds__(256) k_phi(Geo geo, const typename Store<PREC>::S* __restrict__ h,
                                             const typename Store<PREC>::PhiT* __restrict__ shift,
                                             typename Store<PREC>::PhiT* __restrict__ phi) {
  typedef typename Store<PREC>::R R;
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= geo.N) return;
  int x, y, z;
  cell_coords(geo, cell, x, y, z);
  Nb nb;
  make_nb(geo, x, y, z, nb);
  R s = 0;
#pragma unroll
  for (int k = 0; k < QH; ++k) s += load_h<PREC, QH, READ_ODD>(geo, nb, cell, k, h, shift);
  phi[cell] = s;
}

// FP16S fresh state, first pass: the shifts of cells [c0, c0 + count) --
// their own initial phi (FP32) and fp16(p*) -- into hshift and pshift (inputs
// indexed from c0; p0 may be NULL).
static __global__ void k_init_shift(long long c0, long long count, const double* __restrict__ phi0,
                             const double* __restrict__ p0, float* __restrict__ hshift, __half* __restrict__ pshift) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  hshift[c0 + t] = (float)phi0[t];
  pshift[c0 + t] = __float2half_rn(p0 ? (float)p0[t] : 0.0f);
}

// Equilibrium initial state (normal layout) for cells [c0, c0 + count).
// Inputs are FP64 arrays indexed from c0 (phi0, u0x, u0y, u0z, p0; u and p may
// be NULL).  FP16S (after k_init_shift has written every cell's shifts):
// population c of cell x is stored the way a step would have pushed it, against
// the shifts of its writer x - c (of x itself where x - c lies behind a wall),
// so that the readers' convention holds from the first step on and a cell at
// rest in a uniform region is stored exactly.
template <int PREC, int QH>
__global__ void k_init(Geo geo, typename Store<PREC>::S* __restrict__ h, typename Store<PREC>::S* __restrict__ g,
                       long long c0, long long count, const double* __restrict__ phi0,
                       const double* __restrict__ u0x, const double* __restrict__ u0y,
                       const double* __restrict__ u0z, const double* __restrict__ p0,
                       const float* __restrict__ hshift = nullptr, const __half* __restrict__ pshift = nullptr) {
  typedef typename Store<PREC>::R R;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const long long cell = c0 + t;
  const R ph = (R)phi0[t];
  const R ux = u0x ? (R)u0x[t] : (R)0, uy = u0y ? (R)u0y[t] : (R)0, uz = u0z ? (R)u0z[t] : (R)0;
  const R ps = p0 ? (R)p0[t] : (R)0;
  const R uu = ux * ux + uy * uy + uz * uz;
  constexpr int QG = qg_of<QH>();
  Nb nb;
  if constexpr (PREC == 2) {
    int x, y, z;
    cell_coords(geo, cell, x, y, z);
    make_nb(geo, x, y, z, nb);
  }
#pragma unroll
  for (int i = 0; i < QG; ++i) {
    const int j = lq_to27<QG>(i);
    const int cx = q27_cx(j), cy = q27_cy(j), cz = q27_cz(j);
    const R cu = (R)cx * ux + (R)cy * uy + (R)cz * uz;
    if constexpr (PREC == 2) {  // stored directly as g / w - P_writer
      long long from;
      src_index<0>(geo, nb, cell, i, QG - 1 - i, cx, cy, cz, from);
      const R pw = __half2float(pshift[from]);
      g[(size_t)i * geo.N + cell] = __float2half_rn(((ps - pw) + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * uu) * (R)KG16);
    } else {
      st_g<PREC, QG>(g, (size_t)i * geo.N + cell, i, (R)lq_w<QG>(i) * (ps + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * uu));
    }
  }
#pragma unroll
  for (int k = 0; k < QH; ++k) {
    const int cx = hq_cx<QH>(k), cy = hq_cy<QH>(k), cz = hq_cz<QH>(k);
    const R cu = (R)cx * ux + (R)cy * uy + (R)cz * uz;
    R q = ph * ((R)1 + (R)3 * cu);  // h / w
    if constexpr (PREC == 2) {       // less the writer's phi
      long long from;
      src_index<0>(geo, nb, cell, k, QH - 1 - k, cx, cy, cz, from);
      q = (ph - (R)hshift[from]) + ph * (R)3 * cu;
    }
    st_h_q<PREC, QH>(h, (size_t)k * geo.N + cell, k, q);
  }
}

// FP16S fresh state with solid cells: a population of a fluid cell whose
// incoming link now starts in a solid cell counts as bounced back, written by
// the cell itself; re-store it against the cell's own shifts instead of the
// solid neighbour's (fresh states, before the first step).
template <int QH>
__global__ void k_reshift_blocked(Geo geo, __half* __restrict__ h, __half* __restrict__ g,
                                  const float* __restrict__ hshift, const __half* __restrict__ pshift,
                                  const unsigned* __restrict__ links) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= geo.N) return;
  const unsigned blk = links[cell];
  if (!blk || (blk & (1u << 13))) return;
  int x, y, z;
  cell_coords(geo, cell, x, y, z);
  Nb nb;
  make_nb(geo, x, y, z, nb);
  constexpr int QG = qg_of<QH>();
#pragma unroll
  for (int i = 0; i < QG; ++i) {
    const int j = lq_to27<QG>(i);
    const int cx = q27_cx(j), cy = q27_cy(j), cz = q27_cz(j);
    if (!(blk & (1u << ((1 - cx) + 3 * (1 - cy) + 9 * (1 - cz))))) continue;  // neighbour at x - c is solid
    long long from;
    src_index<0>(geo, nb, cell, i, QG - 1 - i, cx, cy, cz, from);
    const size_t idx = (size_t)i * geo.N + cell;
    const float v = __half2float(g[idx]) + (float)KG16 * (__half2float(pshift[from]) - __half2float(pshift[cell]));
    g[idx] = __float2half_rn(v);
  }
#pragma unroll
  for (int k = 0; k < QH; ++k) {
    const int cx = hq_cx<QH>(k), cy = hq_cy<QH>(k), cz = hq_cz<QH>(k);
    if (!(blk & (1u << ((1 - cx) + 3 * (1 - cy) + 9 * (1 - cz))))) continue;
    long long from;
    src_index<0>(geo, nb, cell, k, QH - 1 - k, cx, cy, cz, from);
    const size_t idx = (size_t)k * geo.N + cell;
    const float v = __half2float(h[idx]) + (float)KH16 * (hshift[from] - hshift[cell]);
    h[idx] = __float2half_rn(v);
  }
}

// Macroscopic output: any of phi, rho, p, ux, uy, uz (device FP64, may be NULL).
// With solid cells (links non-NULL) every output is zero in a solid cell.
template <int PREC, int QH, int READ_ODD>
__global__ void __launch_bounds__(256) k_fields(Geo geo, Phys ph, const typename Store<PREC>::S* __restrict__ g,
                                                const typename Store<PREC>::PhiT* __restrict__ phi, double* o_phi, double* o_rho,
                                                double* o_p, double* o_ux, double* o_uy, double* o_uz,
                                                const unsigned* __restrict__ links = nullptr,
                                                const __half* __restrict__ pg = nullptr) {
  typedef typename Store<PREC>::R R;
  constexpr int QG = qg_of<QH>();
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= geo.N) return;
  int x, y, z;
  cell_coords(geo, cell, x, y, z);
  Nb nb;
  make_nb(geo, x, y, z, nb);
  const unsigned blk = links ? links[cell] : 0u;
  if (blk & (1u << 13)) {
    double* outs[6] = {o_phi, o_rho, o_p, o_ux, o_uy, o_uz};
    for (int k = 0; k < 6; ++k)
      if (outs[k]) outs[k][cell] = 0.0;
    return;
  }
  Macro<R> m;
  stencil<PREC, QG>(geo, nb, cell, phi, m, blk);
  R gv[QG];
  hydro_macro<PREC, QG, READ_ODD>(geo, ph, nb, cell, g, m, gv, pg);
  if (o_phi) o_phi[cell] = (double)m.phi;
  if (o_rho) o_rho[cell] = (double)m.rho;
  if (o_p) o_p[cell] = (double)m.pst * (double)m.rho / 3.0;
  if (o_ux) o_ux[cell] = (double)m.ux;
  if (o_uy) o_uy[cell] = (double)m.uy;
  if (o_uz) o_uz[cell] = (double)m.uz;
}

// Population export in canonical layout (FP64): population i of g (is_g) or h.
template <int PREC, int QH, int READ_ODD>
__global__ void k_export(Geo geo, const typename Store<PREC>::S* __restrict__ f,
                         const typename Store<PREC>::PhiT* __restrict__ shift, int is_g, int i,
                         double* __restrict__ out, const __half* __restrict__ pg = nullptr) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= geo.N) return;
  int x, y, z;
  cell_coords(geo, cell, x, y, z);
  Nb nb;
  make_nb(geo, x, y, z, nb);
  if (is_g) {
    constexpr int QG = qg_of<QH>();
#pragma unroll
    for (int j = 0; j < QG; ++j)
      if (j == i) {
        long long from;
        const int k = lq_to27<QG>(j);
        const size_t idx = src_index<READ_ODD>(geo, nb, cell, j, QG - 1 - j, q27_cx(k), q27_cy(k), q27_cz(k), from);
        float psh = 0.0f;
        if constexpr (PREC == 2) psh = ld_pshift(pg, from);
        out[cell] = (double)ld_g<PREC, QG>(f, idx, j, psh);
      }
  } else {
#pragma unroll
    for (int j = 0; j < QH; ++j)
      if (j == i) out[cell] = (double)load_h<PREC, QH, READ_ODD>(geo, nb, cell, j, f, shift);
  }
}

// Population import (normal layout; h and g with zero shifts).
template <int PREC, int QH>
__global__ void k_import(Geo geo, typename Store<PREC>::S* __restrict__ f, int is_g, int i, const double* __restrict__ in) {
  typedef typename Store<PREC>::R R;
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= geo.N) return;
  const size_t idx = (size_t)i * geo.N + cell;
  if constexpr (PREC != 2) {
    f[idx] = (R)in[cell];
  } else if (is_g) {
#pragma unroll
    for (int j = 0; j < qg_of<QH>(); ++j)
      if (j == i) st_g<PREC, qg_of<QH>()>(f, idx, j, (R)in[cell]);
  } else {
#pragma unroll
    for (int j = 0; j < QH; ++j)
      if (j == i) st_h_q<PREC, QH>(f, idx, j, (R)(in[cell] / hq_w<QH>(j)));
  }
}

// FP64 reductions: per-block partial sums of
//   [phi, phi x, phi y, phi z, 1-phi, (1-phi) x, (1-phi) y, (1-phi) z, nonfinite]
// written to part[block * 9 + k]; k_diag_final sums them in a fixed order.
constexpr int DIAG_BLOCKS = 1216;  // 8 x 152 SMs
constexpr int DIAG_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename PhiT>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag(Geo geo, const PhiT* __restrict__ phi, double* __restrict__ part) {
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < geo.N;
       cell += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_coords(geo, cell, x, y, z);
    const double p = (double)phi[cell];
    if (!isfinite(p)) {
      acc[8] += 1.0;
      continue;
    }
    const double q = 1.0 - p;
    acc[0] += p;
    acc[1] += p * x;
    acc[2] += p * y;
    acc[3] += p * z;
    acc[4] += q;
    acc[5] += q * x;
    acc[6] += q * y;
    acc[7] += q * z;
  }
  __shared__ double sm[DIAG_THREADS / 32][9];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double v = warp_sum(acc[k]);
    if (lane == 0) sm[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    double s = 0;
    for (int w = 0; w < DIAG_THREADS / 32; ++w) s += sm[w][threadIdx.x];
    part[(size_t)blockIdx.x * 9 + threadIdx.x] = s;
  }
}

static __global__ void k_diag_final(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  // one warp per quantity, fixed order
  const int k = blockIdx.x;
  double s = 0;
  for (int b = threadIdx.x; b < nblocks; b += 32) s += part[(size_t)b * 9 + k];
  s = warp_sum(s);
  if (threadIdx.x == 0) out[k] = s;
}

// Largest flow speed |u| (u = sum c g + F / (2 rho), as pfl_fields) over the
// fluid cells: each block writes the largest |u|^2 of its cells to
// part[block] (grid-stride over the lattice; a non-finite u counts as +inf);
// k_max_final takes the largest of the partials.  Solid cells (links non-NULL,
// bit 13) are skipped.
template <int PREC, int QH, int READ_ODD>
__global__ void __launch_bounds__(DIAG_THREADS) k_umax(Geo geo, Phys ph, const typename Store<PREC>::S* __restrict__ g,
                                                       const typename Store<PREC>::PhiT* __restrict__ phi,
                                                       double* __restrict__ part,
                                                       const unsigned* __restrict__ links = nullptr,
                                                       const __half* __restrict__ pg = nullptr) {
  typedef typename Store<PREC>::R R;
  constexpr int QG = qg_of<QH>();
  double best = 0.0;
  for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < geo.N;
       cell += (long long)gridDim.x * blockDim.x) {
    const unsigned blk = links ? links[cell] : 0u;
    if (blk & (1u << 13)) continue;
    int x, y, z;
    cell_coords(geo, cell, x, y, z);
    Nb nb;
    make_nb(geo, x, y, z, nb);
    Macro<R> m;
    stencil<PREC, QG>(geo, nb, cell, phi, m, blk);
    R gv[QG];
    hydro_macro<PREC, QG, READ_ODD>(geo, ph, nb, cell, g, m, gv, pg);
    const double u2 = (double)m.ux * (double)m.ux + (double)m.uy * (double)m.uy + (double)m.uz * (double)m.uz;
    best = isfinite(u2) ? fmax(best, u2) : INFINITY;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  __shared__ double sm[DIAG_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sm[wid] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = sm[0];
    for (int w = 1; w < DIAG_THREADS / 32; ++w) b = fmax(b, sm[w]);
    part[blockIdx.x] = b;
  }
}

// out[0] = sqrt of the largest of part[0 .. nblocks) (one warp)
static __global__ void k_max_final(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  double b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += 32) b = fmax(b, part[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  if (threadIdx.x == 0) out[0] = sqrt(b);
}

}  // namespace pfl

namespace pfl {

// Link words from a solid mask (N bytes, nonzero = solid): for each cell, bit
// (cx+1) + 3(cy+1) + 9(cz+1) for each D3Q27 neighbour that is solid (periodic
// wrap; no neighbour beyond a no-slip face) and bit 13 for the cell itself.
static __global__ void k_links(Geo geo, const unsigned char* __restrict__ mask, unsigned* __restrict__ links) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= geo.N) return;
  int x, y, z;
  cell_coords(geo, cell, x, y, z);
  const int n[3] = {geo.nx, geo.ny, geo.nz};
  const int xc[3] = {x, y, z};
  unsigned w = 0;
  for (int i = 0; i < 27; ++i) {
    const int c[3] = {q27_cx(i), q27_cy(i), q27_cz(i)};
    // the neighbour, wrapped on periodic axes and clamped onto the face cell
    // beyond a no-slip face (where the phi stencil reads); a link through a
    // face already bounces, and a clamped solid face cell reads as this cell
    int t[3];
    for (int a = 0; a < 3; ++a) {
      t[a] = xc[a] + c[a];
      if (t[a] < 0 || t[a] >= n[a]) t[a] = geo.wall[a] ? (t[a] < 0 ? 0 : n[a] - 1) : (t[a] + n[a]) % n[a];
    }
    if (mask[t[0] + (long long)n[0] * (t[1] + (long long)n[1] * t[2])]) w |= 1u << i;
  }
  links[cell] = w;
}

// Zero the populations of solid cells (q arrays of N) so that they stay zero:
// no fluid cell writes into a solid one, and solid cells are not updated.
template <int PREC>
__global__ void k_zero_solid(long long N, int q, const unsigned* __restrict__ links,
                             typename Store<PREC>::S* __restrict__ f) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= N || !(links[cell] & (1u << 13))) return;
  for (int i = 0; i < q; ++i) f[(size_t)i * N + cell] = (typename Store<PREC>::S)0.0f;
}

}  // namespace pfl
