// Discrete adjoint of the MRT stream-collide step (FP64 and FP32 storage).
//
// Forward step t maps the populations s^t = (h^t, g^t) to s^{t+1}: phi^t = sum h,
// the D3Q27 stencil of phi^t, the local collision map P (moments -> forces ->
// post-collision populations, see step.cuh) and streaming.  For an objective
// J = sum_o sum_x W_o(x) phi^{t_o}(x) the adjoint recursion is
//   lambda^t = (d s^{t+1} / d s^t)^T lambda^{t+1} + dJ / d s^t,
//   dJ / d theta = sum_t (dP / d theta)^T lambda^+_t,   theta = (M, xi, sigma),
// where lambda^+_t(x, i) is the adjoint of the post-collision population i of
// cell x: lambda^{t+1} at the cell and slot that streaming delivered it to.
//
// k_adj_local (one thread per cell) recomputes P's intermediates from the saved
// state s^t and runs P's reverse sweep: it writes the adjoint of the local
// pre-collision populations through the moments, and per cell the adjoints of
// the stencil outputs (grad phi, lap phi) and of phi(x) itself.  k_adj_phi then
// gathers the stencil's transpose -- every (cell y, direction c) whose stencil
// read phi at x, walls folded in -- into the adjoint of phi(x), plus W_o at
// observation steps.  Since phi = sum h, that value belongs to all 15 h
// adjoints of x; it is kept once per cell (array `acc`) and added by the next
// reverse step as it reads lambda, instead of being written into 15 arrays.
//
// Adjoint populations are kept in the canonical layout [i][cell] (h: QH N,
// then g: QG N) in the arithmetic type; lambda^t = (local part) + acc^t on the
// h entries.
#pragma once
#include "step.cuh"

namespace pfl {

constexpr int ADJ_THREADS = 128;
// Resident blocks of k_adj_local per SM the compiler is asked for, FP32 (FP64
// is left unbounded: it runs on the FP64 units, and 5 blocks already spill 0.5
// KB).  On the 128x384x128 FP32 bubble (400 steps, lambda gathered first),
// adjoint / forward was 3.43 unbounded (128 registers, 4 blocks), 3.33 at 5
// (96, no spill), 3.24 at 6 (80, 56 B of spill), 3.22 at 7, 3.20 at 8 (64, 156
// B); 6 keeps the spill small on every lattice.
#ifndef PFL_ADJ_MINB32
#define PFL_ADJ_MINB32 6
#endif
template <int PREC>
constexpr int adj_minb() {
  return PREC == 1 ? PFL_ADJ_MINB32 : 0;
}
// (An L1 prefetch of the lambda gathers on entry, to overlap them with the
// forward recomputation, doubled the adjoint's time on the same bubble: 831 ->
// 1691 ms.  It is not used.)

// The step's parameters in the arithmetic type R, converted once on the host:
// converting the doubles of Phys in every thread kept the FP64 pipe (1/64 of
// the FP32 rate on this part) three quarters busy in k_adj_local.  (The fused
// forward step keeps Phys: the same change there measured 2.6 % slower in
// FP16S and 0.9 % in FP32, its schedule losing more to load latency than the
// conversions cost.)
template <typename R>
struct PhysR {
  R rho_l, drho, tau_l, dtau, beta, kappa, inv_xi, omega_phi, gx, gy, gz;
};

template <typename R>
inline PhysR<R> phys_r(const Phys& p) {
  PhysR<R> q;
  q.rho_l = (R)p.rho_l;
  q.drho = (R)(p.rho_h - p.rho_l);
  q.tau_l = (R)p.tau_l;
  q.dtau = (R)(p.tau_h - p.tau_l);
  q.beta = (R)p.beta;
  q.kappa = (R)p.kappa;
  q.inv_xi = (R)p.inv_xi;
  q.omega_phi = (R)p.omega_phi;
  q.gx = (R)p.gx;
  q.gy = (R)p.gy;
  q.gz = (R)p.gz;
  return q;
}

// Parameters of the reverse sweep that the forward step folds into Phys.
struct AdjPar {
  double M, xi, sigma;
};

// The chain-rule factors of (M, xi, sigma) in the arithmetic type, formed once
// on the host: beta = 12 sigma / xi, kappa = 1.5 sigma xi, 1 / xi.
template <typename R>
struct AdjParR {
  R xi2;        // xi^2
  R beta_sig;   // d beta / d sigma = 12 / xi
  R kappa_sig;  // d kappa / d sigma = 1.5 xi
  R beta_xi;    // d beta / d xi = -12 sigma / xi^2
  R kappa_xi;   // d kappa / d xi = 1.5 sigma
};

template <typename R>
inline AdjParR<R> adj_par_r(const AdjPar& a) {
  return AdjParR<R>{(R)(a.xi * a.xi), (R)(12.0 / a.xi), (R)(1.5 * a.xi), (R)(-12.0 * a.sigma / (a.xi * a.xi)),
                    (R)(1.5 * a.sigma)};
}

template <typename R>
__device__ __forceinline__ R block_sum3_to(R a, R b, R c, double* out3) {
  // Block reduction of three values, added in FP64 to out3[0..2]: each block
  // owns its three slots and accumulates over the reverse sweep's steps.  The
  // 32 lanes of a warp sum in the arithmetic type, the warps' sums in FP64
  // (FP64 shuffles of every thread's value kept the FP64 pipe busy).
  __shared__ double sm[ADJ_THREADS / 32][3];
  R v[3] = {a, b, c};
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    R s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sm[wid][k] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0;
    for (int w = 0; w < ADJ_THREADS / 32; ++w) s += sm[w][threadIdx.x];
    out3[threadIdx.x] += s;
  }
  return a;
}

template <int PREC, int QH, int READ_ODD>
__global__ void __launch_bounds__(ADJ_THREADS, adj_minb<PREC>()) k_adj_local(Geo32 geo, PhysR<typename Store<PREC>::R> ph,
                                                           AdjParR<typename Store<PREC>::R> ap,
                                                           const typename Store<PREC>::S* __restrict__ h,
                                                           const typename Store<PREC>::S* __restrict__ g,
                                                           const typename Store<PREC>::PhiT* __restrict__ phi,
                                                           const typename Store<PREC>::R* __restrict__ lam_in,
                                                           const typename Store<PREC>::R* __restrict__ acc_in,
                                                           typename Store<PREC>::R* __restrict__ lam_out,
                                                           typename Store<PREC>::R* __restrict__ aux,
                                                           double* __restrict__ part) {
  static_assert(PREC != 2, "the adjoint runs on FP64 or FP32 storage");
  typedef typename Store<PREC>::R R;
  constexpr int QG = qg_of<QH>();   // D2Q9 with the 2-D phase field, else D3Q27
  constexpr int GR = (QG - 1) / 2;  // rest index of g
  const unsigned cell = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = cell < geo.N;
  R bM = 0, bXi = 0, bSig = 0;
  if (active) {
    const unsigned N = geo.N;
    CellOff o;
    cell_off(geo, cell, o);
    // ---------------- adjoints of the post-collision populations
    // Gathered first: they depend on lambda and the offsets only, so their
    // loads overlap those of the saved state, and the twenty sums they reduce
    // to are all that stays live through the forward recomputation (158 -> 128
    // registers at no bound; adjoint / forward on the 128x384x128 FP32 bubble,
    // 400 steps: 3.96 -> 3.43).
    // g: lambda+ of population i of this cell sits where streaming put it
    R b_al = 0, b_bx = 0, b_by = 0, b_bz = 0, b_Gxx = 0, b_Gyy = 0, b_Gzz = 0, b_Gxy = 0, b_Gyz = 0, b_Gxz = 0;
    const R* lg = lam_in + (unsigned)QH * N;
    b_al = (R)lq_w<QG>(GR) * lg[(unsigned)GR * N + cell];
#pragma unroll
    for (int i = 0; i < GR; ++i) {
      const int cx = q27_cx(lq_to27<QG>(i)), cy = q27_cy(lq_to27<QG>(i)), cz = q27_cz(lq_to27<QG>(i));
      const int oi = QG - 1 - i;
      // direction c (index i) went to x + c (slot i) or bounced into slot oi of x
      const R la = o.valid(cx, cy, cz) ? lg[(unsigned)i * N + cell + (unsigned)o.off(cx, cy, cz)]
                                       : lg[(unsigned)oi * N + cell];
      const R lb = o.valid(-cx, -cy, -cz) ? lg[(unsigned)oi * N + cell + (unsigned)o.off(-cx, -cy, -cz)]
                                          : lg[(unsigned)i * N + cell];
      const R w = (R)lq_w<QG>(i);
      const R S = w * (la + lb), D = w * (la - lb);
      b_al += S;
      if (cx) b_bx += cx > 0 ? D : -D;
      if (cy) b_by += cy > 0 ? D : -D;
      if (cz) b_bz += cz > 0 ? D : -D;
      if (cx) b_Gxx += S;
      if (cy) b_Gyy += S;
      if (cz) b_Gzz += S;
      if (cx && cy) b_Gxy += (cx * cy > 0) ? S : -S;
      if (cy && cz) b_Gyz += (cy * cz > 0) ? S : -S;
      if (cx && cz) b_Gxz += (cx * cz > 0) ? S : -S;
    }
    // h
    R c_al = (R)hq_w<QH>(hq_rest<QH>()) * (lam_in[(unsigned)hq_rest<QH>() * N + cell] + acc_in[cell]), c_bx = 0,
      c_by = 0, c_bz = 0;
    R c_Gxx = 0, c_Gyy = 0, c_Gzz = 0, c_Gxy = 0, c_Gyz = 0, c_Gxz = 0;
#pragma unroll
    for (int k = 0; k < hq_rest<QH>(); ++k) {
      const int cx = hq_cx<QH>(k), cy = hq_cy<QH>(k), cz = hq_cz<QH>(k);
      const int ok = QH - 1 - k;
      // the slot read and the cell holding it (whose acc belongs to every h slot)
      const bool va = o.valid(cx, cy, cz), vb = o.valid(-cx, -cy, -cz);
      const unsigned ya = va ? cell + (unsigned)o.off(cx, cy, cz) : cell;
      const unsigned yb = vb ? cell + (unsigned)o.off(-cx, -cy, -cz) : cell;
      const R la = lam_in[(va ? (unsigned)k : (unsigned)ok) * N + ya] + acc_in[ya];
      const R lb = lam_in[(vb ? (unsigned)ok : (unsigned)k) * N + yb] + acc_in[yb];
      const R w = (R)hq_w<QH>(k);
      const R S = w * (la + lb), D = w * (la - lb);
      c_al += S;
      if (cx) c_bx += cx > 0 ? D : -D;
      if (cy) c_by += cy > 0 ? D : -D;
      if (cz) c_bz += cz > 0 ? D : -D;
      if (cx) c_Gxx += S;
      if (cy) c_Gyy += S;
      if (cz) c_Gzz += S;
      if (cx && cy) c_Gxy += (cx * cy > 0) ? S : -S;
      if (cy && cz) c_Gyz += (cy * cz > 0) ? S : -S;
      if (cx && cz) c_Gxz += (cx * cz > 0) ? S : -S;
    }

    // ---------------- forward recomputation (as in k_step_mrt)
    const R pc = (R)phi[cell];
    R gx = 0, gy = 0, gz = 0, lap = 0;
#pragma unroll
    for (int i = 0; i < GR; ++i) {
      const int cx = q27_cx(lq_to27<QG>(i)), cy = q27_cy(lq_to27<QG>(i)), cz = q27_cz(lq_to27<QG>(i));
      const R a = (R)phi[cell + o.soff(cx, cy, cz)];
      const R b = (R)phi[cell + o.soff(-cx, -cy, -cz)];
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

    R pst = g[(unsigned)GR * N + cell], jx = 0, jy = 0, jz = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pyz = 0, pxz = 0;
#pragma unroll
    for (int i = 0; i < GR; ++i) {
      const int cx = q27_cx(lq_to27<QG>(i)), cy = q27_cy(lq_to27<QG>(i)), cz = q27_cz(lq_to27<QG>(i));
      R a, b;
      unsigned fa, fb;
      load_pair<PREC, READ_ODD>(g, N, cell, o, i, QG - 1 - i, cx, cy, cz, a, b, fa, fb);
      const R S = a + b, D = a - b;
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
    R phl = h[(unsigned)hq_rest<QH>() * N + cell], hjx = 0, hjy = 0, hjz = 0, hxx = 0, hyy = 0, hzz = 0, hxy = 0, hyz = 0, hxz = 0;
#pragma unroll
    for (int k = 0; k < hq_rest<QH>(); ++k) {
      const int cx = hq_cx<QH>(k), cy = hq_cy<QH>(k), cz = hq_cz<QH>(k);
      R a, b;
      unsigned fa, fb;
      load_pair<PREC, READ_ODD>(h, N, cell, o, k, QH - 1 - k, cx, cy, cz, a, b, fa, fb);
      const R S = a + b, D = a - b;
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

    const R drho = ph.drho;
    const R dtau = ph.dtau;
    const R rho = ph.rho_l + pc * drho;
    const R tau = ph.tau_l + pc * dtau;
    const R omega = (R)1 / tau;
    const R nu = (tau - (R)0.5) * (R)(1.0 / 3.0);
    const R beta = ph.beta, kappa = ph.kappa;
    const R dw = pc * (pc - (R)1) * (pc - (R)0.5);
    const R mu = (R)4 * beta * dw - kappa * lap;
    const R inv2rho = (R)0.5 / rho;
    const R cp = -pst * (R)(1.0 / 3.0) * drho;
    const R Gx = ph.gx, Gy = ph.gy, Gz = ph.gz;
    const R F0x = (mu + cp) * gx + rho * Gx, F0y = (mu + cp) * gy + rho * Gy, F0z = (mu + cp) * gz + rho * Gz;
    const R p3 = pst * (R)(1.0 / 3.0);
    const R u0x = jx + F0x * inv2rho, u0y = jy + F0y * inv2rho, u0z = jz + F0z * inv2rho;
    const R Nxx = pxx - p3 - u0x * u0x, Nyy = pyy - p3 - u0y * u0y, Nzz = pzz - p3 - u0z * u0z;
    const R Nxy = pxy - u0x * u0y, Nyz = pyz - u0y * u0z, Nxz = pxz - u0x * u0z;
    const R cm = (R)-3 * nu * omega * drho;
    const R NGx = Nxx * gx + Nxy * gy + Nxz * gz;
    const R NGy = Nxy * gx + Nyy * gy + Nyz * gz;
    const R NGz = Nxz * gx + Nyz * gy + Nzz * gz;
    const R Fx = F0x + cm * NGx, Fy = F0y + cm * NGy, Fz = F0z + cm * NGz;
    const R ux = jx + Fx * inv2rho, uy = jy + Fy * inv2rho, uz = jz + Fz * inv2rho;
    const R a2 = ((R)1 - omega) * (R)4.5;
    const R dxx = pxx - p3 - ux * ux, dyy = pyy - p3 - uy * uy;
    const R dzz = QG == 9 ? (R)0 : pzz - p3 - uz * uz;  // 2-D: the trace runs over x and y
    const R fr = (R)1.5 / rho;
    // phase field
    const R omp = ph.omega_phi;
    const R gn = sqrt(gx * gx + gy * gy + gz * gz);
    const R den = gn + (R)1e-6;
    const R theta = (R)4 * pc * ((R)1 - pc) * ph.inv_xi;
    const R sfac = (R)1 - (R)0.5 * omp;
    const R tn = theta / den * sfac;
    const R a1h = ((R)1 - omp) * (R)3, a2h = ((R)1 - omp) * (R)4.5;
    const R ph3 = phl * (R)(1.0 / 3.0);
    const R dhxx = hxx - ph3, dhyy = hyy - ph3, dhzz = QG == 9 ? (R)0 : hzz - ph3;

    // ---------------- reverse sweep of the local map
    // adjoint accumulators of the inputs
    R b_pst = 0, b_jx = 0, b_jy = 0, b_jz = 0, b_pxx = 0, b_pyy = 0, b_pzz = 0, b_pxy = 0, b_pyz = 0, b_pxz = 0;
    R b_phl = 0, b_hjx = 0, b_hjy = 0, b_hjz = 0, b_hxx = 0, b_hyy = 0, b_hzz = 0, b_hxy = 0, b_hyz = 0, b_hxz = 0;
    R b_pc = 0, b_gx = 0, b_gy = 0, b_gz = 0, b_lap = 0;
    // intermediates
    R b_ux = 0, b_uy = 0, b_uz = 0, b_Fx = 0, b_Fy = 0, b_Fz = 0, b_rho = 0, b_omega = 0;

    // g: al = pst - 1.5 uu - a2 (dxx + dyy + dzz) / 3 ; b = 3 u + fr F ;
    //    Gaa = 4.5 ua^2 + a2 daa ; Gab = 2 (4.5 - a2) ua ub + 2 a2 pab
    {
      R b_a2 = 0, b_dxx = 0, b_dyy = 0, b_dzz = 0, b_fr = 0;
      b_pst += b_al;
      b_ux += (R)-3 * ux * b_al;
      b_uy += (R)-3 * uy * b_al;
      b_uz += (R)-3 * uz * b_al;
      b_a2 += -b_al * (dxx + dyy + dzz) * (R)(1.0 / 3.0);
      const R btr = -b_al * a2 * (R)(1.0 / 3.0);
      b_dxx += btr;
      b_dyy += btr;
      b_dzz += btr;
      // b
      b_ux += (R)3 * b_bx;
      b_uy += (R)3 * b_by;
      b_uz += (R)3 * b_bz;
      b_Fx += fr * b_bx;
      b_Fy += fr * b_by;
      b_Fz += fr * b_bz;
      b_fr += Fx * b_bx + Fy * b_by + Fz * b_bz;
      // diagonal G
      b_ux += (R)9 * ux * b_Gxx;
      b_uy += (R)9 * uy * b_Gyy;
      b_uz += (R)9 * uz * b_Gzz;
      b_a2 += dxx * b_Gxx + dyy * b_Gyy + dzz * b_Gzz;
      b_dxx += a2 * b_Gxx;
      b_dyy += a2 * b_Gyy;
      b_dzz += a2 * b_Gzz;
      // off-diagonal G (stored with the factor 2)
      const R k2 = (R)2 * ((R)4.5 - a2);
      b_ux += k2 * (uy * b_Gxy + uz * b_Gxz);
      b_uy += k2 * (ux * b_Gxy + uz * b_Gyz);
      b_uz += k2 * (uy * b_Gyz + ux * b_Gxz);
      b_a2 += (R)2 * ((pxy - ux * uy) * b_Gxy + (pyz - uy * uz) * b_Gyz + (pxz - ux * uz) * b_Gxz);
      b_pxy += (R)2 * a2 * b_Gxy;
      b_pyz += (R)2 * a2 * b_Gyz;
      b_pxz += (R)2 * a2 * b_Gxz;
      if (QG == 9) b_dzz = 0;  // 2-D: d_zz is no variable
      // d_aa = p_aa - p3 - ua^2
      b_pxx += b_dxx;
      b_pyy += b_dyy;
      b_pzz += b_dzz;
      b_pst += -(b_dxx + b_dyy + b_dzz) * (R)(1.0 / 3.0);
      b_ux += (R)-2 * ux * b_dxx;
      b_uy += (R)-2 * uy * b_dyy;
      b_uz += (R)-2 * uz * b_dzz;
      b_rho += (R)-1.5 / (rho * rho) * b_fr;
      b_omega += (R)-4.5 * b_a2;
    }

    // h: al = phl - a2h (sum dh) / 3 ; b = (3 - a1h) phl u + a1h hj + tn grad ;
    //    Gaa = a2h dhaa ; Gab = 2 a2h hab
    {
      R b_a1h = 0, b_a2h = 0, b_tn = 0;
      const R sdh = dhxx + dhyy + dhzz;
      b_phl += c_al;
      b_a2h += -c_al * sdh * (R)(1.0 / 3.0);
      const R bsd = -c_al * a2h * (R)(1.0 / 3.0);
      b_hxx += bsd;
      b_hyy += bsd;
      b_hzz += bsd;
      b_phl += (QG == 9 ? (R)(-2.0 / 3.0) : (R)-1) * bsd;  // -1/3 from each diagonal term of the trace
      b_a2h += dhxx * c_Gxx + dhyy * c_Gyy + dhzz * c_Gzz;
      b_hxx += a2h * c_Gxx;
      b_hyy += a2h * c_Gyy;
      b_hzz += a2h * c_Gzz;
      b_phl += -a2h * (R)(1.0 / 3.0) * (c_Gxx + c_Gyy + c_Gzz);
      b_a2h += (R)2 * (hxy * c_Gxy + hyz * c_Gyz + hxz * c_Gxz);
      b_hxy += (R)2 * a2h * c_Gxy;
      b_hyz += (R)2 * a2h * c_Gyz;
      b_hxz += (R)2 * a2h * c_Gxz;
      const R k3 = (R)3 - a1h;
      b_phl += k3 * (ux * c_bx + uy * c_by + uz * c_bz);
      b_ux += k3 * phl * c_bx;
      b_uy += k3 * phl * c_by;
      b_uz += k3 * phl * c_bz;
      b_a1h += (hjx - phl * ux) * c_bx + (hjy - phl * uy) * c_by + (hjz - phl * uz) * c_bz;
      b_hjx += a1h * c_bx;
      b_hjy += a1h * c_by;
      b_hjz += a1h * c_bz;
      b_tn += gx * c_bx + gy * c_by + gz * c_bz;
      b_gx += tn * c_bx;
      b_gy += tn * c_by;
      b_gz += tn * c_bz;
      // tn = theta / den * sfac, den = |grad| + eps
      const R b_theta = sfac / den * b_tn;
      const R b_den = -theta * sfac / (den * den) * b_tn;
      const R b_sfac = theta / den * b_tn;
      if (gn > (R)0) {
        b_gx += gx / gn * b_den;
        b_gy += gy / gn * b_den;
        b_gz += gz / gn * b_den;
      }
      // theta = 4 pc (1 - pc) / xi
      b_pc += (R)4 * ((R)1 - (R)2 * pc) * ph.inv_xi * b_theta;
      const R b_invxi = (R)4 * pc * ((R)1 - pc) * b_theta;
      bXi += -b_invxi / ap.xi2;
      // omega_phi -> M
      const R b_omp = (R)-3 * b_a1h - (R)4.5 * b_a2h - (R)0.5 * b_sfac;
      bM += (R)-3 * omp * omp * b_omp;
    }

    // u = j + F inv2rho ; F = F0 + cm NG ; NG = N grad ; u0 = j + F0 inv2rho
    {
      R b_inv2rho = 0;
      b_jx += b_ux;
      b_jy += b_uy;
      b_jz += b_uz;
      b_Fx += inv2rho * b_ux;
      b_Fy += inv2rho * b_uy;
      b_Fz += inv2rho * b_uz;
      b_inv2rho += Fx * b_ux + Fy * b_uy + Fz * b_uz;
      // F = F0 + cm NG
      R b_F0x = b_Fx, b_F0y = b_Fy, b_F0z = b_Fz;
      const R b_cm = NGx * b_Fx + NGy * b_Fy + NGz * b_Fz;
      const R bNGx = cm * b_Fx, bNGy = cm * b_Fy, bNGz = cm * b_Fz;
      // NG_a = sum_b N_ab g_b (N symmetric)
      const R b_Nxx = bNGx * gx, b_Nyy = bNGy * gy, b_Nzz = bNGz * gz;
      const R b_Nxy = bNGx * gy + bNGy * gx, b_Nyz = bNGy * gz + bNGz * gy, b_Nxz = bNGx * gz + bNGz * gx;
      b_gx += Nxx * bNGx + Nxy * bNGy + Nxz * bNGz;
      b_gy += Nxy * bNGx + Nyy * bNGy + Nyz * bNGz;
      b_gz += Nxz * bNGx + Nyz * bNGy + Nzz * bNGz;
      // cm = -3 nu omega drho
      R b_nu = (R)-3 * omega * drho * b_cm;
      b_omega += (R)-3 * nu * drho * b_cm;
      // N_aa = p_aa - p3 - u0a^2 ; N_ab = p_ab - u0a u0b
      b_pxx += b_Nxx;
      b_pyy += b_Nyy;
      b_pzz += b_Nzz;
      b_pxy += b_Nxy;
      b_pyz += b_Nyz;
      b_pxz += b_Nxz;
      b_pst += -(b_Nxx + b_Nyy + b_Nzz) * (R)(1.0 / 3.0);
      const R b_u0x = (R)-2 * u0x * b_Nxx - u0y * b_Nxy - u0z * b_Nxz;
      const R b_u0y = (R)-2 * u0y * b_Nyy - u0x * b_Nxy - u0z * b_Nyz;
      const R b_u0z = (R)-2 * u0z * b_Nzz - u0y * b_Nyz - u0x * b_Nxz;
      // u0 = j + F0 inv2rho
      b_jx += b_u0x;
      b_jy += b_u0y;
      b_jz += b_u0z;
      b_F0x += inv2rho * b_u0x;
      b_F0y += inv2rho * b_u0y;
      b_F0z += inv2rho * b_u0z;
      b_inv2rho += F0x * b_u0x + F0y * b_u0y + F0z * b_u0z;
      // F0 = (mu + cp) grad + rho G
      const R b_mcp = gx * b_F0x + gy * b_F0y + gz * b_F0z;
      b_gx += (mu + cp) * b_F0x;
      b_gy += (mu + cp) * b_F0y;
      b_gz += (mu + cp) * b_F0z;
      b_rho += Gx * b_F0x + Gy * b_F0y + Gz * b_F0z;
      // cp = -pst drho / 3
      b_pst += -drho * (R)(1.0 / 3.0) * b_mcp;
      // mu = 4 beta dw(pc) - kappa lap
      b_pc += (R)4 * beta * ((R)3 * pc * pc - (R)3 * pc + (R)0.5) * b_mcp;
      b_lap += -kappa * b_mcp;
      const R b_beta = (R)4 * dw * b_mcp;
      const R b_kappa = -lap * b_mcp;
      // beta = 12 sigma / xi, kappa = 1.5 sigma xi
      bSig += ap.beta_sig * b_beta + ap.kappa_sig * b_kappa;
      bXi += ap.beta_xi * b_beta + ap.kappa_xi * b_kappa;
      // inv2rho = 0.5 / rho ; nu = (tau - 0.5) / 3 ; omega = 1 / tau
      b_rho += (R)-0.5 / (rho * rho) * b_inv2rho;
      R b_tau = b_nu * (R)(1.0 / 3.0) - omega * omega * b_omega;
      b_pc += dtau * b_tau + drho * b_rho;
    }

    // ---------------- adjoints of the local pre-collision populations
    R* og = lam_out + (unsigned)QH * N;
    og[(unsigned)GR * N + cell] = b_pst;
#pragma unroll
    for (int i = 0; i < GR; ++i) {
      const int cx = q27_cx(lq_to27<QG>(i)), cy = q27_cy(lq_to27<QG>(i)), cz = q27_cz(lq_to27<QG>(i));
      R E = b_pst;
      if (cx) E += b_pxx;
      if (cy) E += b_pyy;
      if (cz) E += b_pzz;
      if (cx && cy) E += (cx * cy > 0) ? b_pxy : -b_pxy;
      if (cy && cz) E += (cy * cz > 0) ? b_pyz : -b_pyz;
      if (cx && cz) E += (cx * cz > 0) ? b_pxz : -b_pxz;
      R L = 0;
      if (cx) L += cx > 0 ? b_jx : -b_jx;
      if (cy) L += cy > 0 ? b_jy : -b_jy;
      if (cz) L += cz > 0 ? b_jz : -b_jz;
      og[(unsigned)i * N + cell] = E + L;
      og[(unsigned)(QG - 1 - i) * N + cell] = E - L;
    }
    lam_out[(unsigned)hq_rest<QH>() * N + cell] = b_phl;
#pragma unroll
    for (int k = 0; k < hq_rest<QH>(); ++k) {
      const int cx = hq_cx<QH>(k), cy = hq_cy<QH>(k), cz = hq_cz<QH>(k);
      R E = b_phl;
      if (cx) E += b_hxx;
      if (cy) E += b_hyy;
      if (cz) E += b_hzz;
      if (cx && cy) E += (cx * cy > 0) ? b_hxy : -b_hxy;
      if (cy && cz) E += (cy * cz > 0) ? b_hyz : -b_hyz;
      if (cx && cz) E += (cx * cz > 0) ? b_hxz : -b_hxz;
      R L = 0;
      if (cx) L += cx > 0 ? b_hjx : -b_hjx;
      if (cy) L += cy > 0 ? b_hjy : -b_hjy;
      if (cz) L += cz > 0 ? b_hjz : -b_hjz;
      lam_out[(unsigned)k * N + cell] = E + L;
      lam_out[(unsigned)(QH - 1 - k) * N + cell] = E - L;
    }
    aux[0u * N + cell] = b_gx;
    aux[1u * N + cell] = b_gy;
    aux[2u * N + cell] = b_gz;
    aux[3u * N + cell] = b_lap;
    aux[4u * N + cell] = b_pc;
  }
  block_sum3_to<R>(bM, bXi, bSig, part + 3u * blockIdx.x);
}

// Transpose of the phi stencil: acc(x) = adjoint of phi(x) = aux_pc(x) -
// 6 (1 - w_0) aux_lap(x) + sum over (y, c) whose stencil read x of
// w_c (6 aux_lap(y) + 3 c . aux_grad(y)), plus W(x) at an observation step.
//
// On a periodic lattice the reader of x in direction c is y = x - c.  The
// forward stencil mirrors across a no-slip face (a read beyond the face cell
// returns the face cell itself), so a face cell x also receives, for each
// direction c that leaves through the face, the term of its own reading
// cell y = x - c with the normal component of c reversed.  Both cases become
// one plain gather over a halo one cell wide whose ghost beyond a face holds
// the face cell's values with the normal gradient component negated (an even
// reflection of aux_lap and of the tangential components, an odd one of the
// normal component, about the face cell): the ghost's term for c then equals
// the mirrored term for c with its normal component reversed, the weights
// being equal.
//
// Blocks of ZM_TX x ZM_TY threads march zc planes along z and keep three
// planes of the four gathered aux fields (tile plus halo) in shared memory.
template <typename R, int QG>
__global__ void __launch_bounds__(ZM_TX * ZM_TY) k_adj_phi(Geo32 geo, const R* __restrict__ aux,
                                                           R* __restrict__ acc_out, const double* __restrict__ W,
                                                           int zc) {
  constexpr int NT = ZM_TX * ZM_TY;
  constexpr int PW = ZM_TX + 2, PH = ZM_TY + 2, PS = PW * PH;
  __shared__ R ring[3][4][PS];
  const unsigned N = geo.N;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * ZM_TX + tx;
  const int x0 = blockIdx.x * ZM_TX, y0 = blockIdx.y * ZM_TY;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, (int)geo.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < (int)geo.nx && y < (int)geo.ny;

  // source coordinate of a (possibly ghost) position along one axis, and
  // whether the normal component flips (ghost beyond a no-slip face)
  auto src = [](int p, int n, int wall, bool& flip) -> unsigned {
    flip = false;
    if (wall) {
      if (p < 0) {
        flip = true;
        return 0u;
      }
      if (p >= n) {
        flip = p == n;
        return (unsigned)(n - 1);
      }
      return (unsigned)p;
    }
    return (unsigned)(((p % n) + n) % n);
  };

  // The four aux fields of plane zp at this thread's ring positions (tid and
  // tid + NT) into registers, then into a ring slot: a plane's loads are
  // issued one plane ahead, so they are in flight over the barrier and the
  // sums of the plane before.
  constexpr int NPOS = (PS + NT - 1) / NT;
  R pre[NPOS][4];
  auto load_plane = [&](int zp) {
    bool fz;
    const unsigned sz = src(zp, (int)geo.nz, geo.wall[2], fz);
#pragma unroll
    for (int k = 0; k < NPOS; ++k) {
      const int r = tid + k * NT;
      if (r < PS) {
        const int i = r % PW, j = r / PW;
        bool fx, fy;
        const unsigned sx = src(x0 - 1 + i, (int)geo.nx, geo.wall[0], fx);
        const unsigned sy = src(y0 - 1 + j, (int)geo.ny, geo.wall[1], fy);
        const unsigned c = sx + geo.nx * (sy + geo.ny * sz);
        const R a0 = aux[c], a1 = aux[N + c], a2 = aux[2u * N + c];
        pre[k][0] = fx ? -a0 : a0;
        pre[k][1] = fy ? -a1 : a1;
        pre[k][2] = fz ? -a2 : a2;
        pre[k][3] = aux[3u * N + c];
      }
    }
  };
  auto store_plane = [&](int slot) {
#pragma unroll
    for (int k = 0; k < NPOS; ++k) {
      const int r = tid + k * NT;
      if (r < PS) {
#pragma unroll
        for (int f = 0; f < 4; ++f) ring[slot][f][r] = pre[k][f];
      }
    }
  };
  auto fill = [&](int zp, int slot) {
    load_plane(zp);
    store_plane(slot);
  };

  // The weights factor per axis, w(o) = w1(o_x) w1(o_y) w1(o_z) with w1 = 1/6,
  // 2/3, 1/6 (D2Q9: w1(o_x) w1(o_y)), so with o = -c the sum is
  //   acc = aux_pc - 6 aux_lap(x) + 6 sum_o w(o) lap(x + o)
  //         - 3 sum_o w(o) (o_x g_x + o_y g_y + o_z g_z)(x + o),
  // formed as four 3x3 sums in each plane (lap with w1 w1, g_x with o_x w1 w1,
  // g_y with w1 o_y w1, g_z with w1 w1) and their combination over the planes
  // z - 1, z, z + 1 (weights w1, or o_z w1 for g_z), kept in registers as the
  // march goes: 30 shared-memory reads per cell instead of 80.
  constexpr bool FLAT2 = QG == 9;
  const R w1e = (R)(1.0 / 6.0), w1c = (R)(2.0 / 3.0);
  const int i0 = (ty + 1) * PW + (tx + 1);
  auto plane_sums = [&](int slot, R out[4]) {
    const R* L = ring[slot][3];
    const R* GX = ring[slot][0];
    const R* GY = ring[slot][1];
    const R* GZ = ring[slot][2];
    // rows y - 1, y, y + 1 of lap and g_z, smoothed along x (w1); g_x differenced along x
    R la[3], gz[3], gx[3], gyr[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int r = i0 + (j - 1) * PW;
      la[j] = w1e * (L[r - 1] + L[r + 1]) + w1c * L[r];
      gz[j] = w1e * (GZ[r - 1] + GZ[r + 1]) + w1c * GZ[r];
      gx[j] = w1e * (GX[r + 1] - GX[r - 1]);
      gyr[j] = (j == 1) ? (R)0 : w1e * (GY[r - 1] + GY[r + 1]) + w1c * GY[r];
    }
    out[0] = w1e * (la[0] + la[2]) + w1c * la[1];      // lap, w1 w1
    out[1] = w1e * (gx[0] + gx[2]) + w1c * gx[1];      // g_x, o_x w1 . w1
    out[2] = w1e * (gyr[2] - gyr[0]);                  // g_y, w1 . o_y w1
    out[3] = w1e * (gz[0] + gz[2]) + w1c * gz[1];      // g_z, w1 w1
  };

  fill(z0 - 1, 0);
  fill(z0, 1);
  if (!FLAT2) load_plane(z0 + 1);
  __syncthreads();
  R Sm[4] = {0, 0, 0, 0}, S0[4], Sp[4];
  if (!FLAT2) plane_sums(0, Sm);
  plane_sums(1, S0);
  for (int z = z0; z < z1; ++z) {
    const int b = z - (z0 - 1);
    // plane z + 1 (loaded one plane ago) goes into the slot of plane z - 2,
    // whose sums were taken two planes ago (barriers since); plane z's slot
    // stays for its centre value; plane z + 2's loads go out now
    if (!FLAT2) {
      store_plane((b + 1) % 3);
      if (z + 2 <= z1) load_plane(z + 2);
    }
    __syncthreads();
    if (!FLAT2) plane_sums((b + 1) % 3, Sp);
    if (active) {
      const unsigned cell = (unsigned)x + geo.nx * ((unsigned)y + geo.ny * (unsigned)z);
      R sl, sx, sy, sz;
      if (FLAT2) {
        sl = S0[0];
        sx = S0[1];
        sy = S0[2];
        sz = 0;
      } else {
        sl = w1e * (Sm[0] + Sp[0]) + w1c * S0[0];
        sx = w1e * (Sm[1] + Sp[1]) + w1c * S0[1];
        sy = w1e * (Sm[2] + Sp[2]) + w1c * S0[2];
        sz = w1e * (Sp[3] - Sm[3]);
      }
      R acc = aux[4u * N + cell] - (R)6 * ring[b % 3][3][i0] + (R)6 * sl - (R)3 * (sx + sy + sz);
      if (W) acc += (R)W[cell];
      acc_out[cell] = acc;
    }
    if (!FLAT2) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Sm[k] = S0[k];
        S0[k] = Sp[k];
      }
    }
  }
}

// dot = sum_x W(x) phi(x) in FP64 (per-block partials, fixed order).
template <typename PhiT>
__global__ void __launch_bounds__(256) k_dot(unsigned N, const double* __restrict__ W, const PhiT* __restrict__ phi,
                                             double* __restrict__ part) {
  double s = 0;
  for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
    s += W[c] * (double)phi[c];
  __shared__ double sm[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < 8; ++w) t += sm[w];
    part[blockIdx.x] = t;
  }
}

// Sum of n partials of stride `stride` (component k) into out[k], one warp.
static __global__ void k_sum_parts(const double* __restrict__ part, int n, int stride, double* __restrict__ out) {
  const int k = blockIdx.x;
  double s = 0;
  for (int b = threadIdx.x; b < n; b += 32) s += part[(size_t)b * stride + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[k] += s;
}

}  // namespace pfl
