// Plain FP64 CPU oracle of the conservative Allen-Cahn phase-field LBM (PFLBM).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
// calls this file; only the tests, the smoke check and the CPU-baseline leg of
// the benchmark load it.  It shares no code, header or table with the CUDA path.
//
// What it computes (section "Conservative Allen-Cahn model" of the paper, and
// the LBM basics of section "The lattice Boltzmann method"):
//   * phase-field PDFs h_i on D3Q15, hydrodynamic PDFs g_i on D3Q27;
//   * phi = sum_i h_i (zeroth moment), p* = sum_i g_i (normalised pressure);
//   * weighted-orthogonal MRT collision  Omega = M^-1 S M (f^eq - f)  (Eq. mrt),
//     with the moment matrices built here by Gram-Schmidt under the lattice
//     weights from a list of monomials, graded by polynomial degree;
//   * Guo forcing applied in moment space, (I - S/2) M F;
//   * forces F = F_s + F_b + F_p + F_mu with F_s = mu_phi grad(phi), F_b = rho g,
//     F_p = -p* c_s^2 (rho_H - rho_L) grad(phi),
//     F_mu = nu (rho_H - rho_L) [grad u + grad u^T] . grad(phi), the strain rate
//     taken from the non-equilibrium second moment of g (no finite differences
//     on u);
//   * rho(phi) and tau(phi) linear interpolation between the phases;
//   * conservative Allen-Cahn forcing F^phi = 4 phi (1 - phi) / xi * n;
//   * streaming with periodic wrap or halfway bounce-back at no-slip faces.
//
// Readings where the paper is silent or garbled:
//   tau_phi = M / c_s^2 is the shifted relaxation time, omega_phi = 1/(3M + 1/2);
//   mu_phi = 4 beta phi (phi - 1)(phi - 1/2) - kappa lap(phi), beta = 12 sigma / xi,
//     kappa = 3 sigma xi / 2;
//   grad/laplacian of phi: D3Q27-weighted central stencil, phi mirrored at walls;
//   h^eq_i = w_i phi (1 + c_i.u / c_s^2);  h source S_i = w_i c_i . (F^phi);
//   g source G_i = w_i c_i . F / (rho c_s^2);  u = sum c g + F / (2 rho);
//   F_mu uses the non-equilibrium part relative to g^eq(p*, u0) with
//     u0 = sum c g + (F_s + F_b + F_p) / (2 rho);
//   rates: g -- degree 2 at omega(phi), degree >= 3 at 1; h -- degrees 1 and 2
//     at omega_phi, degree >= 3 at 1; conserved moments at 0 / 1 (irrelevant);
//   n = grad(phi) / (|grad(phi)| + 1e-6): the regularisation sits far below the
//     gradients of the interface region and far above the rounding noise of
//     the stencil, so that n stays well conditioned where grad(phi) -> 0.
//
// Schedule per step: both collisions use phi^t and its stencil, u^t from g in
// the same cell; then both sets stream; then phi^{t+1} = sum h.  A sequential
// order (phase field first, the hydrodynamics at phi^{t+1}) is kept as an
// option for studies of how much that reading matters.
//
// Built with -O2 -ffp-contract=off so the arithmetic is plain IEEE FP64.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double CS2 = 1.0 / 3.0;

// ------------------------------------------------------------ dual numbers --
// Forward-mode differentiation (dual numbers, Wengert 1964): a value and its
// derivative with respect to one chosen parameter, carried through every
// operation by the chain rule.  The simulation below is written once for a
// scalar type T; T = double is the oracle, T = Dual gives the exact
// derivative of any result with respect to M, xi or sigma (the tangent of the
// same arithmetic, no finite-difference truncation).
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
inline Dual& operator-=(Dual& a, Dual b) { return a = a - b; }
inline Dual& operator*=(Dual& a, Dual b) { return a = a * b; }
inline Dual& operator/=(Dual& a, Dual b) { return a = a / b; }
inline Dual sqrt(Dual a) {
  const double r = std::sqrt(a.v);
  return Dual(r, a.v > 0 ? a.d / (2.0 * r) : 0.0);
}
inline double value(double a) { return a; }
inline double value(Dual a) { return a.v; }
inline double deriv(double) { return 0.0; }
inline double deriv(Dual a) { return a.d; }

// ---------------------------------------------------------------- lattices --
struct Lattice {
  int q = 0;
  std::vector<int> c;        // q x 3
  std::vector<double> w;     // q
  std::vector<int> opp;      // q
  std::vector<int> degree;   // q, polynomial degree of moment k
  std::vector<double> M;     // q x q, row k = moment polynomial k at c_i
  std::vector<double> Minv;  // q x q
};

// Canonical velocity order: loop cz, cy, cx over -1, 0, 1 (cx fastest) and
// keep the members of the set.  D3Q27 keeps all, D3Q15 keeps |c|^2 in {0,1,3},
// D2Q9 keeps cz = 0 (weights 4/9, 1/9, 1/36).
void make_velocities(Lattice& L, bool q15, bool q9 = false) {
  L.c.clear();
  L.w.clear();
  for (int cz = -1; cz <= 1; ++cz)
    for (int cy = -1; cy <= 1; ++cy)
      for (int cx = -1; cx <= 1; ++cx) {
        int n2 = cx * cx + cy * cy + cz * cz;
        double w;
        if (q9) {
          if (cz != 0) continue;
          w = (n2 == 0) ? 4.0 / 9.0 : (n2 == 1) ? 1.0 / 9.0 : 1.0 / 36.0;
        } else if (q15) {
          if (n2 == 2) continue;
          w = (n2 == 0) ? 2.0 / 9.0 : (n2 == 1) ? 1.0 / 9.0 : 1.0 / 72.0;
        } else {
          w = (n2 == 0) ? 8.0 / 27.0 : (n2 == 1) ? 2.0 / 27.0 : (n2 == 2) ? 1.0 / 54.0 : 1.0 / 216.0;
        }
        L.c.push_back(cx);
        L.c.push_back(cy);
        L.c.push_back(cz);
        L.w.push_back(w);
      }
  L.q = (int)L.w.size();
  L.opp.assign(L.q, -1);
  for (int i = 0; i < L.q; ++i)
    for (int j = 0; j < L.q; ++j)
      if (L.c[3 * j] == -L.c[3 * i] && L.c[3 * j + 1] == -L.c[3 * i + 1] && L.c[3 * j + 2] == -L.c[3 * i + 2])
        L.opp[i] = j;
}

// Monomials x^a y^b z^c, listed by increasing degree.  Gram-Schmidt under
// <u, v> = sum_i w_i u(c_i) v(c_i) turns them into weighted-orthogonal moment
// polynomials; M^-1 = W M^T N^-1 with N_k = <P_k, P_k>.
void build_moments(Lattice& L, const std::vector<int>& mono /* triples a,b,c */) {
  const int q = L.q;
  std::vector<double> P((size_t)q * q);
  L.degree.assign(q, 0);
  for (int k = 0; k < q; ++k) {
    int a = mono[3 * k], b = mono[3 * k + 1], cc = mono[3 * k + 2];
    L.degree[k] = a + b + cc;
    for (int i = 0; i < q; ++i)
      P[(size_t)k * q + i] = std::pow((double)L.c[3 * i], a) * std::pow((double)L.c[3 * i + 1], b) *
                             std::pow((double)L.c[3 * i + 2], cc);
  }
  for (int k = 0; k < q; ++k) {
    for (int j = 0; j < k; ++j) {
      double num = 0, den = 0;
      for (int i = 0; i < q; ++i) {
        num += L.w[i] * P[(size_t)k * q + i] * P[(size_t)j * q + i];
        den += L.w[i] * P[(size_t)j * q + i] * P[(size_t)j * q + i];
      }
      for (int i = 0; i < q; ++i) P[(size_t)k * q + i] -= num / den * P[(size_t)j * q + i];
    }
  }
  L.M = P;
  L.Minv.assign((size_t)q * q, 0.0);
  for (int k = 0; k < q; ++k) {
    double nk = 0;
    for (int i = 0; i < q; ++i) nk += L.w[i] * P[(size_t)k * q + i] * P[(size_t)k * q + i];
    for (int i = 0; i < q; ++i) L.Minv[(size_t)i * q + k] = L.w[i] * P[(size_t)k * q + i] / nk;
  }
}

Lattice make_d3q27() {
  Lattice L;
  make_velocities(L, false);
  std::vector<int> mono;
  for (int deg = 0; deg <= 6; ++deg)
    for (int a = 0; a <= 2; ++a)
      for (int b = 0; b <= 2; ++b)
        for (int cc = 0; cc <= 2; ++cc)
          if (a + b + cc == deg) {
            mono.push_back(a);
            mono.push_back(b);
            mono.push_back(cc);
          }
  build_moments(L, mono);
  return L;
}

Lattice make_d3q15() {
  Lattice L;
  make_velocities(L, true);
  // degree 0..2 complete; degree 3: xyz, x y^2, y z^2, z x^2; degree 4: x^2 y^2.
  const int m[15][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0},
                        {0, 1, 1}, {1, 0, 1}, {1, 1, 1}, {1, 2, 0}, {0, 1, 2}, {2, 0, 1}, {2, 2, 0}};
  std::vector<int> mono;
  for (auto& r : m) {
    mono.push_back(r[0]);
    mono.push_back(r[1]);
    mono.push_back(r[2]);
  }
  build_moments(L, mono);
  return L;
}

Lattice make_d2q9() {
  Lattice L;
  make_velocities(L, false, true);
  std::vector<int> mono;  // x^a y^b, a, b <= 2, by degree
  for (int deg = 0; deg <= 4; ++deg)
    for (int a = 0; a <= 2; ++a)
      for (int b = 0; b <= 2; ++b)
        if (a + b == deg) {
          mono.push_back(a);
          mono.push_back(b);
          mono.push_back(0);
        }
  build_moments(L, mono);
  return L;
}

const Lattice& Q9() {
  static Lattice L = make_d2q9();
  return L;
}
const Lattice& Q27() {
  static Lattice L = make_d3q27();
  return L;
}
const Lattice& Q15() {
  static Lattice L = make_d3q15();
  return L;
}

// ------------------------------------------------------------------ model --
enum { COLL_MRT = 0, COLL_BGK = 1, COLL_MRT_ALL_EQUAL = 2 };

// Order of the two collisions within a step (the paper does not state it).
// CONCURRENT: both collisions at t use phi^t, its stencil and u^t; then both
// sets stream; then phi^{t+1} = sum h.  SEQUENTIAL (for sensitivity studies
// of that reading only): the phase field goes first -- h collides with phi^t
// and u^t, streams, phi^{t+1} = sum h -- and the hydrodynamic collision then
// takes phi^{t+1} and its stencil (rho, tau, every force) with g^t.
enum { SCHED_CONCURRENT = 0, SCHED_SEQUENTIAL = 1 };

struct Params {
  int nx, ny, nz;
  int bc[6];  // -x,+x,-y,+y,-z,+z : 0 periodic, 1 no-slip
  int collision;
  int qh;     // phase-field lattice: 15 (D3Q15), 27 (D3Q27) or 9 (D2Q9, with D2Q9 for g)
  int schedule;  // SCHED_CONCURRENT (the reading used throughout) or SCHED_SEQUENTIAL
  double rho_h, rho_l, nu_h, nu_l, sigma, mobility, xi, g[3];
};

template <typename T>
struct Sim {
  Params P;
  T sigma, mobility, xi;  // P's values, as T (seeded for a derivative)
  long N;
  std::vector<T> h, g, hn, gn, phi;  // populations SoA [i][cell]
  std::vector<unsigned char> solid;  // solid cells (empty: none)
  long step = 0;
};

inline long cell_index(const Params& P, int x, int y, int z) { return x + (long)P.nx * (y + (long)P.ny * z); }

// Neighbour coordinate along one axis; returns false when the link leaves the
// domain through a no-slip face.
inline bool neighbour(int x, int d, int n, int bc_lo, int bc_hi, int& out) {
  int t = x + d;
  if (t < 0) {
    if (bc_lo == 1) return false;
    t += n;
  } else if (t >= n) {
    if (bc_hi == 1) return false;
    t -= n;
  }
  out = t;
  return true;
}

// Index of the cell used for the phi stencil: periodic wrap, or mirror
// (phi outside a wall equals phi in the adjacent cell).
inline int stencil_coord(int x, int d, int n, int bc_lo, int bc_hi) {
  int t = x + d;
  if (t < 0) t = (bc_lo == 1) ? 0 : t + n;
  if (t >= n) t = (bc_hi == 1) ? n - 1 : t - n;
  return t;
}

template <typename T>
struct CellState {
  T phi, gradphi[3], lapphi, rho, tau, omega, nu, mu, pstar, j[3], F[3], u[3];
  T Fs[3], Fb[3], Fp[3], Fmu[3];
};

// The hydrodynamic lattice: D2Q9 with the 2-D phase field, else D3Q27.
const Lattice& g_lattice(const Params& P) { return P.qh == 9 ? Q9() : Q27(); }
const Lattice& h_lattice(const Params& P) { return P.qh == 27 ? Q27() : (P.qh == 9 ? Q9() : Q15()); }

template <typename T>
void geq_of(const Lattice& L, T pstar, const T u[3], T* out) {
  T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < L.q; ++i) {
    T cu = L.c[3 * i] * u[0] + L.c[3 * i + 1] * u[1] + L.c[3 * i + 2] * u[2];
    out[i] = L.w[i] * (pstar + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2));
  }
}

template <typename T>
T rate_g(const Params& P, int degree, T omega) {
  if (P.collision != COLL_MRT) return omega;
  if (degree == 0) return 0.0;
  if (degree == 1) return 1.0;
  if (degree == 2) return omega;
  return 1.0;
}

template <typename T>
T rate_h(const Params& P, int degree, T omega_phi) {
  if (P.collision != COLL_MRT) return omega_phi;
  if (degree == 0) return 0.0;
  if (degree <= 2) return omega_phi;
  return 1.0;
}

// Collision in moment space, Eq. (mrt) plus Guo forcing in collision space:
//   f+ = f + M^-1 [ S M (f^eq - f) + (I - S/2) M src ].
template <typename T>
void mrt_collide(const Lattice& L, const T* f, const T* feq, const T* src, const T* s, T* out) {
  const int q = L.q;
  T r[27];
  for (int k = 0; k < q; ++k) {
    T d = 0, ms = 0;
    for (int i = 0; i < q; ++i) {
      d += L.M[(size_t)k * q + i] * (feq[i] - f[i]);
      ms += L.M[(size_t)k * q + i] * src[i];
    }
    r[k] = s[k] * d + (1.0 - 0.5 * s[k]) * ms;
  }
  for (int i = 0; i < q; ++i) {
    T v = 0;
    for (int k = 0; k < q; ++k) v += L.Minv[(size_t)i * q + k] * r[k];
    out[i] = f[i] + v;
  }
}

// v = M^-1 S M d  (the relaxed non-equilibrium part).
template <typename T>
void mrt_relax(const Lattice& L, const T* d, const T* s, T* out) {
  const int q = L.q;
  T r[27];
  for (int k = 0; k < q; ++k) {
    T m = 0;
    for (int i = 0; i < q; ++i) m += L.M[(size_t)k * q + i] * d[i];
    r[k] = s[k] * m;
  }
  for (int i = 0; i < q; ++i) {
    T v = 0;
    for (int k = 0; k < q; ++k) v += L.Minv[(size_t)i * q + k] * r[k];
    out[i] = v;
  }
}

// Macroscopic state of one cell at the current time level: stencil, forces
// and velocity (steps before the collision).  Needs phi of the neighbours.
template <typename T>
void cell_macro(const Sim<T>& S, int x, int y, int z, const T* gcell, CellState<T>& cs) {
  const Params& P = S.P;
  const Lattice& L27 = g_lattice(P);  // also the stencil lattice
  long c0 = cell_index(P, x, y, z);
  cs.phi = S.phi[c0];
  cs.gradphi[0] = cs.gradphi[1] = cs.gradphi[2] = 0;
  cs.lapphi = 0;
  for (int i = 0; i < L27.q; ++i) {
    int xs = stencil_coord(x, L27.c[3 * i], P.nx, P.bc[0], P.bc[1]);
    int ys = stencil_coord(y, L27.c[3 * i + 1], P.ny, P.bc[2], P.bc[3]);
    int zs = stencil_coord(z, L27.c[3 * i + 2], P.nz, P.bc[4], P.bc[5]);
    const long cn = cell_index(P, xs, ys, zs);
    // a solid neighbour reads as this cell (neutral wetting)
    T pn = (!S.solid.empty() && S.solid[cn]) ? cs.phi : S.phi[cn];
    for (int a = 0; a < 3; ++a) cs.gradphi[a] += L27.w[i] * L27.c[3 * i + a] * pn;
    cs.lapphi += L27.w[i] * (pn - cs.phi);
  }
  for (int a = 0; a < 3; ++a) cs.gradphi[a] /= CS2;
  cs.lapphi *= 2.0 / CS2;

  const double phiL = 0.0, phiH = 1.0, phi0 = 0.5;
  double tauH = P.nu_h / CS2 + 0.5, tauL = P.nu_l / CS2 + 0.5;
  cs.rho = P.rho_l + (cs.phi - phiL) * (P.rho_h - P.rho_l);
  cs.tau = tauL + (cs.phi - phiL) * (tauH - tauL);
  cs.omega = 1.0 / cs.tau;
  cs.nu = CS2 * (cs.tau - 0.5);
  T beta = 12.0 * S.sigma / S.xi, kappa = 1.5 * S.sigma * S.xi;
  cs.mu = 4.0 * beta * (cs.phi - phiL) * (cs.phi - phiH) * (cs.phi - phi0) - kappa * cs.lapphi;

  cs.pstar = 0;
  cs.j[0] = cs.j[1] = cs.j[2] = 0;
  for (int i = 0; i < L27.q; ++i) {
    cs.pstar += gcell[i];
    for (int a = 0; a < 3; ++a) cs.j[a] += L27.c[3 * i + a] * gcell[i];
  }
  double drho = P.rho_h - P.rho_l;
  T u0[3];
  for (int a = 0; a < 3; ++a) {
    cs.Fs[a] = cs.mu * cs.gradphi[a];
    cs.Fb[a] = cs.rho * P.g[a];
    cs.Fp[a] = -cs.pstar * CS2 * drho * cs.gradphi[a];
    u0[a] = cs.j[a] + (cs.Fs[a] + cs.Fb[a] + cs.Fp[a]) / (2.0 * cs.rho);
  }
  // Viscous force from the non-equilibrium moments, M^-1 S M (g - g^eq(p*, u0)).
  T geq0[27], dneq[27], relaxed[27], s[27];
  geq_of(L27, cs.pstar, u0, geq0);
  for (int k = 0; k < L27.q; ++k) s[k] = rate_g(P, L27.degree[k], cs.omega);
  for (int i = 0; i < L27.q; ++i) dneq[i] = gcell[i] - geq0[i];
  mrt_relax(L27, dneq, s, relaxed);
  T Pi[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int i = 0; i < L27.q; ++i)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Pi[a][b] += L27.c[3 * i + a] * L27.c[3 * i + b] * relaxed[i];
  for (int a = 0; a < 3; ++a) {
    T acc = 0;
    for (int b = 0; b < 3; ++b) acc += Pi[a][b] * cs.gradphi[b];
    // [grad u + grad u^T] ~= -(1/c_s^2) (M^-1 S M g^neq)_2
    cs.Fmu[a] = cs.nu * drho * (-acc / CS2);
  }
  for (int a = 0; a < 3; ++a) {
    cs.F[a] = cs.Fs[a] + cs.Fb[a] + cs.Fp[a] + cs.Fmu[a];
    cs.u[a] = cs.j[a] + cs.F[a] / (2.0 * cs.rho);
  }
}

template <typename T>
void compute_phi(Sim<T>& S) {
  const Lattice& LH = h_lattice(S.P);
  for (long c = 0; c < S.N; ++c) {
    T s = 0;
    for (int i = 0; i < LH.q; ++i) s += S.h[(size_t)i * S.N + c];
    S.phi[c] = s;
  }
}

// Hydrodynamic collision of cell (x, y, z) from its macroscopic state cs and
// populations gc, pushed into S.gn (periodic wrap or halfway bounce-back).
template <typename T>
void g_update(Sim<T>& S, int x, int y, int z, const CellState<T>& cs, const T* gc) {
  const Params& P = S.P;
  const Lattice& L27 = g_lattice(P);
  const long N = S.N;
  const long c0 = cell_index(P, x, y, z);
  T geq[27], G[27], gpost[27], s27[27];
  geq_of(L27, cs.pstar, cs.u, geq);
  for (int i = 0; i < L27.q; ++i) {
    T cF = L27.c[3 * i] * cs.F[0] + L27.c[3 * i + 1] * cs.F[1] + L27.c[3 * i + 2] * cs.F[2];
    G[i] = L27.w[i] * cF / (CS2 * cs.rho);
  }
  if (P.collision == COLL_BGK) {
    for (int i = 0; i < L27.q; ++i)
      gpost[i] = gc[i] - cs.omega * (gc[i] - geq[i]) + (1.0 - 0.5 * cs.omega) * G[i];
  } else {
    for (int k = 0; k < L27.q; ++k) s27[k] = rate_g(P, L27.degree[k], cs.omega);
    mrt_collide(L27, gc, geq, G, s27, gpost);
  }
  for (int i = 0; i < L27.q; ++i) {
    int xt, yt, zt;
    bool ok = neighbour(x, L27.c[3 * i], P.nx, P.bc[0], P.bc[1], xt) &&
              neighbour(y, L27.c[3 * i + 1], P.ny, P.bc[2], P.bc[3], yt) &&
              neighbour(z, L27.c[3 * i + 2], P.nz, P.bc[4], P.bc[5], zt);
    if (ok && !S.solid.empty() && S.solid[cell_index(P, xt, yt, zt)]) ok = false;  // bounce at a solid cell
    if (ok)
      S.gn[(size_t)i * N + cell_index(P, xt, yt, zt)] = gpost[i];
    else
      S.gn[(size_t)L27.opp[i] * N + c0] = gpost[i];
  }
}

// Phase-field collision of cell (x, y, z) from cs (phi, its gradient and u)
// and populations hc, pushed into S.hn.
template <typename T>
void h_update(Sim<T>& S, int x, int y, int z, const CellState<T>& cs, const T* hc) {
  using std::sqrt;
  const Params& P = S.P;
  const Lattice& LH = h_lattice(P);  // phase-field lattice
  const long N = S.N;
  const long c0 = cell_index(P, x, y, z);
  const T omega_phi = 1.0 / (S.mobility / CS2 + 0.5);
  T gnorm = sqrt(cs.gradphi[0] * cs.gradphi[0] + cs.gradphi[1] * cs.gradphi[1] + cs.gradphi[2] * cs.gradphi[2]);
  T n[3];
  for (int a = 0; a < 3; ++a) n[a] = cs.gradphi[a] / (gnorm + 1e-6);
  T theta = 4.0 * cs.phi * (1.0 - cs.phi) / S.xi;
  T heq[27], Sh[27], hpost[27], sh_rates[27];
  for (int i = 0; i < LH.q; ++i) {
    T cu = LH.c[3 * i] * cs.u[0] + LH.c[3 * i + 1] * cs.u[1] + LH.c[3 * i + 2] * cs.u[2];
    T cn = LH.c[3 * i] * n[0] + LH.c[3 * i + 1] * n[1] + LH.c[3 * i + 2] * n[2];
    heq[i] = LH.w[i] * cs.phi * (1.0 + cu / CS2);
    Sh[i] = LH.w[i] * theta * cn;
  }
  if (P.collision == COLL_BGK) {
    for (int i = 0; i < LH.q; ++i)
      hpost[i] = hc[i] - omega_phi * (hc[i] - heq[i]) + (1.0 - 0.5 * omega_phi) * Sh[i];
  } else {
    for (int k = 0; k < LH.q; ++k) sh_rates[k] = rate_h(P, LH.degree[k], omega_phi);
    mrt_collide(LH, hc, heq, Sh, sh_rates, hpost);
  }
  for (int i = 0; i < LH.q; ++i) {
    int xt, yt, zt;
    bool ok = neighbour(x, LH.c[3 * i], P.nx, P.bc[0], P.bc[1], xt) &&
              neighbour(y, LH.c[3 * i + 1], P.ny, P.bc[2], P.bc[3], yt) &&
              neighbour(z, LH.c[3 * i + 2], P.nz, P.bc[4], P.bc[5], zt);
    if (ok && !S.solid.empty() && S.solid[cell_index(P, xt, yt, zt)]) ok = false;
    if (ok)
      S.hn[(size_t)i * N + cell_index(P, xt, yt, zt)] = hpost[i];
    else
      S.hn[(size_t)LH.opp[i] * N + c0] = hpost[i];
  }
}

// One time step in the order of P.schedule.
template <typename T>
void do_step(Sim<T>& S) {
  const Params& P = S.P;
  const Lattice& L27 = g_lattice(P);
  const Lattice& LH = h_lattice(P);
  const long N = S.N;
  // the state of a fluid cell at the current phi: populations and macroscopic values
  auto load = [&](int x, int y, int z, T* gc, T* hc, CellState<T>& cs) {
    const long c0 = cell_index(P, x, y, z);
    for (int i = 0; i < L27.q; ++i) gc[i] = S.g[(size_t)i * N + c0];
    for (int i = 0; i < LH.q; ++i) hc[i] = S.h[(size_t)i * N + c0];
    cell_macro(S, x, y, z, gc, cs);
  };
  auto fluid = [&](int x, int y, int z) { return S.solid.empty() || !S.solid[cell_index(P, x, y, z)]; };
  if (P.schedule == SCHED_CONCURRENT) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P.nz; ++z)
      for (int y = 0; y < P.ny; ++y)
        for (int x = 0; x < P.nx; ++x) {
          if (!fluid(x, y, z)) continue;  // solid cells are not updated
          T gc[27], hc[27];
          CellState<T> cs;
          load(x, y, z, gc, hc, cs);
          g_update(S, x, y, z, cs, gc);
          h_update(S, x, y, z, cs, hc);
        }
    std::swap(S.g, S.gn);
    std::swap(S.h, S.hn);
    compute_phi(S);
  } else {
    // phase field first: h at phi^t and u^t, then phi^{t+1} = sum h
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P.nz; ++z)
      for (int y = 0; y < P.ny; ++y)
        for (int x = 0; x < P.nx; ++x) {
          if (!fluid(x, y, z)) continue;
          T gc[27], hc[27];
          CellState<T> cs;
          load(x, y, z, gc, hc, cs);
          h_update(S, x, y, z, cs, hc);
        }
    std::swap(S.h, S.hn);
    compute_phi(S);
    // then the hydrodynamics with g^t at phi^{t+1}
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P.nz; ++z)
      for (int y = 0; y < P.ny; ++y)
        for (int x = 0; x < P.nx; ++x) {
          if (!fluid(x, y, z)) continue;
          T gc[27], hc[27];
          CellState<T> cs;
          load(x, y, z, gc, hc, cs);
          g_update(S, x, y, z, cs, gc);
        }
    std::swap(S.g, S.gn);
  }
  S.step += 1;
}

// The initial state: parameters from (ip, dp) and populations at their
// equilibria h^eq(phi0, u0), g^eq(p0, u0).
template <typename T>
void init_sim(Sim<T>& S, const int* ip, const double* dp, const double* phi0, const double* u0, const double* p0) {
  Params& P = S.P;
  P.nx = ip[0];
  P.ny = ip[1];
  P.nz = ip[2];
  for (int k = 0; k < 6; ++k) P.bc[k] = ip[3 + k];
  P.collision = ip[9];
  P.qh = ip[10] == 27 ? 27 : (ip[10] == 9 ? 9 : 15);
  P.schedule = ip[11] == SCHED_SEQUENTIAL ? SCHED_SEQUENTIAL : SCHED_CONCURRENT;
  P.rho_h = dp[0];
  P.rho_l = dp[1];
  P.nu_h = dp[2];
  P.nu_l = dp[3];
  P.sigma = dp[4];
  P.mobility = dp[5];
  P.xi = dp[6];
  P.g[0] = dp[7];
  P.g[1] = dp[8];
  P.g[2] = dp[9];
  S.sigma = P.sigma;
  S.mobility = P.mobility;
  S.xi = P.xi;
  S.N = (long)P.nx * P.ny * P.nz;
  const long N = S.N;
  S.h.assign((size_t)P.qh * N, T(0.0));
  S.hn.assign((size_t)P.qh * N, T(0.0));
  const Lattice& LG = g_lattice(P);
  S.g.assign((size_t)LG.q * N, T(0.0));
  S.gn.assign((size_t)LG.q * N, T(0.0));
  S.phi.assign(N, T(0.0));
  const Lattice& LH = h_lattice(P);
  for (long c = 0; c < N; ++c) {
    T u[3] = {0.0, 0.0, 0.0};
    if (u0)
      for (int a = 0; a < 3; ++a) u[a] = u0[a * N + c];
    T ps = p0 ? p0[c] : 0.0;
    T geq[27];
    geq_of(LG, ps, u, geq);
    for (int i = 0; i < LG.q; ++i) S.g[(size_t)i * N + c] = geq[i];
    for (int i = 0; i < LH.q; ++i) {
      double cu = LH.c[3 * i] * value(u[0]) + LH.c[3 * i + 1] * value(u[1]) + LH.c[3 * i + 2] * value(u[2]);
      S.h[(size_t)i * N + c] = LH.w[i] * phi0[c] * (1.0 + cu / CS2);
    }
  }
  compute_phi(S);
}

typedef Sim<double> SimD;

}  // namespace

extern "C" {

// iparams: nx, ny, nz, bc[6], collision, h lattice (15, 27, or 9 for D2Q9 h and g),
//          schedule (0 concurrent, 1 sequential)   (12 ints)
// dparams: rho_h, rho_l, nu_h, nu_l, sigma, mobility, xi, gx, gy, gz (10 doubles)
// phi0 (N), u0 (3N SoA, nullable), p0 (N, nullable): initial state; the
// populations start at their equilibria h^eq(phi0, u0), g^eq(p0, u0).
void* ora_new(const int* ip, const double* dp, const double* phi0, const double* u0, const double* p0) {
  SimD* S = new SimD();
  init_sim(*S, ip, dp, phi0, u0, p0);
  return S;
}

// Exact derivative, by forward-mode differentiation of the same arithmetic, of
// J = sum_o sum_x W_o(x) phi^{t_o}(x) after n steps from the initial state of
// ora_new, with respect to parameter `which` (0: M, 1: xi, 2: sigma).
// obs_steps (n_obs, each in [0, n]) and obs_w (n_obs x N, row-major).
// Writes J and dJ / d(parameter).
void ora_tangent(const int* ip, const double* dp, const double* phi0, const double* u0, const double* p0, int which,
                 int n, int n_obs, const int* obs_steps, const double* obs_w, int nthreads, double* J, double* dJ) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  Sim<Dual> S;
  init_sim(S, ip, dp, phi0, u0, p0);
  if (which == 0) S.mobility.d = 1.0;
  if (which == 1) S.xi.d = 1.0;
  if (which == 2) S.sigma.d = 1.0;
  double j = 0.0, dj = 0.0;
  for (int k = 0; k <= n; ++k) {
    for (int o = 0; o < n_obs; ++o)
      if (obs_steps[o] == k) {
        const double* W = obs_w + (size_t)o * S.N;
        for (long c = 0; c < S.N; ++c) {
          j += W[c] * S.phi[c].v;
          dj += W[c] * S.phi[c].d;
        }
      }
    if (k < n) do_step(S);
  }
  *J = j;
  *dJ = dj;
}

void ora_free(void* s) { delete (SimD*)s; }

// Solid cells (mask of N bytes, nonzero = solid): links into them bounce
// back half-way, stencil reads of them return the reading cell's phi, they are
// not updated and hold zero populations.
void ora_set_solid(void* s, const unsigned char* mask) {
  SimD* S = (SimD*)s;
  S->solid.assign(mask, mask + S->N);
  for (long c = 0; c < S->N; ++c)
    if (S->solid[c]) {
      for (size_t i = 0; i < S->h.size() / S->N; ++i) S->h[i * S->N + c] = 0.0;
      for (size_t i = 0; i < S->g.size() / S->N; ++i) S->g[i * S->N + c] = 0.0;
    }
  compute_phi(*S);
}

void ora_step(void* s, int n, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  for (int k = 0; k < n; ++k) do_step(*(SimD*)s);
}

long ora_time(void* s) { return ((SimD*)s)->step; }

// Populations in canonical order, SoA [i][cell].
void ora_get_pops(void* s, double* h, double* g) {
  SimD* S = (SimD*)s;
  if (h) std::memcpy(h, S->h.data(), sizeof(double) * S->h.size());
  if (g) std::memcpy(g, S->g.data(), sizeof(double) * S->g.size());
}

void ora_set_pops(void* s, const double* h, const double* g) {
  SimD* S = (SimD*)s;
  if (h) std::memcpy(S->h.data(), h, sizeof(double) * S->h.size());
  if (g) std::memcpy(S->g.data(), g, sizeof(double) * S->g.size());
  compute_phi(*S);
}

// Macroscopic fields at the current time level (any output may be NULL):
// phi, rho(phi), p = p* rho c_s^2, u = sum c g + F/(2 rho) (3N SoA).
void ora_fields(void* s, double* phi, double* rho, double* p, double* u) {
  SimD* S = (SimD*)s;
  const Params& P = S->P;
  const long N = S->N;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < P.nz; ++z)
    for (int y = 0; y < P.ny; ++y)
      for (int x = 0; x < P.nx; ++x) {
        long c0 = cell_index(P, x, y, z);
        if (!S->solid.empty() && S->solid[c0]) {  // every output is zero in a solid cell
          if (phi) phi[c0] = 0;
          if (rho) rho[c0] = 0;
          if (p) p[c0] = 0;
          if (u)
            for (int a = 0; a < 3; ++a) u[a * N + c0] = 0;
          continue;
        }
        double gc[27];
        for (int i = 0; i < g_lattice(P).q; ++i) gc[i] = S->g[(size_t)i * N + c0];
        CellState<double> cs;
        cell_macro(*S, x, y, z, gc, cs);
        if (phi) phi[c0] = cs.phi;
        if (rho) rho[c0] = cs.rho;
        if (p) p[c0] = cs.pstar * cs.rho * CS2;
        if (u)
          for (int a = 0; a < 3; ++a) u[a * N + c0] = cs.u[a];
      }
}

// Lattice tables for the pin tests: q = 15 or 27.
int ora_tables(int q, int* c, double* w, int* opp, int* degree, double* M, double* Minv) {
  const Lattice* L = (q == 15) ? &Q15() : (q == 27) ? &Q27() : (q == 9) ? &Q9() : nullptr;
  if (!L) return -1;
  for (int i = 0; i < L->q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = L->c[3 * i + a];
    w[i] = L->w[i];
    opp[i] = L->opp[i];
    degree[i] = L->degree[i];
  }
  for (int k = 0; k < L->q * L->q; ++k) {
    M[k] = L->M[k];
    Minv[k] = L->Minv[k];
  }
  return L->q;
}

// One collision of a single g cell through the MRT machinery, for pin tests:
// f, feq, src, rates (q each) -> out.
void ora_mrt_collide(int q, const double* f, const double* feq, const double* src, const double* s, double* out) {
  const Lattice& L = (q == 15) ? Q15() : (q == 9) ? Q9() : Q27();
  mrt_collide(L, f, feq, src, s, out);
}

}  // extern "C"
