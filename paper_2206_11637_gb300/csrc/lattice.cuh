// Lattice constants and population storage formats of the PFLBM kernels.
//
// D3Q27 (hydrodynamics g) and D3Q15 or D3Q27 (phase field h), or D2Q9 for both in
// 2-D, in the canonical order of
// the C interface: cz, cy, cx each over -1, 0, 1 with cx fastest.  For D3Q27
// this gives i = (cx+1) + 3(cy+1) + 9(cz+1), so velocities, weights and
// opposites are closed-form functions of i that fold to constants inside
// fully unrolled loops.  D3Q15 keeps the members with |c|^2 in {0, 1, 3};
// member k sits at D3Q27 index 2k (k < 7), 13 (k = 7) or 2k - 2 (k > 7), and
// its opposite is 14 - k.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pfl {

__host__ __device__ constexpr int q27_cx(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int q27_cy(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int q27_cz(int i) { return i / 9 - 1; }
__host__ __device__ constexpr int q27_n2(int i) {
  return q27_cx(i) * q27_cx(i) + q27_cy(i) * q27_cy(i) + q27_cz(i) * q27_cz(i);
}
__host__ __device__ constexpr int q27_opp(int i) { return 26 - i; }
// weights 8/27, 2/27, 1/54, 1/216 by |c|^2 = 0, 1, 2, 3
__host__ __device__ constexpr double q27_w(int i) {
  return q27_n2(i) == 0 ? 8.0 / 27.0 : q27_n2(i) == 1 ? 2.0 / 27.0 : q27_n2(i) == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
}

__host__ __device__ constexpr int q15_to27(int k) { return k < 7 ? 2 * k : (k == 7 ? 13 : 2 * k - 2); }
__host__ __device__ constexpr int q15_cx(int k) { return q27_cx(q15_to27(k)); }
__host__ __device__ constexpr int q15_cy(int k) { return q27_cy(q15_to27(k)); }
__host__ __device__ constexpr int q15_cz(int k) { return q27_cz(q15_to27(k)); }
__host__ __device__ constexpr int q15_opp(int k) { return 14 - k; }
// weights 2/9, 1/9, 1/72 by |c|^2 = 0, 1, 3
__host__ __device__ constexpr double q15_w(int k) {
  return q27_n2(q15_to27(k)) == 0 ? 2.0 / 9.0 : q27_n2(q15_to27(k)) == 1 ? 1.0 / 9.0 : 1.0 / 72.0;
}

// D2Q9 (the 2-D lattice of both sets) is the cz = 0 slice of D3Q27: member j
// sits at D3Q27 index 9 + j, its opposite is 8 - j; weights 4/9, 1/9, 1/36 by
// |c|^2 = 0, 1, 2.
__host__ __device__ constexpr double q9_w(int j) {
  return q27_n2(9 + j) == 0 ? 4.0 / 9.0 : q27_n2(9 + j) == 1 ? 1.0 / 9.0 : 1.0 / 36.0;
}

// A lattice by its size Q = 27 (D3Q27), 15 (D3Q15) or 9 (D2Q9).  In each
// order member k pairs with Q - 1 - k, members k < (Q - 1) / 2 are one of each
// opposite pair, and (Q - 1) / 2 is the rest velocity.
template <int Q>
__host__ __device__ constexpr int lq_to27(int k) {
  return Q == 27 ? k : (Q == 15 ? q15_to27(k) : 9 + k);
}
template <int Q>
__host__ __device__ constexpr double lq_w(int k) {
  return Q == 27 ? q27_w(k) : (Q == 15 ? q15_w(k) : q9_w(k));
}

// The phase-field lattice QH = 15 (D3Q15), 27 (D3Q27) or 9 (D2Q9); the
// hydrodynamic lattice that goes with it is D2Q9 for QH = 9, else D3Q27.
template <int QH>
__host__ __device__ constexpr int qg_of() {
  return QH == 9 ? 9 : 27;
}
template <int QH>
__host__ __device__ constexpr int hq_to27(int k) {
  return lq_to27<QH>(k);
}
template <int QH>
__host__ __device__ constexpr int hq_cx(int k) {
  return q27_cx(hq_to27<QH>(k));
}
template <int QH>
__host__ __device__ constexpr int hq_cy(int k) {
  return q27_cy(hq_to27<QH>(k));
}
template <int QH>
__host__ __device__ constexpr int hq_cz(int k) {
  return q27_cz(hq_to27<QH>(k));
}
template <int QH>
__host__ __device__ constexpr double hq_w(int k) {
  return lq_w<QH>(k);
}
template <int QH>
__host__ __device__ constexpr int hq_rest() {
  return (QH - 1) / 2;
}

// FP16S format (shifted FP16 storage, FP32 arithmetic), per population and
// divided by its weight:
//   h: stored = fp16(KH16 * (h_i / w_i - phi_x)), x the writing cell and phi_x
//      its phase field at the step of writing (a double-buffered per-cell
//      FP32 array), so that only the non-equilibrium and velocity parts are
//      stored;
//   g: stored = fp16(KG16 * (g_i / w_i - P_x)), P_x = fp16(p*_x) the
//      normalised pressure of the writing cell at the step of writing, itself
//      kept in a double-buffered per-cell FP16 array (reader and writer use
//      the same rounded value).  g_i / w_i = p* + O(u): without the shift, the
//      FP16 rounding of p* alone (5e-4 p*) swamps u where p* >> |u|, as in the
//      gas of a bubble (p* = 3 p / rho_L).
// Fresh states (initialisation) are stored against their own initial phi and
// p*, so that a state at rest is stored exactly.  The power-of-two scales lift
// small values out of the FP16 subnormal range while keeping
// |h_i / w_i - phi| up to 64 and |g_i / w_i - P| up to 256 representable.
constexpr double KH16 = 1024.0;
constexpr double KG16 = 256.0;

template <int PREC>
struct Store;

template <>
struct Store<0> {  // FP64 storage and arithmetic
  typedef double S;
  typedef double R;
  typedef double PhiT;
};

template <>
struct Store<1> {  // FP32 storage and arithmetic
  typedef float S;
  typedef float R;
  typedef float PhiT;
};

template <>
struct Store<2> {  // shifted FP16 storage, FP32 arithmetic
  typedef __half S;
  typedef float R;
  typedef float PhiT;
};

// g population i: load / store in the arithmetic type; pshift is the p*
// shift of the writing cell (FP16S only, zero otherwise).
template <int PREC, int QG = 27>
__device__ __forceinline__ typename Store<PREC>::R ld_g(const typename Store<PREC>::S* a, size_t idx, int i,
                                                        typename Store<PREC>::R pshift = 0) {
  if constexpr (PREC == 2)
    return (__half2float(a[idx]) * (float)(1.0 / KG16) + pshift) * (float)lq_w<QG>(i);
  else
    return a[idx];
}
template <int PREC, int QG = 27>
__device__ __forceinline__ void st_g(typename Store<PREC>::S* a, size_t idx, int i, typename Store<PREC>::R v,
                                     typename Store<PREC>::R pshift = 0) {
  if constexpr (PREC == 2)
    a[idx] = __float2half_rn((v * (float)(1.0 / lq_w<QG>(i)) - pshift) * (float)KG16);
  else
    a[idx] = v;
}

// p* shift of the cells that wrote the stored g (FP16S), as the arithmetic type.
__device__ __forceinline__ float ld_pshift(const __half* p, size_t cell) { return __half2float(__ldg(p + cell)); }

// h population k: load adds back the shift phi_src (FP16S only).
template <int PREC, int QH>
__device__ __forceinline__ typename Store<PREC>::R ld_h(const typename Store<PREC>::S* a, size_t idx, int k,
                                                        typename Store<PREC>::R phi_src) {
  if constexpr (PREC == 2)
    return (__half2float(a[idx]) * (float)(1.0 / KH16) + phi_src) * (float)hq_w<QH>(k);
  else
    return a[idx];
}
// Store of h from q = h_i / w_i - shift (the shift is zero for FP64 / FP32).
template <int PREC, int QH>
__device__ __forceinline__ void st_h_q(typename Store<PREC>::S* a, size_t idx, int k, typename Store<PREC>::R q) {
  typedef typename Store<PREC>::R R;
  if constexpr (PREC == 2)
    a[idx] = __float2half_rn(q * (float)KH16);
  else
    a[idx] = (R)hq_w<QH>(k) * q;
}

}  // namespace pfl
