// lj_pair.cuh -- the Lennard-Jones pair term shared by the full-list and
// half-list force kernels (only the CUDA sources include it).
//
// V(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] - shift, cut at rc (Sec.
// "Potentials support"); shift_mode 1 subtracts V(rc), shift_mode 2 also
// the slope term (r - rc) V'(rc), so value and force vanish at rc.
#pragma once

#include "k_pair.cuh"

namespace mdk {
namespace pair {

// the LJ constants in the pair precision
template <class R>
struct LJc {
  R rc2, sig2, eps24, eps4, ush, durc, rcut;
  __device__ __forceinline__ explicit LJc(const LJParams &lp) {
    const bool f64 = sizeof(R) == 8;
    rc2 = f64 ? (R)lp.rc2 : (R)lp.rc2f;
    sig2 = f64 ? (R)lp.sig2 : (R)lp.sig2f;
    eps24 = f64 ? (R)lp.eps24 : (R)lp.eps24f;
    eps4 = f64 ? (R)lp.eps4 : (R)lp.eps4f;
    ush = f64 ? (R)lp.u_shift : (R)lp.u_shiftf;
    durc = f64 ? (R)lp.du_rc : (R)lp.du_rcf;
    rcut = f64 ? (R)lp.rc : (R)lp.rcf;
  }
};

// For r^2 < rc^2: fr = V'(r) / r, and with ENERGY the pair energy v = V(r).
// FP32: rounded in the packed LJ walk's order, fr = (-24 eps (2 s6 - 1))
// (s6 / r^2), so every mixed LJ kernel gives a pair the same force.
template <class GP, int SHIFT, bool ENERGY, class R>
__device__ __forceinline__ void lj_pair(const LJc<R> &c, R r2, R &fr, R &v) {
  const R inv = GP::rcp(r2);
  const R s2 = c.sig2 * inv;
  const R s6 = s2 * s2 * s2;
  if constexpr (sizeof(R) == 4)
    fr = __fmul_rn(__fmul_rn(-c.eps24, __fmaf_rn(s6, 2.0f, -1.0f)), __fmul_rn(s6, inv));
  else
    fr = -c.eps24 * (R(2) * s6 * s6 - s6) * inv;
  R r = 0;
  if (SHIFT == 2) {
    r = GP::sqr(r2);
    fr -= c.durc / r;
  }
  if (ENERGY) {
    v = c.eps4 * (s6 * s6 - s6) - c.ush;
    if (SHIFT == 2) v -= (r - c.rcut) * c.durc;
  }
}

}  // namespace pair
}  // namespace mdk
