// k_pair.cuh -- device helpers shared by the pair kernels (k_lj.cu, k_eam.cu):
// precision traits of the gather copy, spline pieces, the neighbour walk and
// the fused velocity-Verlet epilogue.  Only the CUDA sources include it.
#pragma once

#include <math.h>

#include "mdk_internal.cuh"

namespace mdk {
namespace pair {

// cubic Hermite piece on [k, k+1] with knots (y, h*m): value and h*derivative
template <class R>
__device__ __forceinline__ R herm_val(R t, R y0, R m0, R y1, R m1) {
  const R t2 = t * t, t3 = t2 * t;
  const R h01 = R(3) * t2 - R(2) * t3;
  const R h10 = t3 - R(2) * t2 + t;
  const R h11 = t3 - t2;
  return y0 + h01 * (y1 - y0) + h10 * m0 + h11 * m1;
}
template <class R>
__device__ __forceinline__ R herm_der(R t, R y0, R m0, R y1, R m1) {
  const R t2 = t * t;
  const R d00 = R(6) * t2 - R(6) * t;
  const R d10 = R(3) * t2 - R(4) * t + R(1);
  const R d11 = R(3) * t2 - R(2) * t;
  return d00 * (y0 - y1) + d10 * m0 + d11 * m1;
}

// ---- gather-copy access per precision ---------------------------------------
template <class P>
struct G;
template <>
struct G<Fp64> {
  using R = double;
  using V = dvec4;
  using T2 = double2;
  static __device__ __forceinline__ dvec4 ld(const dvec4 *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    dvec4 r;
    r.x = a.x;
    r.y = a.y;
    r.z = b.x;
    r.w = b.y;
    return r;
  }
  static __device__ __forceinline__ void st(dvec4 *p, double a, double b, double c,
                                            uint32_t w) {
    double2 *q = reinterpret_cast<double2 *>(p);
    q[0] = make_double2(a, b);
    q[1] = make_double2(c, __longlong_as_double((long long)w));
  }
  static __device__ __forceinline__ uint32_t info(const dvec4 &p) {
    return (uint32_t)__double_as_longlong(p.w);
  }
  static __device__ __forceinline__ void h(const Grid &g, double &hx, double &hy, double &hz) {
    hx = g.h[0];
    hy = g.h[1];
    hz = g.h[2];
  }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
  static __device__ __forceinline__ double sqr(double x) { return sqrt(x); }
  // EAM tables: (y_k, h m_k) per knot
  using Tab1 = double2;
  using Tab2 = double2;
  static __device__ __forceinline__ const double2 *tab1(const EAMParams &e) { return e.rho64; }
  static __device__ __forceinline__ const double2 *rho2(const EAMParams &e) { return e.rho64; }
  static __device__ __forceinline__ int n1(const EAMParams &e) { return e.nr; }
  static __device__ __forceinline__ double val1(const double2 *t, int k, double u) {
    const double2 a = t[k], b = t[k + 1];
    return herm_val<double>(u, a.x, a.y, b.x, b.y);
  }
  // h * derivative
  static __device__ __forceinline__ double der2(const double2 *t, int k, double u) {
    const double2 a = t[k], b = t[k + 1];
    return herm_der<double>(u, a.x, a.y, b.x, b.y);
  }
  // force pass: interleaved phi / rho knots, h * derivatives of both
  using TabPR = dvec4;
  static __device__ __forceinline__ const dvec4 *pr(const EAMParams &e) { return e.pr64; }
  static __device__ __forceinline__ void der_pr(const dvec4 *t, int k, double u, double &dphi,
                                                double &drho) {
    const dvec4 a = t[k], b = t[k + 1];
    dphi = herm_der<double>(u, a.x, a.y, b.x, b.y);
    drho = herm_der<double>(u, a.z, a.w, b.z, b.w);
  }
  static __device__ __forceinline__ double val_pr(const dvec4 *t, const EAMParams &, int k,
                                                  double u) {
    const dvec4 a = t[k], b = t[k + 1];
    return herm_val<double>(u, a.x, a.y, b.x, b.y);
  }
  // gather copy with F'(rho) in place of the info word
  static __device__ __forceinline__ void st_fp(dvec4 *p, const dvec4 &q, double fp) {
    double2 *o = reinterpret_cast<double2 *>(p);
    o[0] = make_double2(q.x, q.y);
    o[1] = make_double2(q.z, fp);
  }
  static __device__ __forceinline__ double fp_of(const dvec4 &q) { return q.w; }
};
template <>
struct G<Mixed> {
  using R = float;
  using V = float4;
  using T2 = float2;
  static __device__ __forceinline__ float4 ld(const float4 *p) { return __ldg(p); }
  static __device__ __forceinline__ void st(float4 *p, double a, double b, double c,
                                            uint32_t w) {
    *p = make_float4((float)a, (float)b, (float)c, __uint_as_float(w));
  }
  static __device__ __forceinline__ uint32_t info(const float4 &p) {
    return __float_as_uint(p.w);
  }
  static __device__ __forceinline__ void h(const Grid &g, float &hx, float &hy, float &hz) {
    hx = g.hf[0];
    hy = g.hf[1];
    hz = g.hf[2];
  }
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
  static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ float sqr(float x) { return sqrtf(x); }
  // EAM tables rounded from FP64 differences (no FP32 cancellation):
  // density pass per interval (y_k, dy_k, h m_k, h m_{k+1}); rho per knot
  // (dy_k, h m_k) for the adjoint
  using Tab1 = float4;
  using Tab2 = float2;
  static __device__ __forceinline__ const float4 *tab1(const EAMParams &e) { return e.rho_i32; }
  static __device__ __forceinline__ const float2 *rho2(const EAMParams &e) { return e.rho_d32; }
  static __device__ __forceinline__ int n1(const EAMParams &e) { return e.nr - 1; }
  static __device__ __forceinline__ float val1(const float4 *t, int k, float u) {
    const float4 q = t[k];
    const float u2 = u * u, u3 = u2 * u;
    return q.x + (3.0f * u2 - 2.0f * u3) * q.y + (u3 - 2.0f * u2 + u) * q.z + (u3 - u2) * q.w;
  }
  static __device__ __forceinline__ float der2(const float2 *t, int k, float u) {
    const float2 a = t[k], b = t[k + 1];
    const float u2 = u * u;
    return (6.0f * u - 6.0f * u2) * a.x + (3.0f * u2 - 4.0f * u + 1.0f) * a.y +
           (3.0f * u2 - 2.0f * u) * b.y;
  }
  // force pass: interleaved phi / rho differences and slopes, h * derivatives
  using TabPR = float4;
  static __device__ __forceinline__ const float4 *pr(const EAMParams &e) { return e.pr32; }
  // derivatives (and the phi value) of interval k from a = pr32[k] and the
  // next knot's slopes in b.y (phi) and b.w (rho)
  static __device__ __forceinline__ void der_ab(const float4 &a, const float4 &b, float u,
                                                float &dphi, float &drho) {
    const float u2 = u * u;
    const float w0 = 6.0f * u - 6.0f * u2, w1 = 3.0f * u2 - 4.0f * u + 1.0f,
                w3 = 3.0f * u2 - 2.0f * u;
    dphi = w0 * a.x + w1 * a.y + w3 * b.y;
    drho = w0 * a.z + w1 * a.w + w3 * b.w;
  }
  static __device__ __forceinline__ float val_ab(float phi_k, const float4 &a, const float4 &b,
                                                 float u) {
    const float u2 = u * u, u3 = u2 * u;
    return phi_k + (3.0f * u2 - 2.0f * u3) * a.x + (u3 - 2.0f * u2 + u) * a.y + (u3 - u2) * b.y;
  }
  static __device__ __forceinline__ void der_pr(const float4 *t, int k, float u, float &dphi,
                                                float &drho) {
    der_ab(t[k], t[k + 1], u, dphi, drho);
  }
  static __device__ __forceinline__ float val_pr(const float4 *t, const EAMParams &e, int k,
                                                 float u) {
    return val_ab(__ldg(e.phi_v32 + k), t[k], t[k + 1], u);
  }
  // the 32-byte interval records (pr8): one 256-bit read-only load per pair
  static __device__ __forceinline__ const float4 *pr8(const EAMParams &e) { return e.pr8; }
  static __device__ __forceinline__ void ld_pr8(const float4 *t, int k, float4 &a, float4 &b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(t + 2 * (size_t)k));
  }
  static __device__ __forceinline__ float val_ab(const float4 &a, const float4 &b, float u) {
    return val_ab(b.x, a, b, u);
  }
  static __device__ __forceinline__ void st_fp(float4 *p, const float4 &q, double fp) {
    *p = make_float4(q.x, q.y, q.z, (float)fp);
  }
  static __device__ __forceinline__ float fp_of(const float4 &q) { return q.w; }
};

// F(rho) and F'(rho) in FP64 from the F table (once per atom): cubic
// Hermite inside (the first piece extended below), linear continuation of
// the last knot above rho_max (flagged), NaN flagged.
__device__ __forceinline__ void embed_fp64(const Sys &s, const EAMParams &ep, double rho_i,
                                           double &Fv, double &dF) {
  if (rho_i > ep.rho_max) {
    const int n = ep.nrho;
    const double2 a0 = ep.F64[n - 2], a1 = ep.F64[n - 1];
    const double d1 = herm_der<double>(1.0, a0.x, a0.y, a1.x, a1.y) * ep.inv_drho;
    Fv = a1.x + d1 * (rho_i - ep.rho_max);
    dF = d1;
    atomicOr(&s.st->bits, isfinite(rho_i) ? kStRhoRange : kStNonfinite);
  } else if (!(rho_i == rho_i)) {
    Fv = 0.0;
    dF = 0.0;
    atomicOr(&s.st->bits, kStNonfinite);
  } else {
    const double u = rho_i * ep.inv_drho;
    int kk = (int)floor(u);
    kk = kk > ep.nrho - 2 ? ep.nrho - 2 : (kk < 0 ? 0 : kk);
    const double t = u - (double)kk;
    const double2 a0 = ep.F64[kk], a1 = ep.F64[kk + 1];
    Fv = herm_val<double>(t, a0.x, a0.y, a1.x, a1.y);
    dF = herm_der<double>(t, a0.x, a0.y, a1.x, a1.y) * ep.inv_drho;
  }
}

// ---- the neighbour walk ------------------------------------------------------------
// Stencil offset of a list entry times 4^d, exactly, in the pair precision,
// without an int-to-float conversion: the entry's 2-bit code c = s_d + 1 sits
// at bits 2d..2d+1, so (e & (3 << 2d)) = 4^d c lands in the low mantissa bits
// of 2^23 (2^52) with one AND/OR, and 2^23 + 4^d (2^52 + 4^d) is subtracted.
// With the cell size pre-scaled by 4^-d (an exact power-of-two scaling),
// s_scaled(e, d) * (h_d / 4^d) is exactly s_d h_d.
__device__ __forceinline__ float s_scaled(float, uint32_t e, int d) {
  return __uint_as_float((e & (3u << (2 * d))) | 0x4B000000u) - (8388608.0f + (float)(1 << (2 * d)));
}
__device__ __forceinline__ double s_scaled(double, uint32_t e, int d) {
  return __longlong_as_double((long long)(e & (3u << (2 * d))) | 0x4330000000000000LL) -
         (4503599627370496.0 + (double)(1 << (2 * d)));
}
// The pair vector component (p_j - p_i) + s h and r^2, rounded in one fixed
// order that every list kernel (and the packed LJ walk) shares: the
// difference, then the shift by one FMA; r^2 = fma(dz, dz, fma(dy, dy, dx dx)).
// Seen from j the vector is exactly minus the one seen from i, so both atoms
// of a pair get the same r^2, bit for bit, and the same cutoff decision.
__device__ __forceinline__ float pvec(float pj, float pi, float sh, float h) {
  return __fmaf_rn(sh, h, __fsub_rn(pj, pi));
}
__device__ __forceinline__ double pvec(double pj, double pi, double sh, double h) {
  return __fma_rn(sh, h, __dsub_rn(pj, pi));
}
__device__ __forceinline__ float r2_of(float dx, float dy, float dz) {
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}
__device__ __forceinline__ double r2_of(double dx, double dy, double dz) {
  return __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
}

// the cell size scaled for s_scaled: (h_x, h_y / 4, h_z / 16)
template <class R>
__device__ __forceinline__ void h_scaled(R &hx, R &hy, R &hz) {
  hy *= R(0.25);
  hz *= R(0.0625);
}

// Walk the list of one atom with T lanes: lane t takes the groups of 8 list
// words t, t + T, t + 2T, ...  A group comes in one 32-byte load; its
// neighbour records are loaded four at a time before the four bodies run,
// so each thread keeps several independent loads in flight.  `commit` runs
// after every four pairs: the compensated per-atom sums take one block sum
// per four pairs instead of one term per pair.
template <int T, class Load, class Body, class Commit>
__device__ __forceinline__ void walk(const uint32_t *__restrict__ nbr, size_t Nc, int i, int nn,
                                     int t, Load &&load, Body &&body, Commit &&commit) {
  using Rec = decltype(load(0u));
  const size_t gstride = Nc * 2;  // uint4 per group row
  const uint4 *__restrict__ row = reinterpret_cast<const uint4 *>(nbr) + (size_t)i * 2 +
                                  (size_t)t * gstride;
  // the next group's load is issued before this group's pairs run, so
  // the list latency overlaps the neighbour gathers and the arithmetic
  uint4 na = make_uint4(0, 0, 0, 0), nb = na;
  if (kGroup * t < nn) {
    ld_group(row, na, nb);
  }
  for (int k = kGroup * t; k < nn; k += kGroup * T) {
    const uint4 a = na, b = nb;
    row += gstride * T;
    if (k + kGroup * T < nn) {
      ld_group(row, na, nb);
    }
    const uint32_t e[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    const int m = nn - k;  // valid entries in this group
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      Rec q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (4 * h + u < m) q[u] = load((uint32_t)nbr_j(e[4 * h + u]));
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (4 * h + u < m) body(e[4 * h + u], q[u]);
      commit();
    }
  }
}

// sum of v over the T lanes of one atom (fixed order: deterministic)
template <int T, class R>
__device__ __forceinline__ R lanes_sum(R v) {
#pragma unroll
  for (int o = 1; o < T; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Atoms are handed out in warp tiles of 32/T atoms (T lanes each) over a
// persistent grid; every lane of a warp runs the same number of tiles, so the
// lanes_sum shuffles always see the whole warp.
template <int T>
struct Tiles {
  static constexpr int kPerWarp = 32 / T;
  int lane, t, w0, nw;
  __device__ __forceinline__ Tiles() {
    lane = threadIdx.x & 31;
    t = lane & (T - 1);
    w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    nw = (gridDim.x * blockDim.x) >> 5;
  }
  __device__ __forceinline__ int atom(int w) const { return w * kPerWarp + lane / T; }
};

// what the accumulators s.hacc hold per precision (half lists, BPNN):
// int64 fixed point in units of 2^-40 in the mixed path, FP64 otherwise
template <class P>
struct HalfAcc;
template <>
struct HalfAcc<Mixed> {
  using Q = long long;
  static __device__ __forceinline__ long long q(float v) {
    return __float2ll_rn(v * 1099511627776.0f);  // 2^40, exact power of two
  }
  static __device__ __forceinline__ long long qd(double v) {  // a per-atom FP64 value
    return __double2ll_rn(v * kHalfScale);
  }
  static __device__ __forceinline__ void red(long long *p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
  }
  static __device__ __forceinline__ double take(long long *p) {
    const long long v = *p;
    *p = 0;
    return (double)v * (1.0 / kHalfScale);
  }
};
template <>
struct HalfAcc<Fp64> {
  using Q = double;
  static __device__ __forceinline__ double q(double v) { return v; }
  static __device__ __forceinline__ double qd(double v) { return v; }
  static __device__ __forceinline__ void red(long long *p, double v) {
    atomicAdd(reinterpret_cast<double *>(p), v);
  }
  static __device__ __forceinline__ double take(long long *p) {
    const double v = __longlong_as_double(*p);
    *p = 0;  // the bit pattern of +0.0
    return v;
  }
};

// ---- per-atom epilogue: store forces or integrate -----------------------------
template <class P>
__device__ __forceinline__ void drift_publish(const Sys &s, const StepArgs &a, int i,
                                              uint32_t inf, double vx, double vy, double vz) {
  using GP = G<P>;
  const size_t Nc = s.N_cap;
  double x = s.x[i] + a.dt * vx;
  double y = s.x[Nc + i] + a.dt * vy;
  double z = s.x[2 * Nc + i] + a.dt * vz;
  s.x[i] = x;
  s.x[Nc + i] = y;
  s.x[2 * Nc + i] = z;
  s.v[i] = vx;
  s.v[Nc + i] = vy;
  s.v[2 * Nc + i] = vz;
  const double ex = x - s.xref[i], ey = y - s.xref[Nc + i], ez = z - s.xref[2 * Nc + i];
  const double d2 = ex * ex + ey * ey + ez * ez;
  const bool bad = !isfinite(d2);
  const bool trig = bad || d2 > s.half_skin2;
  const unsigned act = __activemask();
  const unsigned m = __ballot_sync(act, trig);
  if (m && (threadIdx.x & 31) == (__ffs(m) - 1)) atomicOr(&s.st->rebuild, 1);
  if (bad) atomicOr(&s.st->bits, kStNonfinite);
  const Grid &g = s.grid[inf >> 8];
  const uint32_t cc = s.cellc[i];
  typename GP::V *out = (typename GP::V *)s.pg[a.cur ^ 1];
  GP::st(out + i, x - cell_center(g, 0, cell_coord(cc, 0)),
         y - cell_center(g, 1, cell_coord(cc, 1)), z - cell_center(g, 2, cell_coord(cc, 2)),
         inf);
}

// Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC 2011): ten rounds of two
// 64x64 -> 128-bit products on the counter, key bumped by Weyl constants.
__device__ __forceinline__ void philox4x64(unsigned long long c[4], unsigned long long k0,
                                           unsigned long long k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B97F4A7C15ULL;
      k1 += 0xBB67AE8584CAA73BULL;
    }
    const unsigned long long m0 = 0xD2E7470EE14C6C93ULL, m1 = 0xCA5A826395121157ULL;
    const unsigned long long hi0 = __umul64hi(m0, c[0]), lo0 = m0 * c[0];
    const unsigned long long hi1 = __umul64hi(m1, c[2]), lo1 = m1 * c[2];
    const unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Langevin force of atom i (once per atom and step; regions along x at the
// new positions, half-step velocity in s.v):
//   F += g (v - u) + sigma (xi - 1/2),  g = -beta m / A,
//   sigma = sqrt(24 beta m k_B T / (dt A)),
// xi uniform on [0, 1) from Philox4x64-10 with counter (id, step) and key
// (seed, 0).  FP64 path: xi = (out >> 11) 2^-53, FP64 arithmetic with the
// friction factor g precomputed per region and type (a few ulps of the
// friction force away from -beta m (v - u) / A evaluated per atom).  Mixed
// path: the thermostat force is computed in FP32 (it
// is noise and friction, on GB300's fast pipe), xi = (out >> 40) 2^-24.
template <class P>
__device__ __forceinline__ void langevin(const Sys &s, int i, uint32_t inf, double &Fx,
                                         double &Fy, double &Fz) {
  const size_t Nc = s.N_cap;
  const int type = inf & 15u;
  double g, sig, u[3] = {0.0, 0.0, 0.0};
  if (s.lang_rep_on) {  // the atom's replica, as a whole, at rest
    const double *q = s.lang_rep + ((size_t)(inf >> 8) * kMaxTypes + type) * 2;
    g = q[0];
    sig = q[1];
  } else {
    const double x = s.x[i];
    int r = -1;
    for (int q = 0; q < s.n_lang && r < 0; ++q)
      if (x >= s.lang_xlo[q] && x < s.lang_xhi[q]) r = q;
    if (r < 0) return;
    g = s.lang_g[r][type];
    sig = s.lang_sig[r][type];
    u[0] = s.lang_u[r][0];
    u[1] = s.lang_u[r][1];
    u[2] = s.lang_u[r][2];
  }
  unsigned long long c[4] = {(unsigned long long)s.id[i],
                             (unsigned long long)s.st->n_steps, 0ull, 0ull};
  philox4x64(c, s.lang_seed, 0ull);
  double *F[3] = {&Fx, &Fy, &Fz};
  if (sizeof(typename G<P>::R) == 8) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double xi = __dmul_rn((double)(c[d] >> 11), 0x1.0p-53);
      const double fr = __dmul_rn(g, __dadd_rn(s.v[d * Nc + i], -u[d]));
      const double fn = __dmul_rn(sig, __dadd_rn(xi, -0.5));
      *F[d] = __dadd_rn(__dadd_rn(*F[d], fr), fn);
    }
  } else {
    const float gf = (float)g, sigf = (float)sig;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float xi = (float)(unsigned)(c[d] >> 40) * 0x1.0p-24f;
      const float dv = (float)(s.v[d * Nc + i] - u[d]);
      *F[d] += (double)(gf * dv + sigf * (xi - 0.5f));
    }
  }
}

template <class P, int MODE, bool ENERGY>
__device__ __forceinline__ void epilogue64(const Sys &s, const StepArgs &a, int i, uint32_t inf,
                                           double Fx, double Fy, double Fz) {
  const size_t Nc = s.N_cap;
  if (MODE == kForceOnly) {
    s.f[i] = Fx;
    s.f[Nc + i] = Fy;
    s.f[2 * Nc + i] = Fz;
    if (!(isfinite(Fx) && isfinite(Fy) && isfinite(Fz))) atomicOr(&s.st->bits, kStNonfinite);
    return;
  }
  const int type = inf & 15u;
  const bool piston = (inf & kInfoPiston) != 0;
  if ((s.n_lang > 0 || s.lang_rep_on) && !piston) langevin<P>(s, i, inf, Fx, Fy, Fz);
  const double c = 0.5 * a.dt * s.acc_over_m[type];
  double vx = s.v[i], vy = s.v[Nc + i], vz = s.v[2 * Nc + i];
  if (piston) {
    vx = s.u_p;
    vy = 0.0;
    vz = 0.0;
  } else {
    vx += c * Fx;
    vy += c * Fy;
    vz += c * Fz;
  }
  if (ENERGY) s.ka[i] = s.ke_m[type] * (vx * vx + vy * vy + vz * vz);
  if (MODE == kFinal) {
    s.v[i] = vx;
    s.v[Nc + i] = vy;
    s.v[2 * Nc + i] = vz;
    s.f[i] = Fx;
    s.f[Nc + i] = Fy;
    s.f[2 * Nc + i] = Fz;
    if (!(isfinite(Fx) && isfinite(Fy) && isfinite(Fz))) atomicOr(&s.st->bits, kStNonfinite);
    return;
  }
  if (!piston) {
    vx += c * Fx;
    vy += c * Fy;
    vz += c * Fz;
  }
  drift_publish<P>(s, a, i, inf, vx, vy, vz);
}

// The mixed path's end of a step with FP32 forces: the kick increments
// dt/2 F/m are formed in FP32 (the forces carry FP32 precision) and added to
// the FP64 velocities; positions advance in FP64; the next gather copy is
// rounded from FP64 as always; the displacement since the last build is
// measured between the new and the build-time FP32 cell offsets (the same
// cell, both rounded from FP64: a few 1e-7 A against skin/2), except for
// atoms flagged far, which keep the FP64 test.  This keeps GB300's slow FP64
// pipe to the state updates themselves.
__device__ __forceinline__ void langevin_f(const Sys &s, int i, uint32_t inf, float &Fx,
                                           float &Fy, float &Fz) {
  const size_t Nc = s.N_cap;
  const int type = inf & 15u;
  double g, sig, u[3] = {0.0, 0.0, 0.0};
  if (s.lang_rep_on) {
    const double *q = s.lang_rep + ((size_t)(inf >> 8) * kMaxTypes + type) * 2;
    g = q[0];
    sig = q[1];
  } else {
    const double x = s.x[i];
    int r = -1;
    for (int q = 0; q < s.n_lang && r < 0; ++q)
      if (x >= s.lang_xlo[q] && x < s.lang_xhi[q]) r = q;
    if (r < 0) return;
    g = s.lang_g[r][type];
    sig = s.lang_sig[r][type];
    u[0] = s.lang_u[r][0];
    u[1] = s.lang_u[r][1];
    u[2] = s.lang_u[r][2];
  }
  unsigned long long c[4] = {(unsigned long long)s.id[i],
                             (unsigned long long)s.st->n_steps, 0ull, 0ull};
  philox4x64(c, s.lang_seed, 0ull);
  const float gf = (float)g, sigf = (float)sig;
  float *F[3] = {&Fx, &Fy, &Fz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float xi = (float)(unsigned)(c[d] >> 40) * 0x1.0p-24f;
    const float dv = (float)(s.v[d * Nc + i] - u[d]);
    *F[d] += gf * dv + sigf * (xi - 0.5f);
  }
}

// the mixed path's drift with the new velocities: positions advance in FP64,
// the displacement since the last build is tested in FP32 on the cell offsets
// (FP64 for far atoms), and the next gather copy is published
__device__ __forceinline__ void drift32(const Sys &s, const StepArgs &a, int i, uint32_t inf,
                                        double vx, double vy, double vz) {
  const size_t Nc = s.N_cap;
  // the state streams through once per step: evict-first loads and stores
  // leave L1 to the neighbour records
  const double x = __ldcs(s.x + i) + a.dt * vx;
  const double y = __ldcs(s.x + Nc + i) + a.dt * vy;
  const double z = __ldcs(s.x + 2 * Nc + i) + a.dt * vz;
  __stcs(s.x + i, x);
  __stcs(s.x + Nc + i, y);
  __stcs(s.x + 2 * Nc + i, z);
  __stcs(s.v + i, vx);
  __stcs(s.v + Nc + i, vy);
  __stcs(s.v + 2 * Nc + i, vz);
  const Grid &g = s.grid[inf >> 8];
  const uint32_t cc = s.cellc[i];
  const float px = (float)(x - cell_center(g, 0, cell_coord(cc, 0)));
  const float py = (float)(y - cell_center(g, 1, cell_coord(cc, 1)));
  const float pz = (float)(z - cell_center(g, 2, cell_coord(cc, 2)));
  bool bad, trig;
  if (!(inf & kInfoFar)) {
    const float4 q = __ldcs(s.pf + i);  // the build-time offset in the same cell
    const float ex = px - q.x, ey = py - q.y, ez = pz - q.z;
    const float d2 = ex * ex + ey * ey + ez * ez;
    bad = !isfinite(d2);
    trig = bad || d2 > s.half_skin2f;
  } else {
    const double ex = x - s.xref[i], ey = y - s.xref[Nc + i], ez = z - s.xref[2 * Nc + i];
    const double d2 = ex * ex + ey * ey + ez * ez;
    bad = !isfinite(d2);
    trig = bad || d2 > s.half_skin2;
  }
  const unsigned act = __activemask();
  const unsigned m = __ballot_sync(act, trig);
  if (m && (threadIdx.x & 31) == (__ffs(m) - 1)) atomicOr(&s.st->rebuild, 1);
  if (bad) atomicOr(&s.st->bits, kStNonfinite);
  float4 *out = (float4 *)s.pg[a.cur ^ 1];
  out[i] = make_float4(px, py, pz, __uint_as_float(inf));
}

// the mixed path's kick increment dt/2 F/m, formed in FP32
__device__ __forceinline__ double kick32(const Sys &s, const StepArgs &a, int type, float F) {
  return (double)(a.hdtf * s.acc_over_mf[type] * F);
}

template <int MODE, bool ENERGY>
__device__ __forceinline__ void epilogue32(const Sys &s, const StepArgs &a, int i, uint32_t inf,
                                           float Fx, float Fy, float Fz) {
  const size_t Nc = s.N_cap;
  if (MODE == kForceOnly) {
    s.f[i] = Fx;
    s.f[Nc + i] = Fy;
    s.f[2 * Nc + i] = Fz;
    if (!(isfinite(Fx) && isfinite(Fy) && isfinite(Fz))) atomicOr(&s.st->bits, kStNonfinite);
    return;
  }
  const int type = inf & 15u;
  const bool piston = (inf & kInfoPiston) != 0;
  if ((s.n_lang > 0 || s.lang_rep_on) && !piston) langevin_f(s, i, inf, Fx, Fy, Fz);
  const double dx = kick32(s, a, type, Fx), dy = kick32(s, a, type, Fy),
               dz = kick32(s, a, type, Fz);
  double vx = __ldcs(s.v + i), vy = __ldcs(s.v + Nc + i), vz = __ldcs(s.v + 2 * Nc + i);
  if (piston) {
    vx = s.u_p;
    vy = 0.0;
    vz = 0.0;
  } else {
    vx += dx;
    vy += dy;
    vz += dz;
  }
  if (ENERGY) s.ka[i] = s.ke_m[type] * (vx * vx + vy * vy + vz * vz);
  if (MODE == kFinal) {
    s.v[i] = vx;
    s.v[Nc + i] = vy;
    s.v[2 * Nc + i] = vz;
    s.f[i] = Fx;
    s.f[Nc + i] = Fy;
    s.f[2 * Nc + i] = Fz;
    if (!(isfinite(Fx) && isfinite(Fy) && isfinite(Fz))) atomicOr(&s.st->bits, kStNonfinite);
    return;
  }
  if (!piston) {
    vx += dx;
    vy += dy;
    vz += dz;
  }
  drift32(s, a, i, inf, vx, vy, vz);
}

// Finish the step of atom i from its total force: FP32 forces (the mixed
// path's pair sums) take epilogue32, FP64 forces the FP64 state arithmetic.
template <class P, int MODE, bool ENERGY, class F>
__device__ __forceinline__ void epilogue(const Sys &s, const StepArgs &a, int i, uint32_t inf,
                                         F Fx, F Fy, F Fz) {
  if (sizeof(F) == 4)
    epilogue32<MODE, ENERGY>(s, a, i, inf, (float)Fx, (float)Fy, (float)Fz);
  else
    epilogue64<P, MODE, ENERGY>(s, a, i, inf, (double)Fx, (double)Fy, (double)Fz);
}

}  // namespace pair
}  // namespace mdk
