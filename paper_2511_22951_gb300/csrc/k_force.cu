// k_force.cu -- force loop and velocity-Verlet update (GB300, sm_103a).
//
// Paper passages:
//  * pair force  f_i = sum_j V'(r_ij) r_ji / r_ji   (Sec. "Potentials support")
//  * Lennard-Jones and single-element EAM from a table (same section and the
//    Al Hugoniot section); EAM energy U = 1/2 sum phi(r_ij) + sum F(rho_i),
//    rho_i = sum_j rho(r_ij), force
//    f_i = sum_j [phi'(r) + (F'(rho_i) + F'(rho_j)) rho'(r)] r_ji / r
//  * m r'' = f integrated by velocity Verlet (Sec. "Molecular dynamics")
//
// One thread owns one atom i and walks its Verlet list (full list, so no
// atomics and a fixed summation order).  The list is stored column-major
// in groups of 8 entries per atom (one 32-byte sector, two 16-byte loads per
// thread; a warp's loads of one group are 1 KB contiguous).  Neighbour positions come from the per-step gather copy,
// float4 (mixed) or 32-byte FP64 vectors, holding x - centre(cell): the pair
// vector is d = (p_j - p_i) + s h, s the stencil offset stored in the list
// entry, so FP32 pair math never subtracts two large coordinates.
//
// The velocity-Verlet update is fused into the force kernel's epilogue
// (second half-kick of step n, first half-kick and drift of step n+1), which
// also writes the next gather copy and raises the rebuild flag when an atom
// has moved more than skin/2 since the last build.  Reading pg[cur] while
// writing pg[cur^1] keeps the neighbours' positions of this step intact.
#include <math.h>

#include "mdk_internal.cuh"

namespace mdk {

namespace {

constexpr int kBlk = 256;
constexpr int kEamBlk = 512;

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
  // EAM tables: (y_k, h m_k) per knot for both passes
  using Tab1 = double2;
  using Tab2 = double2;
  static __device__ __forceinline__ const double2 *tab1(const EAMParams &e) { return e.rho64; }
  static __device__ __forceinline__ const double2 *phi2(const EAMParams &e) { return e.phi64; }
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
  static __device__ __forceinline__ double val2(const double2 *t, const EAMParams &, int k,
                                                double u) {
    const double2 a = t[k], b = t[k + 1];
    return herm_val<double>(u, a.x, a.y, b.x, b.y);
  }
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
  // pass 1 per interval (y_k, dy_k, h m_k, h m_{k+1}); pass 2 per knot (dy_k, h m_k)
  using Tab1 = float4;
  using Tab2 = float2;
  static __device__ __forceinline__ const float4 *tab1(const EAMParams &e) { return e.rho_i32; }
  static __device__ __forceinline__ const float2 *phi2(const EAMParams &e) { return e.phi_d32; }
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
  static __device__ __forceinline__ float val2(const float2 *t, const EAMParams &e, int k,
                                               float u) {
    const float2 a = t[k], b = t[k + 1];
    const float u2 = u * u, u3 = u2 * u;
    return __ldg(e.phi_v32 + k) + (3.0f * u2 - 2.0f * u3) * a.x + (u3 - 2.0f * u2 + u) * a.y +
           (u3 - u2) * b.y;
  }
};

// ---- the neighbour walk ------------------------------------------------------------
// Unit stencil offset s_d in {-1, 0, 1} of a list entry, exactly, in the pair
// precision, without an int-to-float conversion: the 2-bit code c = s_d + 1 is
// placed in the low mantissa bits of 2^23 (2^52) and 2^23 + 1 (2^52 + 1) is
// subtracted.
__device__ __forceinline__ float s_unit(float, uint32_t e, int d) {
  return __uint_as_float(((e >> (26 + 2 * d)) & 3u) | 0x4B000000u) - 8388609.0f;
}
__device__ __forceinline__ double s_unit(double, uint32_t e, int d) {
  return __longlong_as_double((long long)((e >> (26 + 2 * d)) & 3u) | 0x4330000000000000LL) -
         4503599627370497.0;
}

// Walk the list of one atom: a group of 8 list words comes in two 16-byte
// loads; its neighbour records are loaded four at a time before the four
// bodies run, so each thread keeps several independent loads in flight.
// `commit` runs after every four pairs: the compensated per-atom sums take one
// block sum per four pairs instead of one term per pair.
template <class Load, class Body, class Commit>
__device__ __forceinline__ void walk(const uint32_t *__restrict__ nbr, size_t Nc, int i, int nn,
                                     Load &&load, Body &&body, Commit &&commit) {
  using Rec = decltype(load(0u));
  const uint4 *__restrict__ row = reinterpret_cast<const uint4 *>(nbr) + (size_t)i * 2;
  const size_t gstride = Nc * 2;
  for (int k = 0; k < nn; k += kGroup, row += gstride) {
    const uint4 a = __ldcs(row), b = __ldcs(row + 1);
    const uint32_t e[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    const int m = nn - k;  // valid entries in this group
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      Rec q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (4 * h + u < m) q[u] = load(e[4 * h + u] & kJMask);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (4 * h + u < m) body(e[4 * h + u], q[u]);
      commit();
    }
  }
}

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

template <class P, int MODE, bool ENERGY>
__device__ __forceinline__ void epilogue(const Sys &s, const StepArgs &a, int i, uint32_t inf,
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

// ---- Lennard-Jones ---------------------------------------------------------------
template <class P, int MODE, bool ENERGY, int SHIFT>
__global__ void __launch_bounds__(kBlk) k_lj(Sys s, LJParams lp, StepArgs a) {
  using GP = G<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  const int N = s.st->N;
  const int i = blockIdx.x * kBlk + threadIdx.x;
  if (i >= N) return;
  const size_t Nc = s.N_cap;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const V pi = GP::ld(pg + i);
  const uint32_t inf = GP::info(pi);
  const Grid &g = s.grid[inf >> 8];
  R hx, hy, hz;
  GP::h(g, hx, hy, hz);
  const bool f64 = sizeof(R) == 8;
  const R rc2 = f64 ? (R)lp.rc2 : (R)lp.rc2f;
  const R sig2 = f64 ? (R)lp.sig2 : (R)lp.sig2f;
  const R eps24 = f64 ? (R)lp.eps24 : (R)lp.eps24f;
  const R eps4 = f64 ? (R)lp.eps4 : (R)lp.eps4f;
  const R ush = f64 ? (R)lp.u_shift : (R)lp.u_shiftf;
  const R durc = f64 ? (R)lp.du_rc : (R)lp.du_rcf;
  const R rcut = f64 ? (R)lp.rc : (R)lp.rcf;
  int nn = s.nnbr[i];
  if (nn > s.nmax) nn = s.nmax;
  Acc<R> fx, fy, fz;
  R e = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
  R bx = 0, by = 0, bz = 0;  // block sums of four pairs
  walk(
      s.nbr, Nc, i, nn, [&](uint32_t j) { return GP::ld(pg + j); },
      [&](uint32_t ent, const V &pj) {
        const R dx = (R)(pj.x - pi.x) + s_unit(R(0), ent, 0) * hx;
        const R dy = (R)(pj.y - pi.y) + s_unit(R(0), ent, 1) * hy;
        const R dz = (R)(pj.z - pi.z) + s_unit(R(0), ent, 2) * hz;
        const R r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < rc2) {
          const R inv = GP::rcp(r2);
          const R s2 = sig2 * inv;
          const R s6 = s2 * s2 * s2;
          R fr = -eps24 * (R(2) * s6 * s6 - s6) * inv;  // V'(r)/r
          R r = 0;
          if (SHIFT == 2) {
            r = GP::sqr(r2);
            fr -= durc / r;
          }
          bx += fr * dx;
          by += fr * dy;
          bz += fr * dz;
          if (ENERGY) {
            R v = eps4 * (s6 * s6 - s6) - ush;
            if (SHIFT == 2) v -= (r - rcut) * durc;
            e += R(0.5) * v;
            const R hf = R(-0.5) * fr;  // r_ij = -d
            w0 += hf * dx * dx;
            w1 += hf * dy * dy;
            w2 += hf * dz * dz;
            w3 += hf * dx * dy;
            w4 += hf * dx * dz;
            w5 += hf * dy * dz;
          }
        }
      },
      [&] {
        fx.add(bx);
        fy.add(by);
        fz.add(bz);
        bx = by = bz = 0;
      });
  if (ENERGY) {
    s.ea[i] = (double)e;
    s.wa[i] = w0;
    s.wa[Nc + i] = w1;
    s.wa[2 * Nc + i] = w2;
    s.wa[3 * Nc + i] = w3;
    s.wa[4 * Nc + i] = w4;
    s.wa[5 * Nc + i] = w5;
  }
  epilogue<P, MODE, ENERGY>(s, a, i, inf, fx.get(), fy.get(), fz.get());
}

// ---- EAM pass 1: densities, F(rho_i), F'(rho_i) -------------------------------------
template <class P, bool ENERGY>
__global__ void __launch_bounds__(kEamBlk) k_rho(Sys s, EAMParams ep, StepArgs a) {
  using GP = G<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  using T1 = typename GP::Tab1;
  extern __shared__ __align__(16) unsigned char smem[];
  T1 *rt = reinterpret_cast<T1 *>(smem);
  {
    const T1 *src = GP::tab1(ep);
    const int n = GP::n1(ep);
    for (int q = threadIdx.x; q < n; q += blockDim.x) rt[q] = src[q];
  }
  __syncthreads();
  const int N = s.st->N;
  const size_t Nc = s.N_cap;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const R rc2 = sizeof(R) == 8 ? (R)ep.rc2 : (R)ep.rc2f;
  const R inv_dr = sizeof(R) == 8 ? (R)ep.inv_dr : (R)ep.inv_drf;
  const int kmax = ep.nr - 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const V pi = GP::ld(pg + i);
    const uint32_t inf = GP::info(pi);
    const Grid &g = s.grid[inf >> 8];
    R hx, hy, hz;
    GP::h(g, hx, hy, hz);
    int nn = s.nnbr[i];
    if (nn > s.nmax) nn = s.nmax;
    Acc<R> rho;
    R br = 0;
    walk(
        s.nbr, Nc, i, nn, [&](uint32_t j) { return GP::ld(pg + j); },
        [&](uint32_t ent, const V &pj) {
          const R dx = (R)(pj.x - pi.x) + s_unit(R(0), ent, 0) * hx;
          const R dy = (R)(pj.y - pi.y) + s_unit(R(0), ent, 1) * hy;
          const R dz = (R)(pj.z - pi.z) + s_unit(R(0), ent, 2) * hz;
          const R r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < rc2) {
            const R r = GP::sqr(r2);
            const R u = r * inv_dr;
            int kk = (int)u;
            kk = kk > kmax ? kmax : kk;
            const R t = u - (R)kk;
            br += GP::val1(rt, kk, t);
          }
        },
        [&] {
          rho.add(br);
          br = 0;
        });
    const double rho_i = rho.get();
    // F(rho_i) and F'(rho_i) in FP64 (once per atom)
    double Fv, dF;
    if (rho_i > ep.rho_max) {
      // above the table: linear continuation of the last knot
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
      // inside (or below, by the first piece extended) the table
      const double u = rho_i * ep.inv_drho;
      int kk = (int)floor(u);
      kk = kk > ep.nrho - 2 ? ep.nrho - 2 : (kk < 0 ? 0 : kk);
      const double t = u - (double)kk;
      const double2 a0 = ep.F64[kk], a1 = ep.F64[kk + 1];
      Fv = herm_val<double>(t, a0.x, a0.y, a1.x, a1.y);
      dF = herm_der<double>(t, a0.x, a0.y, a1.x, a1.y) * ep.inv_drho;
    }
    s.rho[i] = rho_i;
    ((R *)s.fp)[i] = (R)dF;
    if (ENERGY) s.ea[i] = Fv;
  }
}

// ---- EAM pass 2: forces (+ integration) ----------------------------------------------
template <class P, int MODE, bool ENERGY>
__global__ void __launch_bounds__(kEamBlk) k_eam(Sys s, EAMParams ep, StepArgs a) {
  using GP = G<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  using T2 = typename GP::Tab2;
  extern __shared__ __align__(16) unsigned char smem[];
  T2 *pt = reinterpret_cast<T2 *>(smem);
  T2 *rt = pt + ep.nr;
  {
    const T2 *sp = GP::phi2(ep), *sr = GP::rho2(ep);
    for (int q = threadIdx.x; q < ep.nr; q += blockDim.x) {
      pt[q] = sp[q];
      rt[q] = sr[q];
    }
  }
  __syncthreads();
  const int N = s.st->N;
  const size_t Nc = s.N_cap;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const R *__restrict__ fpa = (const R *)s.fp;
  const R rc2 = sizeof(R) == 8 ? (R)ep.rc2 : (R)ep.rc2f;
  const R inv_dr = sizeof(R) == 8 ? (R)ep.inv_dr : (R)ep.inv_drf;
  const int kmax = ep.nr - 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const V pi = GP::ld(pg + i);
    const uint32_t inf = GP::info(pi);
    const Grid &g = s.grid[inf >> 8];
    R hx, hy, hz;
    GP::h(g, hx, hy, hz);
    const R fpi = fpa[i];
    int nn = s.nnbr[i];
    if (nn > s.nmax) nn = s.nmax;
    Acc<R> fx, fy, fz;
    R e = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    struct Rec {
      V p;
      R fp;
    };
    R bx = 0, by = 0, bz = 0;
    walk(
        s.nbr, Nc, i, nn,
        [&](uint32_t j) {
          Rec q;
          q.p = GP::ld(pg + j);
          q.fp = __ldg(fpa + j);
          return q;
        },
        [&](uint32_t ent, const Rec &q) {
          const V &pj = q.p;
          const R dx = (R)(pj.x - pi.x) + s_unit(R(0), ent, 0) * hx;
          const R dy = (R)(pj.y - pi.y) + s_unit(R(0), ent, 1) * hy;
          const R dz = (R)(pj.z - pi.z) + s_unit(R(0), ent, 2) * hz;
          const R r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < rc2) {
            const R inv_r = GP::rsq(r2);
            const R r = r2 * inv_r;
            const R u = r * inv_dr;
            int kk = (int)u;
            kk = kk > kmax ? kmax : kk;
            const R t = u - (R)kk;
            const R dphi = GP::der2(pt, kk, t) * inv_dr;
            const R drho = GP::der2(rt, kk, t) * inv_dr;
            const R fr = (dphi + (fpi + q.fp) * drho) * inv_r;  // V'(r)/r
            bx += fr * dx;
            by += fr * dy;
            bz += fr * dz;
            if (ENERGY) {
              e += R(0.5) * GP::val2(pt, ep, kk, t);
              const R hf = R(-0.5) * fr;
              w0 += hf * dx * dx;
              w1 += hf * dy * dy;
              w2 += hf * dz * dz;
              w3 += hf * dx * dy;
              w4 += hf * dx * dz;
              w5 += hf * dy * dz;
            }
          }
        },
        [&] {
          fx.add(bx);
          fy.add(by);
          fz.add(bz);
          bx = by = bz = 0;
        });
    if (ENERGY) {
      s.ea[i] = s.ea[i] + (double)e;
      s.wa[i] = w0;
      s.wa[Nc + i] = w1;
      s.wa[2 * Nc + i] = w2;
      s.wa[3 * Nc + i] = w3;
      s.wa[4 * Nc + i] = w4;
      s.wa[5 * Nc + i] = w5;
    }
    epilogue<P, MODE, ENERGY>(s, a, i, inf, fx.get(), fy.get(), fz.get());
  }
}

// ---- first half-kick + drift from the stored forces ---------------------------------
template <class P>
__global__ void __launch_bounds__(kBlk) k_kick_drift(Sys s, StepArgs a) {
  const int N = s.st->N;
  const int i = blockIdx.x * kBlk + threadIdx.x;
  if (i >= N) return;
  const size_t Nc = s.N_cap;
  const uint32_t inf = s.info[i];
  const int type = inf & 15u;
  double vx = s.v[i], vy = s.v[Nc + i], vz = s.v[2 * Nc + i];
  if (inf & kInfoPiston) {
    vx = s.u_p;
    vy = 0.0;
    vz = 0.0;
  } else {
    const double c = 0.5 * a.dt * s.acc_over_m[type];
    vx += c * s.f[i];
    vy += c * s.f[Nc + i];
    vz += c * s.f[2 * Nc + i];
  }
  drift_publish<P>(s, a, i, inf, vx, vy, vz);
}

// ---- deterministic per-replica sums (fixed order, no atomics) -----------------------
constexpr int kRedThreads = 1024;
__global__ void __launch_bounds__(kRedThreads) k_reduce(Sys s, int with_ke) {
  const int r = blockIdx.x;
  const Grid &g = s.grid[r];
  const int a0 = g.atom_off;
  const int n = (s.n_rep == 1) ? s.st->N : g.n_atoms;
  const size_t Nc = s.N_cap;
  double acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0.0;
  for (int q = threadIdx.x; q < n; q += kRedThreads) {
    const int i = a0 + q;
    acc[0] += with_ke ? s.ka[i] : 0.0;
    acc[1] += s.ea[i];
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[2 + c] += s.wa[c * Nc + i];
  }
  __shared__ double sh[kRedThreads];
  for (int c = 0; c < 8; ++c) {
    sh[threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) s.red[r * 9 + c] = sh[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) s.red[r * 9 + 8] = (double)n;
}

// ---- state in / out in the caller's order -------------------------------------------
template <class P>
__global__ void __launch_bounds__(kBlk) k_load_state(Sys s, const double *x, const double *v,
                                                     int target_pg) {
  const int N = s.st->N;
  const int i = blockIdx.x * kBlk + threadIdx.x;
  if (i >= N) return;
  const size_t Nc = s.N_cap;
  for (int d = 0; d < 3; ++d) {
    s.x[d * Nc + i] = x[3 * (size_t)i + d];
    s.v[d * Nc + i] = v ? v[3 * (size_t)i + d] : 0.0;
    s.f[d * Nc + i] = 0.0;
  }
  s.id[i] = i;
  s.info[i] = s.info0[i];
}

__global__ void __launch_bounds__(kBlk) k_store_state(Sys s, double *x, double *v) {
  const int N = s.st->N;
  const int i = blockIdx.x * kBlk + threadIdx.x;
  if (i >= N) return;
  const size_t Nc = s.N_cap;
  const size_t o = (size_t)s.id[i];
  for (int d = 0; d < 3; ++d) {
    if (x) x[3 * o + d] = s.x[d * Nc + i];
    if (v) v[3 * o + d] = s.v[d * Nc + i];
  }
}

__global__ void __launch_bounds__(kBlk) k_store_forces(Sys s, double *f) {
  const int N = s.st->N;
  const int i = blockIdx.x * kBlk + threadIdx.x;
  if (i >= N) return;
  const size_t Nc = s.N_cap;
  const size_t o = (size_t)s.id[i];
  for (int d = 0; d < 3; ++d) f[3 * o + d] = s.f[d * Nc + i];
}

__global__ void __launch_bounds__(kBlk) k_store_per_atom(Sys s, double *ua, double *wa) {
  const int N = s.st->N;
  const int i = blockIdx.x * kBlk + threadIdx.x;
  if (i >= N) return;
  const size_t Nc = s.N_cap;
  const size_t o = (size_t)s.id[i];
  if (ua) ua[o] = s.ea[i];
  if (wa)
    for (int c = 0; c < 6; ++c) wa[6 * o + c] = s.wa[c * Nc + i];
}



// ---- EAM tables: knot slopes (3-point differences) -> (y, h*m) per knot --------------
__device__ __forceinline__ double hslope(const double *y, int n, int k) {
  if (k == 0) return 0.5 * (-3.0 * y[0] + 4.0 * y[1] - y[2]);
  if (k == n - 1) return 0.5 * (3.0 * y[n - 1] - 4.0 * y[n - 2] + y[n - 3]);
  return 0.5 * (y[k + 1] - y[k - 1]);
}

__global__ void k_eam_prepare(int nr, int nrho, const double *phi, const double *rho,
                              const double *F, EAMTablesDev o) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nr) {
    const double mp = hslope(phi, nr, k), mr = hslope(rho, nr, k);
    o.phi64[k] = make_double2(phi[k], mp);
    o.rho64[k] = make_double2(rho[k], mr);
    const double dp = k + 1 < nr ? phi[k + 1] - phi[k] : 0.0;
    const double dr = k + 1 < nr ? rho[k + 1] - rho[k] : 0.0;
    o.phi_d32[k] = make_float2((float)dp, (float)mp);
    o.rho_d32[k] = make_float2((float)dr, (float)mr);
    o.phi_v32[k] = (float)phi[k];
    if (k + 1 < nr)
      o.rho_i32[k] = make_float4((float)rho[k], (float)dr, (float)mr, (float)hslope(rho, nr, k + 1));
  }
  if (k < nrho) o.F64[k] = make_double2(F[k], hslope(F, nrho, k));
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

template <class P, int MODE, bool EN>
void lj_disp(const Sys &s, const LJParams &p, StepArgs a, cudaStream_t st) {
  const int g = nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk);
  switch (p.shift_mode) {
    case 2:
      k_lj<P, MODE, EN, 2><<<g, kBlk, 0, st>>>(s, p, a);
      break;
    default:
      k_lj<P, MODE, EN, 1><<<g, kBlk, 0, st>>>(s, p, a);
      break;
  }
}

template <class P, int MODE>
void lj_mode(const Sys &s, const LJParams &p, StepArgs a, cudaStream_t st) {
  if (a.energy)
    lj_disp<P, MODE, true>(s, p, a, st);
  else
    lj_disp<P, MODE, false>(s, p, a, st);
}

template <class P>
void lj_prec(const Sys &s, const LJParams &p, Mode m, StepArgs a, cudaStream_t st) {
  if (m == kForceOnly)
    lj_mode<P, kForceOnly>(s, p, a, st);
  else if (m == kStep)
    lj_mode<P, kStep>(s, p, a, st);
  else
    lj_mode<P, kFinal>(s, p, a, st);
}

int g_sm_count = 0;
int g_eam_grid[2][2] = {{0, 0}, {0, 0}};  // [precision][pass]

int sm_count() {
  if (g_sm_count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (g_sm_count <= 0) g_sm_count = 1;
  }
  return g_sm_count;
}

template <class P, int MODE, bool EN>
void eam_run(const Sys &s, const EAMParams &p, StepArgs a, int prec, cudaStream_t st) {
  const int b1 = eam_smem_bytes(p, prec, 1), b2 = eam_smem_bytes(p, prec, 2);
  const int g1 = g_eam_grid[prec][0] > 0 ? g_eam_grid[prec][0] : sm_count();
  const int g2 = g_eam_grid[prec][1] > 0 ? g_eam_grid[prec][1] : sm_count();
  k_rho<P, EN><<<g1, kEamBlk, b1, st>>>(s, p, a);
  k_eam<P, MODE, EN><<<g2, kEamBlk, b2, st>>>(s, p, a);
}

template <class P>
void eam_prec(const Sys &s, const EAMParams &p, Mode m, StepArgs a, int prec,
              cudaStream_t st) {
  if (m == kForceOnly) {
    if (a.energy)
      eam_run<P, kForceOnly, true>(s, p, a, prec, st);
    else
      eam_run<P, kForceOnly, false>(s, p, a, prec, st);
  } else if (m == kStep) {
    if (a.energy)
      eam_run<P, kStep, true>(s, p, a, prec, st);
    else
      eam_run<P, kStep, false>(s, p, a, prec, st);
  } else {
    if (a.energy)
      eam_run<P, kFinal, true>(s, p, a, prec, st);
    else
      eam_run<P, kFinal, false>(s, p, a, prec, st);
  }
}

template <class P>
int set_attr_all(int b1, int b2) {
  cudaError_t e = cudaSuccess;
#define MDK_ATTR(K, B)                                                                   \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, B);
  MDK_ATTR((k_rho<P, true>), b1)
  MDK_ATTR((k_rho<P, false>), b1)
  MDK_ATTR((k_eam<P, kForceOnly, true>), b2)
  MDK_ATTR((k_eam<P, kForceOnly, false>), b2)
  MDK_ATTR((k_eam<P, kStep, true>), b2)
  MDK_ATTR((k_eam<P, kStep, false>), b2)
  MDK_ATTR((k_eam<P, kFinal, true>), b2)
  MDK_ATTR((k_eam<P, kFinal, false>), b2)
#undef MDK_ATTR
  if (e != cudaSuccess) return -1;
  // persistent grids: as many resident blocks as the SMs hold
  int o1 = 0, o2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_rho<P, false>, kEamBlk, b1);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_eam<P, kStep, false>, kEamBlk, b2);
  const int p = sizeof(typename G<P>::R) == 8 ? 0 : 1;
  g_eam_grid[p][0] = sm_count() * (o1 > 0 ? o1 : 1);
  g_eam_grid[p][1] = sm_count() * (o2 > 0 ? o2 : 1);
  return 0;
}

}  // namespace

int eam_smem_bytes(const EAMParams &p, int precision, int pass) {
  if (precision == 0) return (pass == 1 ? 1 : 2) * p.nr * (int)sizeof(double2);
  return pass == 1 ? (p.nr - 1) * (int)sizeof(float4) : 2 * p.nr * (int)sizeof(float2);
}

int configure_eam_smem(int b1, int b2, int precision) {
  return precision == 0 ? set_attr_all<Fp64>(b1, b2) : set_attr_all<Mixed>(b1, b2);
}

void launch_lj(const Sys &s, const LJParams &p, int precision, Mode mode, StepArgs a,
               cudaStream_t st) {
  if (precision == 0)
    lj_prec<Fp64>(s, p, mode, a, st);
  else
    lj_prec<Mixed>(s, p, mode, a, st);
}

void launch_eam(const Sys &s, const EAMParams &p, int precision, Mode mode, StepArgs a,
                cudaStream_t st) {
  if (precision == 0)
    eam_prec<Fp64>(s, p, mode, a, 0, st);
  else
    eam_prec<Mixed>(s, p, mode, a, 1, st);
}

void launch_kick_drift(const Sys &s, int precision, StepArgs a, cudaStream_t st) {
  const int g = nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk);
  if (precision == 0)
    k_kick_drift<Fp64><<<g, kBlk, 0, st>>>(s, a);
  else
    k_kick_drift<Mixed><<<g, kBlk, 0, st>>>(s, a);
}

void launch_reduce(const Sys &s, int with_ke, cudaStream_t st) {
  k_reduce<<<s.n_rep, kRedThreads, 0, st>>>(s, with_ke);
}

void launch_eam_prepare(const EAMParams &p, const double *phi, const double *rho,
                        const double *F, EAMTablesDev out, cudaStream_t st) {
  const int n = p.nr > p.nrho ? p.nr : p.nrho;
  k_eam_prepare<<<nblk(n, 256), 256, 0, st>>>(p.nr, p.nrho, phi, rho, F, out);
}

void launch_load_state(const Sys &s, const double *x, const double *v, int precision,
                       int target_pg, cudaStream_t st) {
  const int g = nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk);
  if (precision == 0)
    k_load_state<Fp64><<<g, kBlk, 0, st>>>(s, x, v, target_pg);
  else
    k_load_state<Mixed><<<g, kBlk, 0, st>>>(s, x, v, target_pg);
}

void launch_store_state(const Sys &s, double *x, double *v, cudaStream_t st) {
  k_store_state<<<nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk), kBlk, 0, st>>>(s, x, v);
}

void launch_store_forces(const Sys &s, double *f, cudaStream_t st) {
  k_store_forces<<<nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk), kBlk, 0, st>>>(s, f);
}

void launch_store_per_atom(const Sys &s, double *ua, double *wa, cudaStream_t st) {
  k_store_per_atom<<<nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk), kBlk, 0, st>>>(s, ua, wa);
}



}  // namespace mdk
