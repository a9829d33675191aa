// k_bpnn.cu -- Behler-Parrinello neural-network forces (GB300, sm_103a).
//
// Paper passages (Sec. "Molecular dynamics with Behler-Parrinello neural
// networks"): E = sum_i E_i (Eq. E_as_sum); atom i's network input is a set
// of radial (Eqs. G1-G3) and angular (Eqs. G4, G5) symmetry functions of its
// neighbourhood within R_c, cut off by f_c(R) = 1/2 [cos(pi R / R_c) + 1];
// E_i comes from a two-hidden-layer network (Eq. AtomicNN: tanh, tanh,
// linear output); the forces follow Eq. force, F_k = -sum_i sum_mu
// dE_i/dG_mu(i) dG_mu(i)/dR_k, with dE_i/dG from the network's reverse pass
// and dG/dR analytic.  G2 is read with the square, (R - R_s)^2; angular sums
// run over unordered pairs of distinct neighbours.
//
// One warp per atom i:
//  1. the list entries within R_c are compacted into the warp's shared slab:
//     pair vector u_a, R_a, f_c(R_a), f_c'(R_a) and exp(-eta_p R_a^2) for
//     every (eta, kind) group p of the angular functions;
//  2. radial functions, lanes over neighbours; angular functions, lanes over
//     unordered pairs {a, b}; warp sums;
//  3. the network forward and reverse pass (lanes over hidden units, weights
//     staged in shared memory per block) gives E_i and dE_i/dG;
//  4. the gradients g_a = dE_i/dR_(j_a): every unordered pair {a, b} is
//     evaluated once and gives, for its angular terms T(u_a, u_b, s = u_b -
//     u_a), dT/du_a - dT/ds to a and dT/du_b + dT/ds to b.  The pairs run in
//     a rotation schedule -- round k pairs a with (a + k) mod n -- so in one
//     warp instruction no two lanes touch the same neighbour's shared sums
//     (no atomics, and a fixed summation order: reproducible).  Per pair the
//     angular functions are folded group by group: for each (eta, kind)
//     group the sums over its functions of w A and w dA/dc (w = dE_i/dG)
//     multiply the group's Gaussian-cutoff factor and its derivatives.
//     Atom j_a receives -g_a, atom i receives sum_a g_a (E_i depends on
//     relative positions only), and i keeps the virial -sum_a u_a (x) g_a of
//     its own energy.  Forces are added to the per-atom
// accumulators s.hacc (64-bit fixed point in the mixed path, FP64 atomics in
// the FP64 path); launch_half_fin then finishes the step.  The mixed path
// computes in FP32; a neighbour gradient at or above 2^22 eV/A sets the
// non-finite status.
#include "k_pair.cuh"

namespace mdk {
namespace {

using namespace pair;

template <class R>
struct BM;
template <>
struct BM<float> {
  // x in [0, 1] here (R < R_c): the hardware sine/cosine of pi x are within
  // ~1e-6 absolute, far inside the mixed path's bar
  static __device__ __forceinline__ void scpi(float x, float *s, float *c) {
    __sincosf(3.14159265358979f * x, s, c);
  }
  static __device__ __forceinline__ float ex(float x) { return __expf(x); }
  static __device__ __forceinline__ float th(float x) { return tanhf(x); }
  static __device__ __forceinline__ float sq(float x) { return sqrtf(x); }
  static __device__ __forceinline__ void sc(float x, float *s, float *c) { sincosf(x, s, c); }
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
};
template <>
struct BM<double> {
  static __device__ __forceinline__ void scpi(double x, double *s, double *c) {
    sincospi(x, s, c);
  }
  static __device__ __forceinline__ double ex(double x) { return exp(x); }
  static __device__ __forceinline__ double th(double x) { return tanh(x); }
  static __device__ __forceinline__ double sq(double x) { return sqrt(x); }
  static __device__ __forceinline__ void sc(double x, double *s, double *c) { sincos(x, s, c); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
};

// a parameter in the pair precision
template <class R>
__device__ __forceinline__ R pick(double d, float f) {
  return sizeof(R) == 8 ? (R)d : (R)f;
}

// x^e for a small non-negative integer e (uniform across the warp)
template <class R>
__device__ __forceinline__ R ipow(R x, int e) {
  R r = R(1);
  while (e) {
    if (e & 1) r *= x;
    x *= x;
    e >>= 1;
  }
  return r;
}

// the 2 kBpZ per-slot weights of one (eta, kind) group, with vector loads
template <class R>
__device__ __forceinline__ void ld_group(const R *w, R out[2 * kBpZ]) {
  if (sizeof(R) == 4) {
    const float4 *q = reinterpret_cast<const float4 *>(w);
#pragma unroll
    for (int v = 0; v < kBpZ / 2; ++v) {
      const float4 a = q[v];
      out[4 * v] = a.x;
      out[4 * v + 1] = a.y;
      out[4 * v + 2] = a.z;
      out[4 * v + 3] = a.w;
    }
  } else {
    const double2 *q = reinterpret_cast<const double2 *>(w);
#pragma unroll
    for (int v = 0; v < kBpZ; ++v) {
      const double2 a = q[v];
      out[2 * v] = a.x;
      out[2 * v + 1] = a.y;
    }
  }
}

// x^e and y^e together (one loop, uniform across the warp)
template <class R>
__device__ __forceinline__ void ipow2(R x, R y, int e, R &rx, R &ry) {
  rx = R(1);
  ry = R(1);
  while (e) {
    if (e & 1) {
      rx *= x;
      ry *= y;
    }
    x *= x;
    y *= y;
    e >>= 1;
  }
}

// Powers of the angular term per zeta group: x = 1 + c, y = 1 - c.  ZS = 1
// is the zeta set {1, 2, 4, 16} (zeta group z holds zeta = 1, 2, 4, 16): the
// powers come from one ladder of squares; ZS = 0 takes any integer zeta.
// The 2^(1 - zeta) factors are applied outside the pair loops (descriptor
// sums and reverse-pass weights), a power-of-two scaling, so exact.
// x^zeta, y^zeta (descriptor pass)
template <class R, int ZS>
__device__ __forceinline__ void zeta_pow(const BPParams &bp, R x, R y, R px[kBpZ], R py[kBpZ]) {
  if (ZS == 1) {
    const R x2 = x * x, x4 = x2 * x2, x8 = x4 * x4;
    const R y2 = y * y, y4 = y2 * y2, y8 = y4 * y4;
    px[0] = x;
    py[0] = y;
    px[1] = x2;
    py[1] = y2;
    px[2] = x4;
    py[2] = y4;
    px[3] = x8 * x8;
    py[3] = y8 * y8;
  } else {
#pragma unroll
    for (int z = 0; z < kBpZ; ++z) {
      ipow2<R>(x, y, bp.z_pow[z], px[z], py[z]);
      px[z] *= x;
      py[z] *= y;
    }
  }
}
// x^(zeta - 1), y^(zeta - 1) (reverse pass: A = x^(zeta-1) x, dA/dc = zeta x^(zeta-1))
template <class R, int ZS>
__device__ __forceinline__ void zeta_pow_m1(const BPParams &bp, R x, R y, R px[kBpZ],
                                            R py[kBpZ]) {
  if (ZS == 1) {
    const R x2 = x * x, x4 = x2 * x2, x8 = x4 * x4;
    const R y2 = y * y, y4 = y2 * y2, y8 = y4 * y4;
    px[0] = R(1);
    py[0] = R(1);
    px[1] = x;
    py[1] = y;
    px[2] = x2 * x;
    py[2] = y2 * y;
    px[3] = (x8 * x4) * (x2 * x);
    py[3] = (y8 * y4) * (y2 * y);
  } else {
#pragma unroll
    for (int z = 0; z < kBpZ; ++z) ipow2<R>(x, y, bp.z_pow[z], px[z], py[z]);
  }
}

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// per-warp shared slab: per neighbour slot two 4-vectors -- (u_x, u_y, u_z,
// R) and (1/R, f_c, f_c', 0) -- so a pair's operands come in few vector loads,
// the gradient sums (SoA), the exponentials of the (eta, kind) groups in
// pairs of groups ([nY/2][NB][2]); then the descriptor / gradient / hidden
// vectors
template <class R>
struct Slab {
  R *u4, *f4, *e;
  R *gax, *gay, *gaz, *gbx, *gby, *gbz;  // gradient sums (a side, b side)
  int *j;
  R *G, *dG, *h1, *d1, *d2, *wc;  // wc: dE/dG of each angular slot
};
constexpr int kSlabFields = 14;   // per-neighbour reals besides e

template <class R>
struct Q4 {
  R x, y, z, w;
};
// 4 consecutive reals (16-byte aligned for float, 32 for double)
template <class R>
__device__ __forceinline__ Q4<R> ld4(const R *p) {
  if constexpr (sizeof(R) == 4) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {v.x, v.y, v.z, v.w};
  } else {
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    return {a.x, a.y, b.x, b.y};
  }
}
// the exponentials of groups 2k and 2k + 1 at slot q
template <class R>
__device__ __forceinline__ void ld_e2(const R *e, int NB, int k, int q, R &e0, R &e1) {
  if constexpr (sizeof(R) == 4) {
    const float2 v = reinterpret_cast<const float2 *>(e + (size_t)2 * k * NB)[q];
    e0 = v.x;
    e1 = v.y;
  } else {
    const double2 v = reinterpret_cast<const double2 *>(e + (size_t)2 * k * NB)[q];
    e0 = v.x;
    e1 = v.y;
  }
}

constexpr int kVec = 80;  // >= kBpIn, a multiple of 16
static_assert(kVec >= kBpIn, "device network inputs");

template <class R>
__device__ __forceinline__ Slab<R> slab_at(char *base, int NB, int nY) {
  Slab<R> s;
  R *p = reinterpret_cast<R *>(base);
  s.u4 = p;
  s.f4 = p + 4 * NB;
  s.gax = p + 8 * NB;
  s.gay = p + 9 * NB;
  s.gaz = p + 10 * NB;
  s.gbx = p + 11 * NB;
  s.gby = p + 12 * NB;
  s.gbz = p + 13 * NB;
  s.e = p + kSlabFields * NB;
  p += (size_t)(kSlabFields + nY) * NB;
  s.G = p;
  s.dG = p + kVec;
  s.h1 = p + 2 * kVec;
  s.d1 = p + 2 * kVec + 32;
  s.d2 = p + 2 * kVec + 64;
  s.wc = p + 2 * kVec + 96;
  s.j = reinterpret_cast<int *>(p + 2 * kVec + 96 + kBpSlots);
  return s;
}

__host__ __device__ inline size_t slab_bytes(int NB, int nY, size_t rsz) {
  size_t b = rsz * ((size_t)(kSlabFields + nY) * NB + 2 * kVec + 96 + kBpSlots) +
             sizeof(int) * (size_t)NB;
  return (b + 15) / 16 * 16;
}

// radial symmetry function m at R (f = f_c(R), df = f_c'(R)): value and
// derivative
template <class R>
__device__ __forceinline__ void radial(const BPParams &bp, int m, R r, R f, R df, R &val,
                                       R &der) {
  const int kind = bp.rad_kind[m];
  const R p0 = pick<R>(bp.rad_p0[m], bp.rad_p0f[m]);
  if (kind == 1) {
    val = f;
    der = df;
  } else if (kind == 2) {
    const R p1 = pick<R>(bp.rad_p1[m], bp.rad_p1f[m]);
    const R t = r - p1;
    const R e = BM<R>::ex(-p0 * t * t);
    val = e * f;
    der = e * (R(-2) * p0 * t * f + df);
  } else {
    R sn, cs;
    BM<R>::sc(p0 * r, &sn, &cs);
    val = cs * f;
    der = -p0 * sn * f + cs * df;
  }
}

// mixed: 8 warps per block, two blocks per SM (128 registers); FP64: 4 warps
template <class P>
constexpr int bp_threads() {
  return sizeof(typename G<P>::R) == 4 ? 256 : 128;
}
template <class P>
constexpr int bp_blocks() {
  return sizeof(typename G<P>::R) == 4 ? 2 : 1;
}

// NY: the (eta, kind) groups the kernel is compiled for (nY rounded up to an
// even number); the padded groups carry zero exponentials, and slots without
// a function zero weights, so the pair loops run without per-group guards.
// ZS: the zeta set (zeta_pow).
template <class P, bool ENERGY, int NY, int ZS>
__global__ void __launch_bounds__(bp_threads<P>(), bp_blocks<P>())
    k_bpnn(Sys s, BPParams bp, StepArgs a) {
  using GP = G<P>;
  using H = HalfAcc<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  extern __shared__ __align__(16) char smem[];
  const int N = run_n(s.st);
  const size_t Nc = s.N_cap;
  const int NB = s.nmax;
  const int nY = bp.nY, nr = bp.n_rad, H1 = bp.H1, H2 = bp.H2;
  constexpr int NS = 2 * NY * kBpZ;  // angular slots of the compiled groups
  constexpr int n_in = kBpIn;
  const unsigned long long used = bp.slot_mask;
  const R rc = pick<R>(bp.rc, bp.rcf), rc2 = rc * rc, inv_rc = R(1) / rc;
  const R half_pi_rc = R(-0.5) * R(3.14159265358979323846) * inv_rc;
  // weights, once per block
  const int nW = n_in * H1 + H1 + H1 * H2 + 2 * H2;
  R *Wsm = reinterpret_cast<R *>(smem);
  {
    const R *src = sizeof(R) == 8 ? reinterpret_cast<const R *>(bp.w64)
                                  : reinterpret_cast<const R *>(bp.w32);
    for (int q = threadIdx.x; q < nW; q += blockDim.x) Wsm[q] = src[q];
  }
  __syncthreads();
  const R *W01 = Wsm, *b1 = W01 + n_in * H1, *W12 = b1 + H1, *b2 = W12 + H1 * H2,
          *w23 = b2 + H2;
  const size_t wbytes = ((size_t)nW * sizeof(R) + 15) / 16 * 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Slab<R> sl = slab_at<R>(smem + wbytes + (size_t)warp * slab_bytes(NB, NY, sizeof(R)), NB, NY);
  const int i = blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= N) return;  // whole warps leave together

  // ---- 1. the neighbourhood within R_c ----------------------------------
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const V pi = GP::ld(pg + i);
  R hx, hy, hz;
  GP::h(s.grid[GP::info(pi) >> 8], hx, hy, hz);
  h_scaled(hx, hy, hz);  // for s_scaled
  const int nn = min(s.nnbr[i], s.nmax);
  int n = 0;
  for (int k0 = 0; k0 < nn; k0 += 32) {
    const int k = k0 + lane;
    bool keep = false;
    R dx = 0, dy = 0, dz = 0, r2 = 0;
    uint32_t j = 0;
    if (k < nn) {
      const uint32_t ent = s.nbr[ell_index(k, i, Nc)];
      j = dbg_idx(s, nbr_j(ent), Nc, i);
      const V pj = GP::ld(pg + j);
      dx = pvec((R)pj.x, (R)pi.x, s_scaled(R(0), ent, 0), hx);
      dy = pvec((R)pj.y, (R)pi.y, s_scaled(R(0), ent, 1), hy);
      dz = pvec((R)pj.z, (R)pi.z, s_scaled(R(0), ent, 2), hz);
      r2 = r2_of(dx, dy, dz);
      keep = r2 < rc2;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int q = n + __popc(m & ((1u << lane) - 1u));
      const R r = BM<R>::sq(r2);
      R sn, cs;
      BM<R>::scpi(r * inv_rc, &sn, &cs);
      R *u = sl.u4 + 4 * q, *f = sl.f4 + 4 * q;
      u[0] = dx;
      u[1] = dy;
      u[2] = dz;
      u[3] = r;
      f[0] = BM<R>::rcp(r);
      f[1] = R(0.5) * (cs + R(1));
      f[2] = half_pi_rc * sn;
      f[3] = R(0);
      sl.gax[q] = sl.gay[q] = sl.gaz[q] = R(0);
      sl.gbx[q] = sl.gby[q] = sl.gbz[q] = R(0);
#pragma unroll
      for (int p = 0; p < NY; ++p)
        sl.e[(size_t)2 * (p >> 1) * NB + 2 * q + (p & 1)] =
            p < nY ? BM<R>::ex(-pick<R>(bp.y_eta[p], bp.y_etaf[p]) * r2) : R(0);
      sl.j[q] = (int)j;
    }
    n += __popc(m);
  }
  __syncwarp();

  // ---- 2. symmetry functions ----------------------------------------------
  R accr[kBpRad];
#pragma unroll
  for (int m = 0; m < kBpRad; ++m) accr[m] = 0;
  for (int q = lane; q < n; q += 32) {
    const R r = sl.u4[4 * q + 3];
    const Q4<R> fq = ld4<R>(sl.f4 + 4 * q);
    const R f = fq.y, df = fq.z;
#pragma unroll
    for (int m = 0; m < kBpRad; ++m)
      if (m < nr) {
        R v, d;
        radial<R>(bp, m, r, f, df, v, d);
        accr[m] += v;
      }
  }
  R acca[NS];
#pragma unroll
  for (int m = 0; m < NS; ++m) acca[m] = 0;
  {
    const int npair = n * (n - 1) / 2;
    int qa = 0, rel = lane;  // pair t = (qa, qa + 1 + rel), rows in order of qa
    while (qa < n - 1 && rel >= n - 1 - qa) {
      rel -= n - 1 - qa;
      ++qa;
    }
    for (int t = lane; t < npair; t += 32) {
      const int qb = qa + 1 + rel;
      const Q4<R> ua = ld4<R>(sl.u4 + 4 * qa), ub = ld4<R>(sl.u4 + 4 * qb);
      const Q4<R> va = ld4<R>(sl.f4 + 4 * qa), vb = ld4<R>(sl.f4 + 4 * qb);
      const R ax = ua.x, ay = ua.y, az = ua.z, fa = va.y;
      const R bx = ub.x, by = ub.y, bz = ub.z, fb = vb.y;
      const R c = (ax * bx + ay * by + az * bz) * (va.x * vb.x);
      const R sx = bx - ax, sy = by - ay, sz = bz - az;
      const R rab2 = sx * sx + sy * sy + sz * sz;
      const bool near = bp.any4 && rab2 < rc2;
      R fab = 0;
      if (near) {
        R sn, cs;
        BM<R>::scpi(BM<R>::sq(rab2) * inv_rc, &sn, &cs);
        fab = R(0.5) * (cs + R(1));
      }
      R Y[NY];
#pragma unroll
      for (int p = 0; p < NY; p += 2) {
        R ea0, ea1, eb0, eb1;
        ld_e2<R>(sl.e, NB, p >> 1, qa, ea0, ea1);
        ld_e2<R>(sl.e, NB, p >> 1, qb, eb0, eb1);
        Y[p] = ea0 * eb0;
        Y[p + 1] = ea1 * eb1;
      }
      const R fab2 = fa * fb;
#pragma unroll
      for (int p = 0; p < NY; ++p) {
        Y[p] *= fab2;
        if (bp.y_kind[p] == 4)
          Y[p] = near ? Y[p] * BM<R>::ex(-pick<R>(bp.y_eta[p], bp.y_etaf[p]) * rab2) * fab
                      : R(0);
      }
      // (1 +- c)^zeta per zeta group (the factor 2^(1 - zeta) is applied to the sums)
      R Pp[kBpZ], Pm[kBpZ];
      zeta_pow<R, ZS>(bp, R(1) + c, R(1) - c, Pp, Pm);
      // every slot of the used groups (a slot without a function has zero
      // weights, so its sum is never read)
#pragma unroll
      for (int p = 0; p < NY; ++p)
#pragma unroll
        for (int z = 0; z < kBpZ; ++z) {
          const int m = (p * kBpZ + z) * 2;
          acca[m] += Pp[z] * Y[p];
          acca[m + 1] += Pm[z] * Y[p];
        }
      rel += 32;
      while (qa < n - 1 && rel >= n - 1 - qa) {
        rel -= n - 1 - qa;
        ++qa;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kBpRad; ++m)
    if (m < nr) accr[m] = warp_sum(accr[m]);
#pragma unroll
  for (int m = 0; m < NS; ++m)
    if ((used >> m) & 1ull)
      acca[m] = warp_sum(acca[m]) *
                pick<R>(bp.z_coef[(m >> 1) % kBpZ], bp.z_coeff[(m >> 1) % kBpZ]);
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < kBpRad; ++m) sl.G[m] = m < nr ? accr[m] : R(0);
#pragma unroll
    for (int m = 0; m < kBpSlots; ++m)
      sl.G[kBpRad + m] = (m < NS && ((used >> m) & 1ull)) ? acca[m < NS ? m : 0] : R(0);
  }
  __syncwarp();

  // ---- 3. the atomic network and its reverse pass -------------------------
  R h1 = 0;
  if (lane < H1) {
    R z = b1[lane];
    for (int m = 0; m < n_in; ++m) z += sl.G[m] * W01[m * H1 + lane];
    h1 = BM<R>::th(z);
  }
  sl.h1[lane] = h1;
  __syncwarp();
  R h2 = 0;
  if (lane < H2) {
    R z = b2[lane];
    for (int q = 0; q < H1; ++q) z += sl.h1[q] * W12[q * H2 + lane];
    h2 = BM<R>::th(z);
  }
  const R Ei = warp_sum(lane < H2 ? h2 * w23[lane] : R(0)) + pick<R>(bp.b3, bp.b3f);
  sl.d2[lane] = lane < H2 ? w23[lane] * (R(1) - h2 * h2) : R(0);
  __syncwarp();
  R d1 = 0;
  if (lane < H1) {
    for (int q = 0; q < H2; ++q) d1 += W12[lane * H2 + q] * sl.d2[q];
    d1 *= R(1) - h1 * h1;
  }
  sl.d1[lane] = d1;
  __syncwarp();
  for (int m = lane; m < n_in; m += 32) {
    R t = 0;
    for (int q = 0; q < H1; ++q) t += W01[m * H1 + q] * sl.d1[q];
    sl.dG[m] = t;
    if (m >= kBpRad) {
      const int z = ((m - kBpRad) >> 1) % kBpZ;
      sl.wc[m - kBpRad] = t * pick<R>(bp.z_coef[z], bp.z_coeff[z]);
    }
  }
  __syncwarp();

  // ---- 4. gradients with respect to the neighbours ------------------------
  {
    auto grad_pair = [&](const int qa, const int qb) {
      const Q4<R> ua = ld4<R>(sl.u4 + 4 * qa), ub = ld4<R>(sl.u4 + 4 * qb);
      const Q4<R> va = ld4<R>(sl.f4 + 4 * qa), vb = ld4<R>(sl.f4 + 4 * qb);
      const R ax = ua.x, ay = ua.y, az = ua.z, ra = ua.w;
      const R bx = ub.x, by = ub.y, bz = ub.z, rb = ub.w;
      const R ia = va.x, ib = vb.x;
      const R fa = va.y, dfa = va.z, fb = vb.y, dfb = vb.z;
      const R iab = ia * ib;
      const R c = (ax * bx + ay * by + az * bz) * iab;
      const R sx = bx - ax, sy = by - ay, sz = bz - az;
      const R rab2 = sx * sx + sy * sy + sz * sz;
      const bool near = bp.any4 && rab2 < rc2;
      R rab = 0, fab = 0, dfab = 0, irab = 0;
      if (near) {
        rab = BM<R>::sq(rab2);
        R sn, cs;
        BM<R>::scpi(rab * inv_rc, &sn, &cs);
        fab = R(0.5) * (cs + R(1));
        dfab = half_pi_rc * sn;
        irab = BM<R>::rcp(rab);
      }
      // per zeta group: A = (1 +- c)^zeta and dA/dc (2^(1 - zeta) is in the weights)
      R Ap[kBpZ], Am[kBpZ], dAp[kBpZ], dAm[kBpZ];
      R Qp[kBpZ], Qm[kBpZ];
      zeta_pow_m1<R, ZS>(bp, R(1) + c, R(1) - c, Qp, Qm);
#pragma unroll
      for (int z = 0; z < kBpZ; ++z) {
        const R zt = pick<R>(bp.z_zeta[z], bp.z_zetaf[z]);
        const R pp = Qp[z], pm = Qm[z];
        Ap[z] = pp * (R(1) + c);
        Am[z] = pm * (R(1) - c);
        dAp[z] = zt * pp;
        dAm[z] = -zt * pm;
      }
      // per (eta, kind) group: the functions' weighted sums S2 = sum w A,
      // S1 = sum w dA/dc, times the group's factor Y and its derivatives
      // the pair-level factors are taken out of the group sums:
      //   al = f_a f_b sum_p S1 E2 X f_ab,   bu = f_b / R_a sum_p S2 E2 X f_ab (f_a' - 2 eta R_a f_a),
      //   bw = f_a / R_b sum_p S2 E2 X f_ab (f_b' - 2 eta R_b f_b),
      //   gs = f_a f_b / R_ab sum_(G4 groups) S2 E2 X (f_ab' - 2 eta R_ab f_ab)
      // with E2 = exp(-eta (R_a^2 + R_b^2)), X = exp(-eta R_ab^2) and f_ab the R_ab
      // cutoff for G4 groups (0 beyond R_c), X = f_ab = 1 for G5 groups
      R al = 0, bu = 0, bw = 0, gs = 0;
      R ea[NY], eb[NY];
#pragma unroll
      for (int p = 0; p < NY; p += 2) {
        ld_e2<R>(sl.e, NB, p >> 1, qa, ea[p], ea[p + 1]);
        ld_e2<R>(sl.e, NB, p >> 1, qb, eb[p], eb[p + 1]);
      }
      const R rfa = ra * fa, rfb = rb * fb, rfab = rab * fab;
#pragma unroll
      for (int p = 0; p < NY; ++p) {  // padded groups: zero exponentials and weights
        R S1 = 0, S2 = 0;
        R wv[2 * kBpZ];  // the group's slots: (z, lambda = +1), (z, lambda = -1)
        ld_group<R>(sl.wc + p * 2 * kBpZ, wv);
#pragma unroll
        for (int z = 0; z < kBpZ; ++z) {  // slots without a function have w = 0
          S2 += wv[2 * z] * Ap[z] + wv[2 * z + 1] * Am[z];
          S1 += wv[2 * z] * dAp[z] + wv[2 * z + 1] * dAm[z];
        }
        const R m2eta = R(-2) * pick<R>(bp.y_eta[p], bp.y_etaf[p]);
        R Ex = ea[p] * eb[p], Exf = Ex;
        const bool k4 = bp.y_kind[p] == 4;
        if (k4) {
          Ex = near ? Ex * BM<R>::ex(R(0.5) * m2eta * rab2) : R(0);
          Exf = Ex * fab;
        }
        al += S1 * Exf;
        const R T = S2 * Exf;
        bu += T * (m2eta * rfa + dfa);
        bw += T * (m2eta * rfb + dfb);
        if (k4) gs += S2 * Ex * (m2eta * rfab + dfab);
      }
      const R fab2 = fa * fb;
      al *= fab2;
      bu *= fb * ia;
      bw *= fa * ib;
      gs *= fab2 * irab;
      // dc/du_a = u_b/(R_a R_b) - c u_a/R_a^2, dc/du_b = u_a/(R_a R_b) - c u_b/R_b^2;
      // to a: dT/du_a - dT/ds, to b: dT/du_b + dT/ds
      const R ca = c * ia * ia, cb = c * ib * ib;
      sl.gax[qa] += al * (bx * iab - ca * ax) + bu * ax - gs * sx;
      sl.gay[qa] += al * (by * iab - ca * ay) + bu * ay - gs * sy;
      sl.gaz[qa] += al * (bz * iab - ca * az) + bu * az - gs * sz;
      sl.gbx[qb] += al * (ax * iab - cb * bx) + bw * bx + gs * sx;
      sl.gby[qb] += al * (ay * iab - cb * by) + bw * by + gs * sy;
      sl.gbz[qb] += al * (az * iab - cb * bz) + bw * bz + gs * sz;
    };
    const bool even = (n & 1) == 0;
    const int kfull = (n - 1) / 2;  // shifts that pair all n neighbours
    if (n >= 32) {
      // flat schedule over (shift, a): 32 consecutive entries span at most two
      // shifts with disjoint a ranges and disjoint b = a + shift ranges, so
      // no lane of an instruction shares a neighbour's sums with another
      const int T = kfull * n + (even ? n / 2 : 0);
      int k = 1, qa = lane;
      for (int t0 = 0; t0 < T; t0 += 32) {
        if (t0 + lane < T) {
          int qb = qa + k;
          if (qb >= n) qb -= n;
          grad_pair(qa, qb);
        }
        __syncwarp();
        qa += 32;
        if (qa >= n) {
          qa -= n;
          ++k;
        }
      }
    } else {
      for (int k = 1; k <= kfull + (even ? 1 : 0); ++k) {
        const int na_k = k > kfull ? n / 2 : n;  // the last shift of an even n pairs each couple once
        const int qa = lane;
        if (qa < na_k) {
          int qb = qa + k;
          if (qb >= n) qb -= n;
          grad_pair(qa, qb);
        }
        __syncwarp();
      }
    }
  }
  // radial terms, then the scatter: -g to atom j_a, +g to atom i
  using Q = typename H::Q;
  Q fix = 0, fiy = 0, fiz = 0;
  // virial sums in FP64 (ENERGY passes only: thermo and compute)
  double w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
  bool bad = false;
  long long *acc = s.hacc;
  for (int qa = lane; qa < n; qa += 32) {
    const Q4<R> ua = ld4<R>(sl.u4 + 4 * qa), va = ld4<R>(sl.f4 + 4 * qa);
    const R ax = ua.x, ay = ua.y, az = ua.z, ra = ua.w;
    const R fa = va.y, dfa = va.z;
    R sr = 0;
#pragma unroll
    for (int m = 0; m < kBpRad; ++m)
      if (m < nr) {
        R v, d;
        radial<R>(bp, m, ra, fa, dfa, v, d);
        sr += sl.dG[m] * d;
      }
    sr *= va.x;
    const R gx = sr * ax + sl.gax[qa] + sl.gbx[qa];
    const R gy = sr * ay + sl.gay[qa] + sl.gby[qa];
    const R gz = sr * az + sl.gaz[qa] + sl.gbz[qa];
    const int j = sl.j[qa];
    if (sizeof(R) == 4)
      bad = bad || !(fabs(gx) < R(4194304) && fabs(gy) < R(4194304) && fabs(gz) < R(4194304));
    const Q qx = H::q(gx), qy = H::q(gy), qz = H::q(gz);
    H::red(acc + j, -qx);
    H::red(acc + Nc + j, -qy);
    H::red(acc + 2 * Nc + j, -qz);
    fix += qx;
    fiy += qy;
    fiz += qz;
    if (ENERGY) {
      w0 -= (double)(ax * gx);
      w1 -= (double)(ay * gy);
      w2 -= (double)(az * gz);
      w3 -= (double)(ax * gy);
      w4 -= (double)(ax * gz);
      w5 -= (double)(ay * gz);
    }
  }
  fix = warp_sum(fix);
  fiy = warp_sum(fiy);
  fiz = warp_sum(fiz);
  if (ENERGY) {
    w0 = warp_sum(w0);
    w1 = warp_sum(w1);
    w2 = warp_sum(w2);
    w3 = warp_sum(w3);
    w4 = warp_sum(w4);
    w5 = warp_sum(w5);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&s.st->bits, kStNonfinite);
  if (lane == 0) {
    H::red(acc + i, fix);
    H::red(acc + Nc + i, fiy);
    H::red(acc + 2 * Nc + i, fiz);
    if (ENERGY) {
      H::red(acc + 3 * Nc + i, H::q(Ei));
      H::red(acc + 4 * Nc + i, H::qd(w0));
      H::red(acc + 5 * Nc + i, H::qd(w1));
      H::red(acc + 6 * Nc + i, H::qd(w2));
      H::red(acc + 7 * Nc + i, H::qd(w3));
      H::red(acc + 8 * Nc + i, H::qd(w4));
      H::red(acc + 9 * Nc + i, H::qd(w5));
    }
  }
}

int warps_for(int precision) { return precision == 0 ? 4 : 8; }

}  // namespace

// the compiled group count for nY groups: nY rounded up to an even number
int ny_compiled(int nY) { return nY <= 2 ? 2 : (nY <= 4 ? 4 : (nY <= 6 ? 6 : 8)); }

size_t bpnn_smem_bytes(const BPParams &p, int precision, int nmax, int *warps) {
  const size_t rsz = precision == 0 ? 8 : 4;
  const int nW = kBpIn * p.H1 + p.H1 + p.H1 * p.H2 + 2 * p.H2;
  const size_t wbytes = ((size_t)nW * rsz + 15) / 16 * 16;
  const size_t per = slab_bytes(nmax, ny_compiled(p.nY), rsz);
  int w = warps_for(precision);
  while (w > 1 && wbytes + (size_t)w * per > 200 * 1024) --w;
  if (warps) *warps = w;
  return wbytes + (size_t)w * per;
}

namespace {
template <class P, int NY, int ZS>
cudaError_t smem_attr_one(int b) {
  cudaError_t e = cudaFuncSetAttribute(k_bpnn<P, true, NY, ZS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_bpnn<P, false, NY, ZS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  return e;
}
template <class P, int NY>
cudaError_t smem_attr_ny(int b) {
  cudaError_t e = smem_attr_one<P, NY, 0>(b);
  if (e == cudaSuccess) e = smem_attr_one<P, NY, 1>(b);
  return e;
}
template <class P>
cudaError_t smem_attr(int b) {
  cudaError_t e = smem_attr_ny<P, 2>(b);
  if (e == cudaSuccess) e = smem_attr_ny<P, 4>(b);
  if (e == cudaSuccess) e = smem_attr_ny<P, 6>(b);
  if (e == cudaSuccess) e = smem_attr_ny<P, 8>(b);
  return e;
}
template <class P, bool EN, int ZS>
void go_ny(const Sys &s, const BPParams &p, StepArgs a, int grid, int threads, size_t sm,
           cudaStream_t st) {
  switch (ny_compiled(p.nY)) {
    case 2: k_bpnn<P, EN, 2, ZS><<<grid, threads, sm, st>>>(s, p, a); break;
    case 4: k_bpnn<P, EN, 4, ZS><<<grid, threads, sm, st>>>(s, p, a); break;
    case 6: k_bpnn<P, EN, 6, ZS><<<grid, threads, sm, st>>>(s, p, a); break;
    default: k_bpnn<P, EN, 8, ZS><<<grid, threads, sm, st>>>(s, p, a); break;
  }
}
template <class P, bool EN>
void go(const Sys &s, const BPParams &p, StepArgs a, int grid, int threads, size_t sm,
        cudaStream_t st) {
  if (p.zset == 1)
    go_ny<P, EN, 1>(s, p, a, grid, threads, sm, st);
  else
    go_ny<P, EN, 0>(s, p, a, grid, threads, sm, st);
}
}  // namespace

int configure_bpnn_smem(size_t bytes, int precision) {
  const int b = (int)bytes;
  const cudaError_t e = precision == 0 ? smem_attr<Fp64>(b) : smem_attr<Mixed>(b);
  return e == cudaSuccess ? 0 : 1;
}

void launch_bpnn(const Sys &s, const BPParams &p, int precision, Mode mode, StepArgs a,
                 cudaStream_t st) {
  int w = 1;
  const size_t sm = bpnn_smem_bytes(p, precision, s.nmax, &w);
  const long long n = s.N_cap > 0 ? s.N_cap : 1;
  const int grid = (int)((n + w - 1) / w);
  if (precision == 0)
    a.energy ? go<Fp64, true>(s, p, a, grid, 32 * w, sm, st)
             : go<Fp64, false>(s, p, a, grid, 32 * w, sm, st);
  else
    a.energy ? go<Mixed, true>(s, p, a, grid, 32 * w, sm, st)
             : go<Mixed, false>(s, p, a, grid, 32 * w, sm, st);
  launch_half_fin(s, precision, mode, a, st);
}

}  // namespace mdk
