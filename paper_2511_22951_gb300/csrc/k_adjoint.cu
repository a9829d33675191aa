// k_adjoint.cu -- reverse-mode gradient of the tabulated EAM with respect to
// its knot values (GB300, sm_103a).
//
// For L = sum_r gE_r E_r + sum_i gF_i . F_i, with E and f_i the embedded-atom
// energy and forces of the force loop (U = 1/2 sum phi + sum F(rho_i),
// f_i = sum_j V'(r_ij) d^_ij, V'(r) = phi'(r) + (F'(rho_i) + F'(rho_j)) rho'(r)),
// the chain rule gives, per directed pair (i, j) inside rc and per atom i:
//   phi knots:  1/2 gE d phi(r) + (gF_i . d^_ij) d phi'(r)
//   c_i       = sum_j [(gF_i - gF_j) . d^_ij] rho'(r_ij)
//   F knots:    gE d F(rho_i) + c_i d F'(rho_i)
//   lambda_i  = gE F'(rho_i) + c_i F''(rho_i)
//   rho knots:  lambda_i d rho(r) + (gF_i . d^_ij)(F'(rho_i) + F'(rho_j)) d rho'(r)
// where "d s(x)" is the row of Hermite weights of the spline s at x over the
// knot values y and the scaled knot slopes M = h m of its interval.  M is a
// fixed linear map of y (3-point differences), so the weights are summed per
// knot first and M's transpose is applied once at the end (k_adj_fin).
//
// Pair distances are recomputed from the gather copy and the Verlet list (no
// stored r_ij).  Pass c: one thread per atom sums c_i (FP32 pair arithmetic in
// the mixed path, Kahan-compensated), then, once per atom in FP64, scatters
// the F-knot weights (FP64 atomics) and stores lambda_i.  Pass pair: one
// thread per atom scatters the phi- and rho-knot weights of its pairs into
// histograms privatised in shared memory (160 KB for 5000 knots per table)
// that each block adds to the global ones when it is done.  Those sums are
// 64-bit fixed point: every contribution is bounded by B = max(|gE|/2,
// |lambda|) + 1.5 |gF| max(1, 2|F'|) / h (Hermite weights are at most 1,
// their u-derivatives at most 1.5 in magnitude), a knot takes at most
// P = N * (list capacity) of them, and the scale S = 2^floor(61 -
// log2(P B)) keeps every sum below 2^62 while resolving 1/S = P B 2^-61.
// Integer adds are native shared-memory atomics and do not depend on their
// order, so these sums are bit-reproducible; the F-knot sums (FP64 atomics,
// four per atom) are reproducible to rounding.
#include "k_pair.cuh"

namespace mdk {
namespace {

using namespace pair;

constexpr int kAdjBlock = 512;

// atomic max of a non-negative double through its bit pattern (monotone there)
__device__ __forceinline__ void max_bits(long long *slot, double v) {
  if (v > 0.0) atomicMax(slot, __double_as_longlong(v));
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Hermite weights at t of the value (w) and of the u-derivative (dw) for the
// coefficients (y_k, M_k, y_{k+1}, M_{k+1}) of one interval
template <class R>
__device__ __forceinline__ void herm_weights(R t, R w[4], R dw[4]) {
  const R t2 = t * t, t3 = t2 * t;
  w[0] = R(2) * t3 - R(3) * t2 + R(1);
  w[1] = t3 - R(2) * t2 + t;
  w[2] = R(3) * t2 - R(2) * t3;
  w[3] = t3 - t2;
  dw[0] = R(6) * t2 - R(6) * t;
  dw[1] = R(3) * t2 - R(4) * t + R(1);
  dw[2] = R(6) * t - R(6) * t2;
  dw[3] = R(3) * t2 - R(2) * t;
}

// add cv * (value weights) + cd * (derivative weights) to knots k and k + 1
__device__ __forceinline__ void scatter(double2 *acc, int k, double a0, double a1, double a2,
                                        double a3) {
  atomicAdd(&acc[k].x, a0);
  atomicAdd(&acc[k].y, a1);
  atomicAdd(&acc[k + 1].x, a2);
  atomicAdd(&acc[k + 1].y, a3);
}

// A 64-bit fixed-point accumulator in shared memory as two 32-bit words, so
// that every update is a native 32-bit atomic: the low word takes the low 32
// bits, the high word the high 32 bits plus the carry out of the low word
// (sums are exact modulo 2^64, whatever the order).
struct Fx64 {
  unsigned *lo;
  int *hi;
  __device__ __forceinline__ void add(int slot, long long v) const {
    const unsigned vl = (unsigned)v;
    int vh = (int)(v >> 32);
    const unsigned old = atomicAdd(lo + slot, vl);
    if (old + vl < old) vh += 1;
    if (vh != 0) atomicAdd(hi + slot, vh);
  }
  __device__ __forceinline__ long long get(int slot) const {
    return (long long)(((unsigned long long)(unsigned)hi[slot] << 32) | lo[slot]);
  }
};

// value * S rounded to an integer, in the pair precision (S is a power of
// two, so the product is exact; FP64 work per pair is what the FP32 pair
// arithmetic of the mixed path avoids on GB300's slow FP64 pipe)
__device__ __forceinline__ long long to_fx(float v, float S) { return __float2ll_rn(v * S); }
__device__ __forceinline__ long long to_fx(double v, double S) { return __double2ll_rn(v * S); }

// fixed-point add of cv * (value weights) + cd * (derivative weights) to the
// slots (y_k, M_k, y_{k+1}, M_{k+1}) = 2k .. 2k + 3
template <class R>
__device__ __forceinline__ void scatter_fx(const Fx64 &h, int k, R S, R a0, R a1, R a2, R a3) {
  h.add(2 * k, to_fx(a0, S));
  h.add(2 * k + 1, to_fx(a1, S));
  h.add(2 * k + 2, to_fx(a2, S));
  h.add(2 * k + 3, to_fx(a3, S));
}

// add a block's shared histogram to the global one (zeros skipped)
__device__ __forceinline__ void flush(const double2 *sh, double2 *gl, int n) {
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const double2 v = sh[q];
    if (v.x != 0.0) atomicAdd(&gl[q].x, v.x);
    if (v.y != 0.0) atomicAdd(&gl[q].y, v.y);
  }
}
__device__ __forceinline__ void flush(const Fx64 &sh, longlong2 *gl, int n) {
  unsigned long long *p = reinterpret_cast<unsigned long long *>(gl);
  for (int q = threadIdx.x; q < 2 * n; q += blockDim.x) {
    const long long v = sh.get(q);
    if (v != 0) atomicAdd(p + q, (unsigned long long)v);
  }
}

// ---- gF of the caller's order -> internal order, in the gather-copy precision -------
template <class P>
__global__ void __launch_bounds__(256) k_adj_load(Sys s, const double *gF, AdjArgs a) {
  using GP = G<P>;
  using V = typename GP::V;
  const int N = s.st->N;
  const int i = blockIdx.x * 256 + threadIdx.x;
  double gx = 0.0, gy = 0.0, gz = 0.0;
  if (i < N) {
    const size_t o = (size_t)s.id[i];
    if (gF) {
      gx = gF[3 * o];
      gy = gF[3 * o + 1];
      gz = gF[3 * o + 2];
    }
    GP::st((V *)a.gint + i, gx, gy, gz, 0u);
  }
  // bounds for the fixed-point scale: max |gF_i| and (one thread) max |gE_r|
  const double m = warp_max(sqrt(gx * gx + gy * gy + gz * gz));
  if ((threadIdx.x & 31) == 0) max_bits(&a.aux[1], m);
  if (i == 0) {
    double e = 0.0;
    for (int r = 0; r < s.n_rep; ++r) e = fmax(e, fabs(a.gE[r]));
    max_bits(&a.aux[0], e);
  }
}

// ---- pass c: c_i, the F-knot weights and lambda_i --------------------------------------
template <class P>
__global__ void __launch_bounds__(kAdjBlock) k_adj_c(Sys s, EAMParams ep, AdjArgs a) {
  using GP = G<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  using T2 = typename GP::Tab2;
  extern __shared__ __align__(16) unsigned char smem[];
  double2 *accF = reinterpret_cast<double2 *>(smem);
  T2 *rt = reinterpret_cast<T2 *>(smem + (a.f_in_smem ? (size_t)ep.nrho * sizeof(double2) : 0));
  {
    const T2 *sr = GP::rho2(ep);
    for (int q = threadIdx.x; q < ep.nr; q += blockDim.x) rt[q] = sr[q];
    if (a.f_in_smem)
      for (int q = threadIdx.x; q < ep.nrho; q += blockDim.x) accF[q] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  double2 *hF = a.f_in_smem ? accF : a.acc_F;
  const int N = s.st->N;
  const size_t Nc = s.N_cap;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const V *__restrict__ gq = (const V *)a.gint;
  const R rc2 = sizeof(R) == 8 ? (R)ep.rc2 : (R)ep.rc2f;
  const R inv_dr = sizeof(R) == 8 ? (R)ep.inv_dr : (R)ep.inv_drf;
  const int kmax = ep.nr - 2;
  double lam_max = 0.0, fp_max = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const V pi = GP::ld(pg + i);
    const uint32_t inf = GP::info(pi);
    const V gi = GP::ld(gq + i);
    R hx, hy, hz;
    GP::h(s.grid[inf >> 8], hx, hy, hz);
    h_scaled(hx, hy, hz);  // for s_scaled
    const int nn = min(s.nnbr[i], s.nmax);
    struct Rec {
      V p, g;
    };
    Acc<R> cs;
    R bc = 0;
    walk<1>(
        s.nbr, Nc, i, nn, 0,
        [&](uint32_t j) {
          Rec q;
          q.p = GP::ld(pg + j);
          q.g = GP::ld(gq + j);
          return q;
        },
        [&](uint32_t ent, const Rec &q) {
          const R dx = pvec((R)q.p.x, (R)pi.x, s_scaled(R(0), ent, 0), hx);
          const R dy = pvec((R)q.p.y, (R)pi.y, s_scaled(R(0), ent, 1), hy);
          const R dz = pvec((R)q.p.z, (R)pi.z, s_scaled(R(0), ent, 2), hz);
          const R r2 = r2_of(dx, dy, dz);
          if (r2 < rc2) {
            const R inv_r = GP::rsq(r2);
            const R u = r2 * inv_r * inv_dr;
            int kk = (int)u;
            kk = kk > kmax ? kmax : kk;
            const R t = u - (R)kk;
            const R drho = GP::der2(rt, kk, t) * inv_dr;
            const R g = ((R)(gi.x - q.g.x) * dx + (R)(gi.y - q.g.y) * dy +
                         (R)(gi.z - q.g.z) * dz) * inv_r;
            bc += g * drho;
          }
        },
        [&] {
          cs.add(bc);
          bc = 0;
        });
    // once per atom, in FP64: F-knot weights at rho_i and lambda_i
    const double ci = cs.get();
    const double rho_i = s.rho[i];
    const double gE = a.gE[inf >> 8];
    const int n = ep.nrho;
    double lam = 0.0;
    if (rho_i > ep.rho_max) {
      // linear continuation F = y_{n-1} + (M_{n-1}/h)(rho - rho_max): F'' = 0
      const double2 a1 = ep.F64[n - 1];
      atomicAdd(&hF[n - 1].x, gE);
      atomicAdd(&hF[n - 1].y, (gE * (rho_i - ep.rho_max) + ci) * ep.inv_drho);
      lam = gE * a1.y * ep.inv_drho;
    } else if (rho_i == rho_i) {
      const double u = rho_i * ep.inv_drho;
      int kk = (int)floor(u);
      kk = kk > n - 2 ? n - 2 : (kk < 0 ? 0 : kk);
      const double t = u - (double)kk;
      double w[4], dw[4];
      herm_weights<double>(t, w, dw);
      const double cd = ci * ep.inv_drho;
      scatter(hF, kk, gE * w[0] + cd * dw[0], gE * w[1] + cd * dw[1], gE * w[2] + cd * dw[2],
              gE * w[3] + cd * dw[3]);
      const double2 a0 = ep.F64[kk], a1 = ep.F64[kk + 1];
      const double Fp = (dw[0] * a0.x + dw[1] * a0.y + dw[2] * a1.x + dw[3] * a1.y) * ep.inv_drho;
      // second u-derivatives of the four weights
      const double Fpp = ((12.0 * t - 6.0) * (a0.x - a1.x) + (6.0 * t - 4.0) * a0.y +
                          (6.0 * t - 2.0) * a1.y) *
                         ep.inv_drho * ep.inv_drho;
      lam = gE * Fp + ci * Fpp;
    }
    a.lam[i] = lam;
    lam_max = fmax(lam_max, fabs(lam));
    fp_max = fmax(fp_max, fabs((double)((const R *)s.fp)[i]));
  }
  lam_max = warp_max(lam_max);
  fp_max = warp_max(fp_max);
  if ((threadIdx.x & 31) == 0) {
    max_bits(&a.aux[2], lam_max);
    max_bits(&a.aux[3], fp_max);
  }
  if (a.f_in_smem) {
    __syncthreads();
    flush(accF, a.acc_F, ep.nrho);
  }
}

// ---- the fixed-point scale of pass pair (one thread) ---------------------------------
__global__ void k_adj_scale(Sys s, EAMParams ep, AdjArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double gE = __longlong_as_double(a.aux[0]), gF = __longlong_as_double(a.aux[1]);
  const double lam = __longlong_as_double(a.aux[2]), fp = __longlong_as_double(a.aux[3]);
  const double B = fmax(0.5 * gE, lam) + 1.5 * gF * fmax(1.0, 2.0 * fp) * ep.inv_dr;
  const double P = (double)s.st->N * (double)s.nmax;
  double S = 1.0;
  if (P * B > 0.0 && isfinite(P * B)) {
    int e = 61 - (int)ceil(log2(P * B));
    e = e > 100 ? 100 : (e < -100 ? -100 : e);  // a finite FP32 scale too
    S = ldexp(1.0, e);
  }
  a.aux[4] = __double_as_longlong(S);
}

// ---- pass pair: phi- and rho-knot weights of every pair -------------------------------
template <class P>
__global__ void __launch_bounds__(kAdjBlock) k_adj_pair(Sys s, EAMParams ep, AdjArgs a) {
  using GP = G<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  extern __shared__ __align__(16) unsigned char smem[];
  // per table 2 nr low words then 2 nr high words
  unsigned *w = reinterpret_cast<unsigned *>(smem);
  const Fx64 hp{w, reinterpret_cast<int *>(w + 2 * ep.nr)};
  const Fx64 hr{w + 4 * ep.nr, reinterpret_cast<int *>(w + 6 * ep.nr)};
  for (int q = threadIdx.x; q < 8 * ep.nr; q += blockDim.x) w[q] = 0u;
  __syncthreads();
  const R S = (R)__longlong_as_double(a.aux[4]);
  const int N = s.st->N;
  const size_t Nc = s.N_cap;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const V *__restrict__ gq = (const V *)a.gint;
  const R *__restrict__ fpa = (const R *)s.fp;
  const R rc2 = sizeof(R) == 8 ? (R)ep.rc2 : (R)ep.rc2f;
  const R inv_dr = sizeof(R) == 8 ? (R)ep.inv_dr : (R)ep.inv_drf;
  const int kmax = ep.nr - 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const V pi = GP::ld(pg + i);
    const uint32_t inf = GP::info(pi);
    const V gi = GP::ld(gq + i);
    R hx, hy, hz;
    GP::h(s.grid[inf >> 8], hx, hy, hz);
    h_scaled(hx, hy, hz);  // for s_scaled
    const int nn = min(s.nnbr[i], s.nmax);
    const R half_gE = (R)(0.5 * a.gE[inf >> 8]);
    const R lam = (R)a.lam[i];
    const R fpi = fpa[i];
    const R gix = (R)gi.x, giy = (R)gi.y, giz = (R)gi.z;
    struct Rec {
      V p;
      R fp;
    };
    walk<1>(
        s.nbr, Nc, i, nn, 0,
        [&](uint32_t j) {
          Rec q;
          q.p = GP::ld(pg + j);
          q.fp = __ldg(fpa + j);
          return q;
        },
        [&](uint32_t ent, const Rec &q) {
          const R dx = pvec((R)q.p.x, (R)pi.x, s_scaled(R(0), ent, 0), hx);
          const R dy = pvec((R)q.p.y, (R)pi.y, s_scaled(R(0), ent, 1), hy);
          const R dz = pvec((R)q.p.z, (R)pi.z, s_scaled(R(0), ent, 2), hz);
          const R r2 = r2_of(dx, dy, dz);
          if (r2 < rc2) {
            const R inv_r = GP::rsq(r2);
            const R u = r2 * inv_r * inv_dr;
            int kk = (int)u;
            kk = kk > kmax ? kmax : kk;
            const R t = u - (R)kk;
            R w[4], dw[4];
            herm_weights<R>(t, w, dw);
            const R gd = (gix * dx + giy * dy + giz * dz) * inv_r;
            const R cp = gd * inv_dr;                    // phi': (gF_i . d^) / h
            const R cr = gd * (fpi + q.fp) * inv_dr;     // rho': times F'_i + F'_j
            scatter_fx<R>(hp, kk, S, half_gE * w[0] + cp * dw[0], half_gE * w[1] + cp * dw[1],
                          half_gE * w[2] + cp * dw[2], half_gE * w[3] + cp * dw[3]);
            scatter_fx<R>(hr, kk, S, lam * w[0] + cr * dw[0], lam * w[1] + cr * dw[1],
                          lam * w[2] + cr * dw[2], lam * w[3] + cr * dw[3]);
          }
        },
        [] {});
  }
  __syncthreads();
  flush(hp, a.acc_phi, ep.nr);
  flush(hr, a.acc_rho, ep.nr);
}

// ---- knot gradients: d/dy plus the transpose of the slope map applied to d/dM ----------
// Interior M_q = (y_{q+1} - y_{q-1}) / 2; M_0 = (-3 y_0 + 4 y_1 - y_2) / 2;
// M_{n-1} = (3 y_{n-1} - 4 y_{n-2} + y_{n-3}) / 2.  One thread per knot, fixed order.
__global__ void __launch_bounds__(256) k_adj_fin(EAMParams ep, AdjArgs a) {
  const int q = blockIdx.x * 256 + threadIdx.x;
  const int nr = ep.nr, total = 2 * nr + ep.nrho;
  if (q >= total) return;
  int n, k;
  if (q < nr) {
    n = nr;
    k = q;
  } else if (q < 2 * nr) {
    n = nr;
    k = q - nr;
  } else {
    n = ep.nrho;
    k = q - 2 * nr;
  }
  // (d/dy, d/dM) of knot j of this table
  const double inv_S = 1.0 / __longlong_as_double(a.aux[4]);
  auto at = [&](int j) -> double2 {
    if (q >= 2 * nr) return a.acc_F[j];
    const longlong2 v = (q < nr ? a.acc_phi : a.acc_rho)[j];
    return make_double2((double)v.x * inv_S, (double)v.y * inv_S);
  };
  double g = at(k).x;
  if (k - 1 >= 1 && k - 1 <= n - 2) g += 0.5 * at(k - 1).y;
  if (k + 1 >= 1 && k + 1 <= n - 2) g -= 0.5 * at(k + 1).y;
  if (k <= 2) g += (k == 0 ? -1.5 : (k == 1 ? 2.0 : -0.5)) * at(0).y;
  if (k >= n - 3) {
    const int m = n - 1 - k;
    g += (m == 0 ? 1.5 : (m == 1 ? -2.0 : 0.5)) * at(n - 1).y;
  }
  a.out[q] = g;
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

int sm_count_adj() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <class K>
int persistent_grid(K kern, int smem, int N) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kAdjBlock, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  const int g = sm_count_adj() * occ;
  const int need = nblk(N > 0 ? N : 1, kAdjBlock);
  return g < need ? g : need;
}

template <class P>
int run(const Sys &s, const EAMParams &ep, const double *gF, AdjArgs a, int64_t n_atoms,
        cudaStream_t st) {
  using GP = G<P>;
  const int b_c = adjoint_smem_bytes(ep, sizeof(typename GP::R) == 8 ? 0 : 1, 1);
  const int b_p = adjoint_smem_bytes(ep, 0, 2);
  if (b_c < 0 || b_p < 0) return -1;
  a.f_in_smem = adjoint_f_in_smem(ep, sizeof(typename GP::R) == 8 ? 0 : 1);
  if (cudaFuncSetAttribute(k_adj_c<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, b_c) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_adj_pair<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, b_p) !=
          cudaSuccess)
    return -1;
  const int N = (int)n_atoms;
  k_adj_load<P><<<nblk(s.N_cap > 0 ? s.N_cap : 1, 256), 256, 0, st>>>(s, gF, a);
  k_adj_c<P><<<persistent_grid(k_adj_c<P>, b_c, N), kAdjBlock, b_c, st>>>(s, ep, a);
  k_adj_scale<<<1, 32, 0, st>>>(s, ep, a);
  k_adj_pair<P><<<persistent_grid(k_adj_pair<P>, b_p, N), kAdjBlock, b_p, st>>>(s, ep, a);
  k_adj_fin<<<nblk(2 * ep.nr + ep.nrho, 256), 256, 0, st>>>(ep, a);
  return 0;
}

constexpr int kSmemMax = 227 * 1024;

}  // namespace

// shared bytes of pass c (1: rho table + F histogram when it fits) or pass pair (2)
int adjoint_smem_bytes(const EAMParams &ep, int precision, int pass) {
  if (pass == 2) {
    const long long b = 2LL * ep.nr * (long long)sizeof(double2);
    return b <= kSmemMax ? (int)b : -1;
  }
  const long long tab = (long long)ep.nr * (precision == 0 ? 16 : 8);
  const long long full = tab + (long long)ep.nrho * (long long)sizeof(double2);
  if (full <= kSmemMax) return (int)full;
  return tab <= kSmemMax ? (int)tab : -1;
}

int adjoint_f_in_smem(const EAMParams &ep, int precision) {
  const long long tab = (long long)ep.nr * (precision == 0 ? 16 : 8);
  return tab + (long long)ep.nrho * (long long)sizeof(double2) <= kSmemMax ? 1 : 0;
}

int launch_eam_adjoint(const Sys &s, const EAMParams &ep, int precision, const double *gF,
                       const AdjArgs &a, int64_t n_atoms, cudaStream_t st) {
  return precision == 0 ? run<Fp64>(s, ep, gF, a, n_atoms, st)
                        : run<Mixed>(s, ep, gF, a, n_atoms, st);
}

}  // namespace mdk
