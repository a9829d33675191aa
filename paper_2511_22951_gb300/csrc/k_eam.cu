// k_eam.cu -- two-pass embedded-atom force loop (GB300, sm_103a).
//
// Paper passages: single-element EAM read from a table (Sec. "Comparison of
// aluminum shock Hugoniot ..."), forces f_i = sum_j V'(r_ij) r_ji / r_ji
// (Sec. "Potentials support"), in the standard embedded-atom form
//   U = 1/2 sum_ij phi(r_ij) + sum_i F(rho_i),   rho_i = sum_j rho(r_ij),
//   f_i = sum_j [phi'(r) + (F'(rho_i) + F'(rho_j)) rho'(r)] r_ji / r.
// Pass 1 sums rho_i and evaluates F(rho_i), F'(rho_i) (FP64, once per atom);
// pass 2 needs F'(rho_j) of every neighbour, so it is a second launch.  Both
// run on a persistent grid; T lanes own one atom (autotuned), as in the LJ
// kernel.  Where the spline tables are read from:
//  * FP64: staged in shared memory once per block (160 KB for the force pass:
//    one block per SM, up to 128 registers, no spills of the FP64 pair values);
//  * mixed: straight from the workspace through L1 (80 KB per pass, which L1
//    holds once no shared memory is carved out).  A pair's table load lands at
//    a random knot; in shared memory the lanes of a quarter-warp then collide
//    in banks (9.6 / 7.4 wavefronts per 16-byte load instead of 4), and an A/B
//    on one GB300 measured L1 faster: cold-curve batch 1.18e9 against 1.07e9
//    atom-timesteps/s, Al bulk and slab +1%.
#include "k_pair.cuh"

namespace mdk {

// shared memory of the full-list passes (the mixed tables are read through L1)
static int full_pass_smem(const EAMParams &p, int precision, int pass) {
  return precision == 0 ? eam_smem_bytes(p, precision, pass) : 0;
}

namespace {

using namespace pair;

// FP64 passes and the energy passes (thermo and compute steps only): one
// 512-thread block per SM and up to 128 registers (the FP64 pair values, and
// the per-atom energy and virial sums, spill at 64; the 160 KB FP64 force-pass
// tables leave room for one block anyway)
template <class P, bool ENERGY = false>
constexpr int eam_min_blocks() {
  return sizeof(typename G<P>::R) == 4 && !ENERGY ? 2 : 1;
}

template <class P, bool ENERGY, int T>
__global__ void __launch_bounds__(512, eam_min_blocks<P>()) k_rho(Sys s, EAMParams ep, StepArgs a) {
  using GP = G<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  using T1 = typename GP::Tab1;
  extern __shared__ __align__(16) unsigned char smem[];
  const T1 *rt;
  if constexpr (sizeof(R) == 4) {
    rt = GP::tab1(ep);  // mixed: through L1
  } else {
    T1 *w = reinterpret_cast<T1 *>(smem);
    const T1 *src = GP::tab1(ep);
    const int n = GP::n1(ep);
    for (int q = threadIdx.x; q < n; q += blockDim.x) w[q] = src[q];
    __syncthreads();
    rt = w;
  }
  const int N = run_n(s.st);
  const size_t Nc = s.N_cap;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const R rc2 = sizeof(R) == 8 ? (R)ep.rc2 : (R)ep.rc2f;
  const R inv_dr = sizeof(R) == 8 ? (R)ep.inv_dr : (R)ep.inv_drf;
  const int kmax = ep.nr - 2;
  const Tiles<T> tl;
  for (int w = tl.w0; w * Tiles<T>::kPerWarp < N; w += tl.nw) {
    const int i = tl.atom(w);
    const bool valid = i < N;
    V pi;
    R hx = 0, hy = 0, hz = 0;
    int nn = 0;
    if (valid) {
      pi = GP::ld(pg + i);
      GP::h(s.grid[GP::info(pi) >> 8], hx, hy, hz);
      h_scaled(hx, hy, hz);  // for s_scaled
      nn = min(s.nnbr[i], s.nmax);
    }
    Acc<R> rho;
    R br = 0;
    walk<T>(
        s.nbr, Nc, i, nn, tl.t, [&](uint32_t j) { return GP::ld(pg + dbg_idx(s, j, Nc)); },
        [&](uint32_t ent, const V &pj) {
          const R dx = pvec((R)pj.x, (R)pi.x, s_scaled(R(0), ent, 0), hx);
          const R dy = pvec((R)pj.y, (R)pi.y, s_scaled(R(0), ent, 1), hy);
          const R dz = pvec((R)pj.z, (R)pi.z, s_scaled(R(0), ent, 2), hz);
          const R r2 = r2_of(dx, dy, dz);
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
    const double rho_i = lanes_sum<T>(rho.get());
    if (!valid || tl.t != 0) continue;
    // F(rho_i) and F'(rho_i) in FP64 (once per atom)
    double Fv, dF;
    embed_fp64(s, ep, rho_i, Fv, dF);
    __stcs(s.rho + i, rho_i);  // per-atom results: streamed
    __stcs((R *)s.fp + i, (R)dF);
    GP::st_fp((V *)s.pgF + i, pi, dF);
    if (ENERGY) s.ea[i] = Fv;
  }
}

template <class P, int MODE, bool ENERGY, int T>
__global__ void __launch_bounds__(512, eam_min_blocks<P, ENERGY>()) k_eam(Sys s, EAMParams ep,
                                                                       StepArgs a) {
  using GP = G<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  using TP = typename GP::TabPR;
  extern __shared__ __align__(16) unsigned char smem[];
  const TP *tab;
  if constexpr (sizeof(R) == 4) {
    tab = GP::pr8(ep);  // mixed: through L1, one 32-byte record per interval
  } else {
    TP *w = reinterpret_cast<TP *>(smem);
    const TP *src = GP::pr(ep);
    for (int q = threadIdx.x; q < ep.nr; q += blockDim.x) w[q] = src[q];
    __syncthreads();
    tab = w;
  }
  const int N = run_n(s.st);
  const size_t Nc = s.N_cap;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const V *__restrict__ pgf = (const V *)s.pgF;  // neighbours: offsets and F'
  const R *__restrict__ fpa = (const R *)s.fp;
  const R rc2 = sizeof(R) == 8 ? (R)ep.rc2 : (R)ep.rc2f;
  const R inv_dr = sizeof(R) == 8 ? (R)ep.inv_dr : (R)ep.inv_drf;
  const int kmax = ep.nr - 2;
  const Tiles<T> tl;
  for (int w = tl.w0; w * Tiles<T>::kPerWarp < N; w += tl.nw) {
    const int i = tl.atom(w);
    const bool valid = i < N;
    V pi;
    uint32_t inf = 0;
    R hx = 0, hy = 0, hz = 0, fpi = 0;
    int nn = 0;
    if (valid) {
      pi = GP::ld(pg + i);
      inf = GP::info(pi);
      GP::h(s.grid[inf >> 8], hx, hy, hz);
      h_scaled(hx, hy, hz);  // for s_scaled
      fpi = __ldcs(fpa + i);
      nn = min(s.nnbr[i], s.nmax);
    }
    Acc<R> fx, fy, fz;
    // energy and virial (ENERGY passes only: thermo and compute): block sums
    // of four pairs, summed like the forces (mixed: compensated FP32), in FP64
    // once per atom
    R bx = 0, by = 0, bz = 0;
    R be = 0, bw0 = 0, bw1 = 0, bw2 = 0, bw3 = 0, bw4 = 0, bw5 = 0;
    Acc<R> ae, aw0, aw1, aw2, aw3, aw4, aw5;
    walk<T>(
        s.nbr, Nc, i, nn, tl.t, [&](uint32_t j) { return GP::ld(pgf + dbg_idx(s, j, Nc)); },
        [&](uint32_t ent, const V &pj) {
          const R dx = pvec((R)pj.x, (R)pi.x, s_scaled(R(0), ent, 0), hx);
          const R dy = pvec((R)pj.y, (R)pi.y, s_scaled(R(0), ent, 1), hy);
          const R dz = pvec((R)pj.z, (R)pi.z, s_scaled(R(0), ent, 2), hz);
          const R r2 = r2_of(dx, dy, dz);
          if (r2 < rc2) {
            const R inv_r = GP::rsq(r2);
            const R r = r2 * inv_r;
            const R u = r * inv_dr;
            int kk = (int)u;
            kk = kk > kmax ? kmax : kk;
            const R t = u - (R)kk;
            R dphi, drho, vphi = 0;
            if constexpr (sizeof(R) == 4) {
              float4 qa, qb;
              GP::ld_pr8(tab, kk, qa, qb);
              GP::der_ab(qa, qb, t, dphi, drho);
              if (ENERGY) vphi = GP::val_ab(qa, qb, t);
            } else {
              GP::der_pr(tab, kk, t, dphi, drho);
              if (ENERGY) vphi = GP::val_pr(tab, ep, kk, t);
            }
            const R fr = (dphi + (fpi + GP::fp_of(pj)) * drho) * inv_dr * inv_r;  // V'(r)/r
            bx += fr * dx;
            by += fr * dy;
            bz += fr * dz;
            if (ENERGY) {
              be += vphi;
              const R hf = R(-0.5) * fr;
              bw0 += hf * dx * dx;
              bw1 += hf * dy * dy;
              bw2 += hf * dz * dz;
              bw3 += hf * dx * dy;
              bw4 += hf * dx * dz;
              bw5 += hf * dy * dz;
            }
          }
        },
        [&] {
          fx.add(bx);
          fy.add(by);
          fz.add(bz);
          bx = by = bz = 0;
          if (ENERGY) {
            ae.add(R(0.5) * be);
            aw0.add(bw0);
            aw1.add(bw1);
            aw2.add(bw2);
            aw3.add(bw3);
            aw4.add(bw4);
            aw5.add(bw5);
            be = bw0 = bw1 = bw2 = bw3 = bw4 = bw5 = 0;
          }
        });
    const double e = ae.get(), w0 = aw0.get(), w1 = aw1.get(), w2 = aw2.get(), w3 = aw3.get(),
                 w4 = aw4.get(), w5 = aw5.get();
    const R Fx = lanes_sum<T>(fx.getf()), Fy = lanes_sum<T>(fy.getf()),
            Fz = lanes_sum<T>(fz.getf());
    double E = 0, W0 = 0, W1 = 0, W2 = 0, W3 = 0, W4 = 0, W5 = 0;
    if (ENERGY) {
      E = lanes_sum<T>(e);
      W0 = lanes_sum<T>(w0);
      W1 = lanes_sum<T>(w1);
      W2 = lanes_sum<T>(w2);
      W3 = lanes_sum<T>(w3);
      W4 = lanes_sum<T>(w4);
      W5 = lanes_sum<T>(w5);
    }
    if (valid && tl.t == 0) {
      if (ENERGY) {
        s.ea[i] = s.ea[i] + E;
        s.wa[i] = W0;
        s.wa[Nc + i] = W1;
        s.wa[2 * Nc + i] = W2;
        s.wa[3 * Nc + i] = W3;
        s.wa[4 * Nc + i] = W4;
        s.wa[5 * Nc + i] = W5;
      }
      epilogue<P, MODE, ENERGY>(s, a, i, inf, Fx, Fy, Fz);
    }
  }
}

// ---- tables: knot slopes (3-point differences) -> per-knot data ---------------------
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
    o.rho_d32[k] = make_float2((float)dr, (float)mr);
    o.phi_v32[k] = (float)phi[k];
    o.pr32[k] = make_float4((float)dp, (float)mp, (float)dr, (float)mr);
    o.pr8[2 * k] = o.pr32[k];
    o.pr8[2 * k + 1] =
        k + 1 < nr ? make_float4((float)phi[k], (float)hslope(phi, nr, k + 1), 0.0f,
                                 (float)hslope(rho, nr, k + 1))
                   : make_float4((float)phi[k], 0.0f, 0.0f, 0.0f);
    dvec4 q;
    q.x = phi[k];
    q.y = mp;
    q.z = rho[k];
    q.w = mr;
    o.pr64[k] = q;
    if (k + 1 < nr)
      o.rho_i32[k] = make_float4((float)rho[k], (float)dr, (float)mr, (float)hslope(rho, nr, k + 1));
  }
  if (k < nrho) o.F64[k] = make_double2(F[k], hslope(F, nrho, k));
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

int sm_count() {
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
int grid_for(K kern, int block, int smem, long long threads_needed) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  const int g = sm_count() * occ;
  const int need = nblk(threads_needed > 0 ? threads_needed : 1, block);
  return g < need ? g : need;
}

template <class P, int MODE, bool EN, int T>
void go(const Sys &s, const EAMParams &p, StepArgs a, int block, int prec, cudaStream_t st) {
  const int b1 = full_pass_smem(p, prec, 1), b2 = full_pass_smem(p, prec, 2);
  auto k1 = k_rho<P, EN, T>;
  auto k2 = k_eam<P, MODE, EN, T>;
  static int cb = 0, cs = -1, g1 = 0, g2 = 0, cap = -1;
  if (cb != block || cs != b2 || cap != s.N_cap) {
    g1 = grid_for(k1, block, b1, (long long)s.N_cap * T);
    g2 = grid_for(k2, block, b2, (long long)s.N_cap * T);
    cb = block;
    cs = b2;
    cap = s.N_cap;
  }
  k1<<<g1, block, b1, st>>>(s, p, a);
  k2<<<g2, block, b2, st>>>(s, p, a);
}

template <class P, int MODE, bool EN>
void by_tpa(const Sys &s, const EAMParams &p, StepArgs a, const LaunchCfg &c, int prec,
            cudaStream_t st) {
  if (c.tpa == 32)
    go<P, MODE, EN, 32>(s, p, a, c.block, prec, st);
  else if (c.tpa == 8)
    go<P, MODE, EN, 8>(s, p, a, c.block, prec, st);
  else if (c.tpa == 4)
    go<P, MODE, EN, 4>(s, p, a, c.block, prec, st);
  else if (c.tpa == 2)
    go<P, MODE, EN, 2>(s, p, a, c.block, prec, st);
  else
    go<P, MODE, EN, 1>(s, p, a, c.block, prec, st);
}

template <class P, int MODE>
void by_energy(const Sys &s, const EAMParams &p, StepArgs a, const LaunchCfg &c, int prec,
               cudaStream_t st) {
  if (a.energy)
    by_tpa<P, MODE, true>(s, p, a, c, prec, st);
  else
    by_tpa<P, MODE, false>(s, p, a, c, prec, st);
}

template <class P>
void by_mode(const Sys &s, const EAMParams &p, Mode m, StepArgs a, const LaunchCfg &c, int prec,
             cudaStream_t st) {
  if (m == kForceOnly)
    by_energy<P, kForceOnly>(s, p, a, c, prec, st);
  else if (m == kStep)
    by_energy<P, kStep>(s, p, a, c, prec, st);
  else
    by_energy<P, kFinal>(s, p, a, c, prec, st);
}

template <class K>
cudaError_t smem_attr(K k, int bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <class P, int T>
cudaError_t attrs_t(int b1, int b2) {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = smem_attr(k_rho<P, true, T>, b1);
  if (e == cudaSuccess) e = smem_attr(k_rho<P, false, T>, b1);
  if (e == cudaSuccess) e = smem_attr(k_eam<P, kForceOnly, true, T>, b2);
  if (e == cudaSuccess) e = smem_attr(k_eam<P, kForceOnly, false, T>, b2);
  if (e == cudaSuccess) e = smem_attr(k_eam<P, kStep, true, T>, b2);
  if (e == cudaSuccess) e = smem_attr(k_eam<P, kStep, false, T>, b2);
  if (e == cudaSuccess) e = smem_attr(k_eam<P, kFinal, true, T>, b2);
  if (e == cudaSuccess) e = smem_attr(k_eam<P, kFinal, false, T>, b2);
  return e;
}

template <class P>
int attrs(int b1, int b2) {
  cudaError_t e = attrs_t<P, 1>(b1, b2);
  if (e == cudaSuccess) e = attrs_t<P, 2>(b1, b2);
  if (e == cudaSuccess) e = attrs_t<P, 4>(b1, b2);
  if (e == cudaSuccess) e = attrs_t<P, 8>(b1, b2);
  if (e == cudaSuccess) e = attrs_t<P, 32>(b1, b2);
  return e == cudaSuccess ? 0 : -1;
}

}  // namespace

int eam_smem_bytes(const EAMParams &p, int precision, int pass) {
  if (precision == 0) return p.nr * (int)(pass == 1 ? sizeof(double2) : sizeof(dvec4));
  return pass == 1 ? (p.nr - 1) * (int)sizeof(float4) : p.nr * (int)sizeof(float4);
}

int configure_eam_smem(int b1, int b2, int precision) {
  return precision == 0 ? attrs<Fp64>(b1, b2) : attrs<Mixed>(b1, b2);
}

void launch_eam(const Sys &s, const EAMParams &p, int precision, Mode mode, StepArgs a,
                const LaunchCfg &cfg, cudaStream_t st) {
  if (precision == 0)
    by_mode<Fp64>(s, p, mode, a, cfg, 0, st);
  else
    by_mode<Mixed>(s, p, mode, a, cfg, 1, st);
}

namespace {
template <class P, int T>
void rho_only(const Sys &s, const EAMParams &p, StepArgs a, int block, int prec,
              cudaStream_t st) {
  const int b1 = full_pass_smem(p, prec, 1);
  auto k1 = k_rho<P, false, T>;
  k1<<<grid_for(k1, block, b1, (long long)s.N_cap * T), block, b1, st>>>(s, p, a);
}
template <class P>
void rho_by_tpa(const Sys &s, const EAMParams &p, StepArgs a, const LaunchCfg &c, int prec,
                cudaStream_t st) {
  if (c.tpa == 32)
    rho_only<P, 32>(s, p, a, c.block, prec, st);
  else if (c.tpa == 8)
    rho_only<P, 8>(s, p, a, c.block, prec, st);
  else if (c.tpa == 4)
    rho_only<P, 4>(s, p, a, c.block, prec, st);
  else if (c.tpa == 2)
    rho_only<P, 2>(s, p, a, c.block, prec, st);
  else
    rho_only<P, 1>(s, p, a, c.block, prec, st);
}
}  // namespace

void launch_eam_rho(const Sys &s, const EAMParams &p, int precision, StepArgs a,
                    const LaunchCfg &cfg, cudaStream_t st) {
  if (precision == 0)
    rho_by_tpa<Fp64>(s, p, a, cfg, 0, st);
  else
    rho_by_tpa<Mixed>(s, p, a, cfg, 1, st);
}

void launch_eam_prepare(const EAMParams &p, const double *phi, const double *rho,
                        const double *F, EAMTablesDev out, cudaStream_t st) {
  const int n = p.nr > p.nrho ? p.nr : p.nrho;
  k_eam_prepare<<<nblk(n, 256), 256, 0, st>>>(p.nr, p.nrho, phi, rho, F, out);
}

}  // namespace mdk
