// k_eam_half.cu -- the embedded-atom passes on half Verlet lists (each pair
// once, Newton's third law) with accumulating atomics (GB300, sm_103a).
//
// Paper passages: as k_eam.cu (single-element tabulated EAM, f_i = sum_j
// V'(r_ij) r_ji / r_ji with V'(r) = phi'(r) + (F'(rho_i) + F'(rho_j))
// rho'(r)).  On a half list each pair is visited by one of its atoms, so
// both sums -- rho_i = sum_j rho(r_ij) and the forces -- scatter to the
// other atom:
//   k_rho_half   rho(r) of each pair added to both atoms' accumulators
//                (s.hacc row 3, free until the force pass's energies)
//   k_embed      per atom: take rho_i, F(rho_i) and F'(rho_i) in FP64 (the
//                full-list path's arithmetic), the gather copy with F' for
//                the force pass, the embedding energy back into row 3
//   k_eam_half   the pair force added to i and subtracted from j (rows 0-2),
//                half of phi and of the pair virial to each atom
//   k_half_fin   (k_lj_half.cu) takes the totals and finishes the step.
// The tables are staged in shared memory on a persistent grid as in the
// full-list passes.  Mixed path: 64-bit fixed-point accumulators (order-
// independent, reproducible); FP64 path: FP64 reduction atomics.
#include "k_pair.cuh"

namespace mdk {
namespace {

using namespace pair;

// 256 threads and two blocks per SM: 128 registers (the walk's prefetch and
// the accumulators do not fit 64 without spills), tables 2 x 80 KB
template <class P>
__global__ void __launch_bounds__(256, 2) k_rho_half(Sys s, EAMParams ep, StepArgs a) {
  using GP = G<P>;
  using H = HalfAcc<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  using T1 = typename GP::Tab1;
  using Q = typename H::Q;
  extern __shared__ __align__(16) unsigned char smem[];
  T1 *rt = reinterpret_cast<T1 *>(smem);
  {
    const T1 *src = GP::tab1(ep);
    const int n = GP::n1(ep);
    for (int q = threadIdx.x; q < n; q += blockDim.x) rt[q] = src[q];
  }
  __syncthreads();
  const int N = run_n(s.st);
  const size_t Nc = s.N_cap;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const R rc2 = sizeof(R) == 8 ? (R)ep.rc2 : (R)ep.rc2f;
  const R inv_dr = sizeof(R) == 8 ? (R)ep.inv_dr : (R)ep.inv_drf;
  const int kmax = ep.nr - 2;
  long long *acc = s.hacc + 3 * Nc;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const V pi = GP::ld(pg + i);
    R hx, hy, hz;
    GP::h(s.grid[GP::info(pi) >> 8], hx, hy, hz);
    h_scaled(hx, hy, hz);  // for s_scaled
    const int nn = min(s.nnbr[i], s.nmax);
    Q rho = 0;
    walk<1>(
        s.nbr, Nc, i, nn, 0, [&](uint32_t j) { return GP::ld(pg + dbg_idx(s, j, Nc)); },
        [&](uint32_t ent, const V &pj) {
          const R dx = pvec((R)pj.x, (R)pi.x, s_scaled(R(0), ent, 0), hx);
          const R dy = pvec((R)pj.y, (R)pi.y, s_scaled(R(0), ent, 1), hy);
          const R dz = pvec((R)pj.z, (R)pi.z, s_scaled(R(0), ent, 2), hz);
          const R r2 = r2_of(dx, dy, dz);
          if (r2 < rc2) {
            const R u = GP::sqr(r2) * inv_dr;
            int kk = (int)u;
            kk = kk > kmax ? kmax : kk;
            const Q q = H::q(GP::val1(rt, kk, u - (R)kk));
            rho += q;
            H::red(acc + dbg_idx(s, nbr_j(ent), Nc, i), q);
          }
        },
        [] {});
    H::red(acc + i, rho);
  }
}

template <class P, bool ENERGY>
__global__ void __launch_bounds__(256) k_embed(Sys s, EAMParams ep, StepArgs a) {
  using GP = G<P>;
  using H = HalfAcc<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  const int N = run_n(s.st);
  const size_t Nc = s.N_cap;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  long long *acc = s.hacc + 3 * Nc;
  const double rho_i = H::take(acc + i);
  double Fv, dF;
  embed_fp64(s, ep, rho_i, Fv, dF);
  s.rho[i] = rho_i;
  ((R *)s.fp)[i] = (R)dF;
  GP::st_fp((V *)s.pgF + i, GP::ld((const V *)s.pg[a.cur] + i), dF);
  if (ENERGY) H::red(acc + i, H::qd(Fv));
}

template <class P, bool ENERGY>
__global__ void __launch_bounds__(256, 2) k_eam_half(Sys s, EAMParams ep, StepArgs a) {
  using GP = G<P>;
  using H = HalfAcc<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  using TP = typename GP::TabPR;
  using Q = typename H::Q;
  extern __shared__ __align__(16) unsigned char smem[];
  TP *tab = reinterpret_cast<TP *>(smem);
  {
    const TP *src = GP::pr(ep);
    for (int q = threadIdx.x; q < ep.nr; q += blockDim.x) tab[q] = src[q];
  }
  __syncthreads();
  const int N = run_n(s.st);
  const size_t Nc = s.N_cap;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const V *__restrict__ pgf = (const V *)s.pgF;  // neighbours: offsets and F'
  const R *__restrict__ fpa = (const R *)s.fp;
  const R rc2 = sizeof(R) == 8 ? (R)ep.rc2 : (R)ep.rc2f;
  const R inv_dr = sizeof(R) == 8 ? (R)ep.inv_dr : (R)ep.inv_drf;
  const int kmax = ep.nr - 2;
  // |V'(r)/r| below this keeps a pair term under 2^22 eV/A (|d| < rc)
  const R fr_max = (R)(4194304.0 / ep.rc);
  long long *acc = s.hacc;
  bool bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const V pi = GP::ld(pg + i);
    R hx, hy, hz;
    GP::h(s.grid[GP::info(pi) >> 8], hx, hy, hz);
    h_scaled(hx, hy, hz);  // for s_scaled
    const R fpi = fpa[i];
    const int nn = min(s.nnbr[i], s.nmax);
    Q fx = 0, fy = 0, fz = 0, e = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    walk<1>(
        s.nbr, Nc, i, nn, 0, [&](uint32_t j) { return GP::ld(pgf + dbg_idx(s, j, Nc)); },
        [&](uint32_t ent, const V &pj) {
          const R dx = pvec((R)pj.x, (R)pi.x, s_scaled(R(0), ent, 0), hx);
          const R dy = pvec((R)pj.y, (R)pi.y, s_scaled(R(0), ent, 1), hy);
          const R dz = pvec((R)pj.z, (R)pi.z, s_scaled(R(0), ent, 2), hz);
          const R r2 = r2_of(dx, dy, dz);
          if (r2 < rc2) {
            const R inv_r = GP::rsq(r2);
            const R u = r2 * inv_r * inv_dr;
            int kk = (int)u;
            kk = kk > kmax ? kmax : kk;
            const R t = u - (R)kk;
            R dphi, drho;
            GP::der_pr(tab, kk, t, dphi, drho);
            const R fr = (dphi + (fpi + GP::fp_of(pj)) * drho) * inv_dr * inv_r;  // V'(r)/r
            if (sizeof(R) == 4) bad = bad || !(fabs(fr) < fr_max);
            const Q qx = H::q(fr * dx), qy = H::q(fr * dy), qz = H::q(fr * dz);
            const size_t j = dbg_idx(s, nbr_j(ent), Nc, i);
            fx += qx;
            fy += qy;
            fz += qz;
            H::red(acc + j, -qx);
            H::red(acc + Nc + j, -qy);
            H::red(acc + 2 * Nc + j, -qz);
            if (ENERGY) {
              // half of phi and of the pair virial -1/2 r_ij (x) f_ij to each atom
              const R hf = R(-0.5) * fr;
              const Q qe = H::q(R(0.5) * GP::val_pr(tab, ep, kk, t));
              const Q q0 = H::q(hf * dx * dx), q1 = H::q(hf * dy * dy), q2 = H::q(hf * dz * dz);
              const Q q3 = H::q(hf * dx * dy), q4 = H::q(hf * dx * dz), q5 = H::q(hf * dy * dz);
              e += qe;
              w0 += q0;
              w1 += q1;
              w2 += q2;
              w3 += q3;
              w4 += q4;
              w5 += q5;
              H::red(acc + 3 * Nc + j, qe);
              H::red(acc + 4 * Nc + j, q0);
              H::red(acc + 5 * Nc + j, q1);
              H::red(acc + 6 * Nc + j, q2);
              H::red(acc + 7 * Nc + j, q3);
              H::red(acc + 8 * Nc + j, q4);
              H::red(acc + 9 * Nc + j, q5);
            }
          }
        },
        [] {});
    H::red(acc + i, fx);
    H::red(acc + Nc + i, fy);
    H::red(acc + 2 * Nc + i, fz);
    if (ENERGY) {
      H::red(acc + 3 * Nc + i, e);
      H::red(acc + 4 * Nc + i, w0);
      H::red(acc + 5 * Nc + i, w1);
      H::red(acc + 6 * Nc + i, w2);
      H::red(acc + 7 * Nc + i, w3);
      H::red(acc + 8 * Nc + i, w4);
      H::red(acc + 9 * Nc + i, w5);
    }
  }
  if (bad) atomicOr(&s.st->bits, kStNonfinite);
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

int sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// persistent grid: resident blocks per SM x SMs, at most one thread per atom
template <class K>
int pgrid(K kern, int block, int smem, long long atoms) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  const int g = sms() * occ, need = nblk(atoms > 0 ? atoms : 1, block);
  return g < need ? g : need;
}

template <class P, bool EN>
void go(const Sys &s, const EAMParams &p, Mode m, StepArgs a, int block, int prec,
        cudaStream_t st) {
  const int b1 = eam_smem_bytes(p, prec, 1), b2 = eam_smem_bytes(p, prec, 2);
  auto k1 = k_rho_half<P>;
  auto k3 = k_eam_half<P, EN>;
  k1<<<pgrid(k1, block, b1, s.N_cap), block, b1, st>>>(s, p, a);
  k_embed<P, EN><<<nblk(s.N_cap > 0 ? s.N_cap : 1, 256), 256, 0, st>>>(s, p, a);
  k3<<<pgrid(k3, block, b2, s.N_cap), block, b2, st>>>(s, p, a);
  launch_half_fin(s, prec, m, a, st);
}

template <class P>
cudaError_t attrs(int b1, int b2) {
  cudaError_t e = cudaFuncSetAttribute(k_rho_half<P>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, b1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_eam_half<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             b2);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_eam_half<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             b2);
  return e;
}

}  // namespace

int configure_eam_half_smem(int b1, int b2, int precision) {
  return (precision == 0 ? attrs<Fp64>(b1, b2) : attrs<Mixed>(b1, b2)) == cudaSuccess ? 0 : -1;
}

void launch_eam_half(const Sys &s, const EAMParams &p, int precision, Mode mode, StepArgs a,
                     const LaunchCfg &cfg, cudaStream_t st) {
  const int block = cfg.block > 256 ? 256 : cfg.block;
  if (precision == 0)
    a.energy ? go<Fp64, true>(s, p, mode, a, block, 0, st)
             : go<Fp64, false>(s, p, mode, a, block, 0, st);
  else
    a.energy ? go<Mixed, true>(s, p, mode, a, block, 1, st)
             : go<Mixed, false>(s, p, mode, a, block, 1, st);
}

}  // namespace mdk
