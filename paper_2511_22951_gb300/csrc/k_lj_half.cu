// k_lj_half.cu -- Lennard-Jones forces from half Verlet lists (each pair
// once, Newton's third law) with accumulating atomics, and the per-atom
// pass that finishes the step (GB300, sm_103a).
//
// Paper passages: f_i = sum_j V'(r_ij) r_ji / r_ji (Sec. "Potentials
// support"), so the pair (i, j) adds V'(r)/r (r_j - r_i) to f_i and the
// negative to f_j; m r'' = f integrated by velocity Verlet (Sec. "Molecular
// dynamics").
//
// The half list holds each unordered pair once (the build's rule: for
// j != i, in the list of i when (i < j) == (i + j even), which splits every
// atom's neighbours about evenly; for a periodic image of i itself, the
// lexicographically positive stencil offset).  One thread walks atom i's
// half list, sums f_i in registers and adds -f_ij to atom j's accumulator
// with a reduction atomic; at the end it adds its own sum to its own
// accumulator.  Forces of neighbouring threads meet in those accumulators,
// so the velocity-Verlet update cannot be fused into this pass: k_half_fin
// reads each atom's total, clears the accumulator for the next pass and
// runs the same epilogue as the full-list kernel (the Behler-Parrinello
// forces, which scatter to neighbours too, finish their steps with it).
//
// Mixed path: the accumulators are 64-bit fixed point (unit 2^-40 eV/A):
// every pair term is rounded once, integer addition is associative, so the
// result does not depend on the order in which the atomics land (bitwise
// reproducible), and the terms of a pair cancel exactly (sum of the forces
// is exactly zero).  A pair term at or above 2^22 eV/A (overlapping atoms)
// sets the non-finite status instead of wrapping.  FP64 path: FP64
// reduction atomics (results reproducible to rounding, not bitwise).
#include "lj_pair.cuh"

namespace mdk {
namespace {

using namespace pair;

// 64 registers (32 resident warps per SM) for the mixed force-only pass;
// FP64 pair values and the energy/virial sums need more (128)
template <class P>
constexpr int half_min_blocks(bool energy) {
  return sizeof(typename G<P>::R) == 4 && !energy ? 4 : 2;
}

template <class P, bool ENERGY, int SHIFT>
__global__ void __launch_bounds__(256, half_min_blocks<P>(ENERGY))
    k_lj_half(Sys s, LJParams lp, StepArgs a) {
  using GP = G<P>;
  using H = HalfAcc<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  using Q = typename H::Q;
  const int N = run_n(s.st);
  const size_t Nc = s.N_cap;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const LJc<R> lc(lp);
  // |V'(r)/r| below this keeps every component of a pair term below 2^22
  // eV/A in the fixed-point range (|d| < rc)
  const R fr_max = (R)(4194304.0 / lp.rc);
  long long *acc = s.hacc;
  const V pi = GP::ld(pg + i);
  R hx, hy, hz;
  GP::h(s.grid[GP::info(pi) >> 8], hx, hy, hz);
  h_scaled(hx, hy, hz);  // for s_scaled
  const int nn = min(s.nnbr[i], s.nmax);
  Q fx = 0, fy = 0, fz = 0, e = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
  bool bad = false;
  walk<1>(
      s.nbr, Nc, i, nn, 0, [&](uint32_t j) { return GP::ld(pg + dbg_idx(s, j, Nc)); },
      [&](uint32_t ent, const V &pj) {
        const R dx = pvec((R)pj.x, (R)pi.x, s_scaled(R(0), ent, 0), hx);
        const R dy = pvec((R)pj.y, (R)pi.y, s_scaled(R(0), ent, 1), hy);
        const R dz = pvec((R)pj.z, (R)pi.z, s_scaled(R(0), ent, 2), hz);
        const R r2 = r2_of(dx, dy, dz);
        if (r2 < lc.rc2) {
          R fr, v;
          lj_pair<GP, SHIFT, ENERGY>(lc, r2, fr, v);
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
            // half of the pair energy and of the pair virial
            // -1/2 r_ij (x) f_ij (r_ij = -d) to each atom
            const R hf = R(-0.5) * fr;
            const Q qe = H::q(R(0.5) * v);
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
  if (bad) atomicOr(&s.st->bits, kStNonfinite);
}

// Per atom: take the accumulated totals (clearing them), then store the
// force or integrate, exactly as the full-list kernel's epilogue does.
template <class P, int MODE, bool ENERGY>
__global__ void __launch_bounds__(256) k_half_fin(Sys s, StepArgs a) {
  using GP = G<P>;
  using H = HalfAcc<P>;
  using V = typename GP::V;
  const int N = run_n(s.st);
  const size_t Nc = s.N_cap;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  long long *acc = s.hacc;
  const double Fx = H::take(acc + i), Fy = H::take(acc + Nc + i), Fz = H::take(acc + 2 * Nc + i);
  if (ENERGY) {
    s.ea[i] = H::take(acc + 3 * Nc + i);
#pragma unroll
    for (int c = 0; c < 6; ++c) s.wa[c * Nc + i] = H::take(acc + (4 + c) * Nc + i);
  }
  const uint32_t inf = GP::info(GP::ld((const V *)s.pg[a.cur] + i));
  epilogue<P, MODE, ENERGY>(s, a, i, inf, Fx, Fy, Fz);
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

template <class P, bool EN>
void fin(const Sys &s, Mode m, StepArgs a, cudaStream_t st) {
  const int fb = 256, fg = nblk(s.N_cap > 0 ? s.N_cap : 1, fb);
  if (m == kForceOnly)
    k_half_fin<P, kForceOnly, EN><<<fg, fb, 0, st>>>(s, a);
  else if (m == kStep)
    k_half_fin<P, kStep, EN><<<fg, fb, 0, st>>>(s, a);
  else
    k_half_fin<P, kFinal, EN><<<fg, fb, 0, st>>>(s, a);
}

template <class P, bool EN, int SH>
void go(const Sys &s, const LJParams &p, Mode m, StepArgs a, int block, cudaStream_t st) {
  if (block > 256) block = 256;
  const int grid = nblk(s.N_cap > 0 ? s.N_cap : 1, block);
  k_lj_half<P, EN, SH><<<grid, block, 0, st>>>(s, p, a);
  fin<P, EN>(s, m, a, st);
}

template <class P, bool EN>
void by_shift(const Sys &s, const LJParams &p, Mode m, StepArgs a, int block, cudaStream_t st) {
  if (p.shift_mode == 2)
    go<P, EN, 2>(s, p, m, a, block, st);
  else
    go<P, EN, 1>(s, p, m, a, block, st);
}

template <class P>
void by_energy(const Sys &s, const LJParams &p, Mode m, StepArgs a, int block, cudaStream_t st) {
  if (a.energy)
    by_shift<P, true>(s, p, m, a, block, st);
  else
    by_shift<P, false>(s, p, m, a, block, st);
}

}  // namespace

void launch_half_fin(const Sys &s, int precision, Mode mode, StepArgs a, cudaStream_t st) {
  if (precision == 0)
    a.energy ? fin<Fp64, true>(s, mode, a, st) : fin<Fp64, false>(s, mode, a, st);
  else
    a.energy ? fin<Mixed, true>(s, mode, a, st) : fin<Mixed, false>(s, mode, a, st);
}

void launch_lj_half(const Sys &s, const LJParams &p, int precision, Mode mode, StepArgs a,
                    const LaunchCfg &cfg, cudaStream_t st) {
  if (precision == 0)
    by_energy<Fp64>(s, p, mode, a, cfg.block, st);
  else
    by_energy<Mixed>(s, p, mode, a, cfg.block, st);
}

}  // namespace mdk
