// k_lj.cu -- Lennard-Jones force loop with the fused velocity-Verlet update
// (GB300, sm_103a).
//
// Paper passages: f_i = sum_j V'(r_ij) r_ji / r_ji (Sec. "Potentials
// support"); m r'' = f integrated by velocity Verlet (Sec. "Molecular
// dynamics").  V(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] - shift, cut at rc.
//
// Launch bounds: at most 256 threads per block and 4 blocks per SM, so the
// kernel fits 64 registers (32 resident warps per SM).  The registers hold
// the next list group, loaded while the current one runs; measured on the
// 8.4M-atom argon step this beats 48 registers with 40 warps (spills) and
// 80 registers with 24 warps.
// T lanes own one atom (T = 1, 2, 4, 8 or 32 -- a warp per atom --, picked by
// the autotuner by density and list length): lane t walks
// the list groups t, t + T, ... of the full Verlet list, the lanes' sums are
// combined with shuffles in a fixed order, and lane 0 runs the epilogue
// (store the force, or finish step n and start step n + 1).  The pair vector
// is d = (p_j - p_i) + s h with p the cell-centre offsets of the gather copy
// and s the stencil offset stored in the list entry, so FP32 pair arithmetic
// never subtracts two large coordinates.
#include "lj_pair.cuh"

namespace mdk {
namespace {

using namespace pair;

// mixed: 4 blocks of 256 per SM (64 registers); FP64: 2 blocks (128 registers:
// the FP64 pair values and sums need them)
template <class P>
constexpr int lj_min_blocks() {
  return sizeof(typename G<P>::R) == 4 ? 4 : 2;
}

template <class P, int MODE, bool ENERGY, int SHIFT, int T>
__global__ void __launch_bounds__(256, lj_min_blocks<P>()) k_lj(Sys s, LJParams lp, StepArgs a) {
  using GP = G<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  const int N = run_n(s.st);
  const size_t Nc = s.N_cap;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const LJc<R> lc(lp);
  // one warp tile per warp (no shared tables to amortise, so no persistent
  // loop: the loop's extra state costs registers and occupancy)
  const Tiles<T> tl;
  {
    const int w = tl.w0;
    const int i = tl.atom(w);
    // T = 1: a lane is an atom and exits on its own; T > 1: the whole warp
    // stays for the shuffles and idle lanes carry valid = false
    if (T == 1 ? i >= N : w * Tiles<T>::kPerWarp >= N) return;
    const bool valid = T == 1 || i < N;
    V pi;
    uint32_t inf = 0;
    R hx = 0, hy = 0, hz = 0;
    int nn = 0;
    if (valid) {
      pi = GP::ld(pg + i);
      inf = GP::info(pi);
      GP::h(s.grid[inf >> 8], hx, hy, hz);
      nn = min(s.nnbr[i], s.nmax);
    }
    Acc<R> fx, fy, fz;
    // energy and virial sums in FP64 (ENERGY passes only: thermo and compute)
    double e = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    R bx = 0, by = 0, bz = 0;  // block sums of four pairs
    walk<T>(
        s.nbr, Nc, i, nn, tl.t, [&](uint32_t j) { return GP::ld(pg + j); },
        [&](uint32_t ent, const V &pj) {
          const R dx = (R)(pj.x - pi.x) + s_unit(R(0), ent, 0) * hx;
          const R dy = (R)(pj.y - pi.y) + s_unit(R(0), ent, 1) * hy;
          const R dz = (R)(pj.z - pi.z) + s_unit(R(0), ent, 2) * hz;
          const R r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < lc.rc2) {
            R fr, v;
            lj_pair<GP, SHIFT, ENERGY>(lc, r2, fr, v);
            bx += fr * dx;
            by += fr * dy;
            bz += fr * dz;
            if (ENERGY) {
              e += 0.5 * (double)v;
              const R hf = R(-0.5) * fr;  // r_ij = -d
              w0 += (double)(hf * dx * dx);
              w1 += (double)(hf * dy * dy);
              w2 += (double)(hf * dz * dz);
              w3 += (double)(hf * dx * dy);
              w4 += (double)(hf * dx * dz);
              w5 += (double)(hf * dy * dz);
            }
          }
        },
        [&] {
          fx.add(bx);
          fy.add(by);
          fz.add(bz);
          bx = by = bz = 0;
        });
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
        s.ea[i] = E;
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

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

template <class P, int MODE, bool EN, int SH, int T>
void go(const Sys &s, const LJParams &p, StepArgs a, int block, cudaStream_t st) {
  if (block > 256) block = 256;  // the kernel is compiled for <= 256 threads (48 registers)
  const int grid = nblk((long long)(s.N_cap > 0 ? s.N_cap : 1) * T, block);
  k_lj<P, MODE, EN, SH, T><<<grid, block, 0, st>>>(s, p, a);
}

template <class P, int MODE, bool EN, int SH>
void by_tpa(const Sys &s, const LJParams &p, StepArgs a, const LaunchCfg &c, cudaStream_t st) {
  if (c.tpa == 32)
    go<P, MODE, EN, SH, 32>(s, p, a, c.block, st);
  else if (c.tpa == 8)
    go<P, MODE, EN, SH, 8>(s, p, a, c.block, st);
  else if (c.tpa == 4)
    go<P, MODE, EN, SH, 4>(s, p, a, c.block, st);
  else if (c.tpa == 2)
    go<P, MODE, EN, SH, 2>(s, p, a, c.block, st);
  else
    go<P, MODE, EN, SH, 1>(s, p, a, c.block, st);
}

template <class P, int MODE, bool EN>
void by_shift(const Sys &s, const LJParams &p, StepArgs a, const LaunchCfg &c, cudaStream_t st) {
  if (p.shift_mode == 2)
    by_tpa<P, MODE, EN, 2>(s, p, a, c, st);
  else
    by_tpa<P, MODE, EN, 1>(s, p, a, c, st);
}

template <class P, int MODE>
void by_energy(const Sys &s, const LJParams &p, StepArgs a, const LaunchCfg &c, cudaStream_t st) {
  if (a.energy)
    by_shift<P, MODE, true>(s, p, a, c, st);
  else
    by_shift<P, MODE, false>(s, p, a, c, st);
}

template <class P>
void by_mode(const Sys &s, const LJParams &p, Mode m, StepArgs a, const LaunchCfg &c,
             cudaStream_t st) {
  if (m == kForceOnly)
    by_energy<P, kForceOnly>(s, p, a, c, st);
  else if (m == kStep)
    by_energy<P, kStep>(s, p, a, c, st);
  else
    by_energy<P, kFinal>(s, p, a, c, st);
}

}  // namespace

void launch_lj(const Sys &s, const LJParams &p, int precision, Mode mode, StepArgs a,
               const LaunchCfg &cfg, cudaStream_t st) {
  if (precision == 0)
    by_mode<Fp64>(s, p, mode, a, cfg, st);
  else
    by_mode<Mixed>(s, p, mode, a, cfg, st);
}

}  // namespace mdk
