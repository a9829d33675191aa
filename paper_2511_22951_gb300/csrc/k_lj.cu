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

// mixed: 4 blocks of 256 per SM (64 registers); its energy passes (thermo
// and compute steps only) 3 blocks (80 registers: the per-atom energy and
// virial sums spill at 64), 2 with the shifted-force terms; FP64: 2 blocks
// (128 registers: the FP64 pair values need them)
template <class P, bool ENERGY, int SHIFT>
constexpr int lj_min_blocks() {
  return sizeof(typename G<P>::R) == 4 ? (ENERGY ? (SHIFT == 2 ? 2 : 3) : 4) : 2;
}

// ---- the mixed path: two list entries per instruction ------------------------
// GB300's packed FP32 instructions (FADD2 / FMUL2 / FFMA2) apply one operation
// to two FP32 lanes of a register pair, so two list entries share every
// floating-point instruction of the pair vector, the distance, the LJ force
// and the accumulation; the issue slots saved go to the gathers and the list
// decoding.  Each lane's arithmetic is the scalar path's (same roundings, FMA
// where that path contracts).  Entries past the list end (pad_entry) read a
// far-away record (r^2 ~ 1e36 > rc^2), so the cutoff test is the only mask.
// ENERGY passes take the same walk (identical forces) and sum the pair
// energies and virials as the forces (block sums of four, compensated across
// blocks, FP64 once per atom).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int T, int SHIFT, bool ENERGY>
__device__ __forceinline__ void lj_walk_packed(const Sys &s, const float4 *__restrict__ pg,
                                               int i, int nn, int t, const float4 pi,
                                               float hx, float hy, float hz,
                                               const LJc<float> &lc, Acc<float> &fx,
                                               Acc<float> &fy, Acc<float> &fz, double &esum,
                                               double (&w)[6]) {
  const size_t Nc = s.N_cap;
  const size_t gstride = Nc * 2;  // uint4 per group row
  const uint4 *__restrict__ row = reinterpret_cast<const uint4 *>(s.nbr) + (size_t)i * 2 +
                                  (size_t)t * gstride;
  const float2 mpx = f2(-pi.x, -pi.x), mpy = f2(-pi.y, -pi.y), mpz = f2(-pi.z, -pi.z);
  const float2 hx2 = f2(hx, hx), hy2 = f2(hy, hy), hz2 = f2(hz, hz);
  // minus the magic constants of s_scaled (2^23 + 4^d)
  const float2 k0 = f2(-8388609.0f, -8388609.0f), k1 = f2(-8388612.0f, -8388612.0f),
               k2 = f2(-8388624.0f, -8388624.0f);
  const float2 sig2 = f2(lc.sig2, lc.sig2), meps24 = f2(-lc.eps24, -lc.eps24);
  const float2 two = f2(2.0f, 2.0f), mone = f2(-1.0f, -1.0f);
  // ENERGY: compensated FP32 sums of the block sums (as the forces), in FP64
  // once per atom at the end
  Acc<float> ae, aw[6];
  uint4 na = make_uint4(0, 0, 0, 0), nb = na;
  if (kGroup * t < nn) {
    ld_group(row, na, nb);
  }
  for (int k = kGroup * t; k < nn; k += kGroup * T) {
    const uint4 ga = na, gb = nb;
    row += gstride * T;
    if (k + kGroup * T < nn) {
      ld_group(row, na, nb);
    }
    const uint32_t e[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      // whole groups: the slots past the list's length hold pad_entry, whose
      // record lies 1e18 A away (r^2 ~ 1e36 > rc^2)
      float4 q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = __ldg(pg + dbg_idx(s, nbr_j(e[4 * h + u]), Nc + 1));
      float2 bx = f2(0.f, 0.f), by = bx, bz = bx;
      // ENERGY: FP32 sums of this block's four pair energies and virial
      // terms, added to the FP64 per-atom sums once per block
      float2 be = bx, bw0 = bx, bw1 = bx, bw2 = bx, bw3 = bx, bw4 = bx, bw5 = bx;
#pragma unroll
      for (int pr = 0; pr < 2; ++pr) {
        const uint32_t ea = e[4 * h + 2 * pr], eb = e[4 * h + 2 * pr + 1];
        const float4 qa = q[2 * pr], qb = q[2 * pr + 1];
        // stencil shifts s_d 4^d, then d = (p_j - p_i) + s h (h pre-scaled)
        const float2 sx = __fadd2_rn(f2(__uint_as_float((ea & 3u) | 0x4B000000u),
                                        __uint_as_float((eb & 3u) | 0x4B000000u)), k0);
        const float2 sy = __fadd2_rn(f2(__uint_as_float((ea & 12u) | 0x4B000000u),
                                        __uint_as_float((eb & 12u) | 0x4B000000u)), k1);
        const float2 sz = __fadd2_rn(f2(__uint_as_float((ea & 48u) | 0x4B000000u),
                                        __uint_as_float((eb & 48u) | 0x4B000000u)), k2);
        const float2 dx = __ffma2_rn(sx, hx2, __fadd2_rn(f2(qa.x, qb.x), mpx));
        const float2 dy = __ffma2_rn(sy, hy2, __fadd2_rn(f2(qa.y, qb.y), mpy));
        const float2 dz = __ffma2_rn(sz, hz2, __fadd2_rn(f2(qa.z, qb.z), mpz));
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        // V'(r)/r = -24 eps (2 (sigma/r)^12 - (sigma/r)^6) / r^2
        const float2 inv = f2(__fdividef(1.0f, r2.x), __fdividef(1.0f, r2.y));
        const float2 s2 = __fmul2_rn(sig2, inv);
        const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
        float2 fr = __fmul2_rn(__fmul2_rn(meps24, __ffma2_rn(s6, two, mone)),
                               __fmul2_rn(s6, inv));
        if (SHIFT == 2) {  // shifted force: - V'(rc) / r
          fr.x -= lc.durc / sqrtf(r2.x);
          fr.y -= lc.durc / sqrtf(r2.y);
        }
        const bool ina = r2.x < lc.rc2, inb = r2.y < lc.rc2;
        fr.x = ina ? fr.x : 0.0f;
        fr.y = inb ? fr.y : 0.0f;
        bx = __ffma2_rn(fr, dx, bx);
        by = __ffma2_rn(fr, dy, by);
        bz = __ffma2_rn(fr, dz, bz);
        if (ENERGY) {  // energy and virial from the same pair values
          float2 v = __ffma2_rn(f2(lc.eps4, lc.eps4), __ffma2_rn(s6, s6, f2(-s6.x, -s6.y)),
                                f2(-lc.ush, -lc.ush));
          if (SHIFT == 2) {
            v.x -= (sqrtf(r2.x) - lc.rcut) * lc.durc;
            v.y -= (sqrtf(r2.y) - lc.rcut) * lc.durc;
          }
          v.x = ina ? v.x : 0.0f;
          v.y = inb ? v.y : 0.0f;
          be = __fadd2_rn(be, v);
          const float2 hf = __fmul2_rn(f2(-0.5f, -0.5f), fr);  // r_ij = -d
          const float2 hx_ = __fmul2_rn(hf, dx), hy_ = __fmul2_rn(hf, dy);
          bw0 = __ffma2_rn(hx_, dx, bw0);
          bw1 = __ffma2_rn(hy_, dy, bw1);
          bw2 = __ffma2_rn(__fmul2_rn(hf, dz), dz, bw2);
          bw3 = __ffma2_rn(hx_, dy, bw3);
          bw4 = __ffma2_rn(hx_, dz, bw4);
          bw5 = __ffma2_rn(hy_, dz, bw5);
        }
      }
      fx.add(bx.x + bx.y);
      fy.add(by.x + by.y);
      fz.add(bz.x + bz.y);
      if (ENERGY) {
        ae.add(0.5f * (be.x + be.y));
        aw[0].add(bw0.x + bw0.y);
        aw[1].add(bw1.x + bw1.y);
        aw[2].add(bw2.x + bw2.y);
        aw[3].add(bw3.x + bw3.y);
        aw[4].add(bw4.x + bw4.y);
        aw[5].add(bw5.x + bw5.y);
      }
    }
  }
  if (ENERGY) {
    esum += ae.get();
#pragma unroll
    for (int c = 0; c < 6; ++c) w[c] += aw[c].get();
  }
}

template <class P, int MODE, bool ENERGY, int SHIFT, int T>
__global__ void __launch_bounds__(256, lj_min_blocks<P, ENERGY, SHIFT>()) k_lj(Sys s, LJParams lp, StepArgs a) {
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
      h_scaled(hx, hy, hz);  // for s_scaled
      nn = min(s.nnbr[i], s.nmax);
    }
    Acc<R> fx, fy, fz;
    // per-atom energy and virial (ENERGY passes only: thermo and compute):
    // FP64 sums on the FP64 path, the packed walk's compensated sums (in
    // FP64 once per atom) on the mixed path
    double e = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    R bx = 0, by = 0, bz = 0;  // block sums of four pairs
    if constexpr (sizeof(R) == 4) {
      double wv[6] = {0, 0, 0, 0, 0, 0};
      lj_walk_packed<T, SHIFT, ENERGY>(s, reinterpret_cast<const float4 *>(pg), i, nn, tl.t,
                                       *reinterpret_cast<const float4 *>(&pi), hx, hy, hz,
                                       *reinterpret_cast<const LJc<float> *>(&lc), fx, fy, fz,
                                       e, wv);
      w0 = wv[0];
      w1 = wv[1];
      w2 = wv[2];
      w3 = wv[3];
      w4 = wv[4];
      w5 = wv[5];
    } else
    walk<T>(
        s.nbr, Nc, i, nn, tl.t, [&](uint32_t j) { return GP::ld(pg + dbg_idx(s, j, Nc)); },
        [&](uint32_t ent, const V &pj) {
          const R dx = pvec((R)pj.x, (R)pi.x, s_scaled(R(0), ent, 0), hx);
          const R dy = pvec((R)pj.y, (R)pi.y, s_scaled(R(0), ent, 1), hy);
          const R dz = pvec((R)pj.z, (R)pi.z, s_scaled(R(0), ent, 2), hz);
          const R r2 = r2_of(dx, dy, dz);
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
