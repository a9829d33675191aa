// k_lj_cells.cu -- Lennard-Jones forces from the cell lists themselves, one
// warp per cell with the neighbour cells staged in shared memory (GB300,
// sm_103a): the list-free, tiled alternative to the Verlet-list kernel.
//
// Paper passages: the cell grid (bucket sort into cells of size >= R,
// 3 x 3 x 3 cell template; Sec. "Neighbor lists construction") and the force
// sum f_i = sum_j V'(r_ij) r_ji / r_ji (Sec. "Potentials support"); velocity
// Verlet as in k_lj.cu.
//
// The cells are the ones of the last list build (atoms sorted into them,
// cell size h >= r_ns = rc + skin).  While no atom has moved more than
// skin/2 since then, two atoms closer than rc are in the same or adjacent
// build cells, so scanning the 27 cells of the template and testing the
// current distance against rc finds every pair: no Verlet list is written or
// read (the build skips k_build's list).  A warp owns one cell: its lanes are
// the cell's atoms (in chunks of 32), and for every template cell the warp
// copies 32 neighbour records at a time into its shared tile, then every lane
// tests them all against its atom (the loads are shared by the whole cell).
// Each pair is tested ~27 h^3 / (4/3 pi rc^3) times more often than a
// Verlet-list entry is read, in exchange for no list traffic and no list
// build.  The per-atom sums and the epilogue are those of k_lj.
#include "lj_pair.cuh"

namespace mdk {
namespace {

using namespace pair;

// template cell cd + sd of nc cells: index and periodic image (false: none)
__device__ __forceinline__ bool tmpl_cell(int cd, int sd, int nc, int per, int *cell, int *img) {
  int c = cd + sd, n = 0;
  if (per) {
    if (c < 0) {
      c += nc;
      n = -1;
    } else if (c >= nc) {
      c -= nc;
      n = 1;
    }
  } else if (c < 0 || c >= nc) {
    return false;
  }
  *cell = c;
  *img = n;
  return true;
}

constexpr int kCellWarps = 8;  // warps per block (at most 256 threads)

template <class P, int MODE, bool ENERGY, int SHIFT>
__global__ void __launch_bounds__(256, 4) k_lj_cells(Sys s, LJParams lp, StepArgs a) {
  using GP = G<P>;
  using R = typename GP::R;
  using V = typename GP::V;
  __shared__ V tile[kCellWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= s.n_cells || s.st->abort) return;  // whole warps leave together
  const int b0 = s.cell_start[c], b1 = s.cell_start[c + 1];
  if (b0 >= b1) return;
  const size_t Nc = s.N_cap;
  const V *__restrict__ pg = (const V *)s.pg[a.cur];
  const LJc<R> lc(lp);
  const Grid &g = s.grid[GP::info(GP::ld(pg + b0)) >> 8];
  R hx, hy, hz;
  GP::h(g, hx, hy, hz);
  const int loc = c - g.cell_off;
  const int c0 = loc % g.nc[0], c1 = (loc / g.nc[0]) % g.nc[1], c2 = loc / (g.nc[0] * g.nc[1]);
  V *tl = tile[warp];
  for (int i0 = b0; i0 < b1; i0 += 32) {
    const int i = i0 + lane;
    const bool valid = i < b1;
    V pi;
    uint32_t inf = 0;
    if (valid) {
      pi = GP::ld(pg + i);
      inf = GP::info(pi);
    } else {
      pi = GP::ld(pg + b0);
    }
    Acc<R> fx, fy, fz;
    // energy and virial sums in FP64 (ENERGY passes only: thermo and compute)
    double e = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    for (int t = 0; t < 27; ++t) {
      const int sx = t % 3 - 1, sy = (t / 3) % 3 - 1, sz = t / 9 - 1;
      int cx, cy, cz, nx, ny, nz;
      if (!tmpl_cell(c0, sx, g.nc[0], g.per[0], &cx, &nx) ||
          !tmpl_cell(c1, sy, g.nc[1], g.per[1], &cy, &ny) ||
          !tmpl_cell(c2, sz, g.nc[2], g.per[2], &cz, &nz))
        continue;
      const int cj = g.cell_off + cx + g.nc[0] * (cy + g.nc[1] * cz);
      const int a0 = s.cell_start[cj], a1 = s.cell_start[cj + 1];
      // d = (p_j - p_i) + s h, as q = p_i - s h once per template cell
      const R qx = (R)pi.x - (R)sx * hx, qy = (R)pi.y - (R)sy * hy, qz = (R)pi.z - (R)sz * hz;
      const int self = (nx == 0 && ny == 0 && nz == 0 && valid) ? i : -1;
      for (int j0 = a0; j0 < a1; j0 += 32) {
        __syncwarp();
        if (j0 + lane < a1) tl[lane] = GP::ld(pg + j0 + lane);
        __syncwarp();
        const int m = min(32, a1 - j0);
        for (int k = 0; k < m; ++k) {
          const V pj = tl[k];
          const R dx = (R)pj.x - qx, dy = (R)pj.y - qy, dz = (R)pj.z - qz;
          const R r2 = dx * dx + dy * dy + dz * dz;
          if (valid && r2 < lc.rc2 && j0 + k != self) {
            R fr, v;
            lj_pair<GP, SHIFT, ENERGY>(lc, r2, fr, v);
            fx.add(fr * dx);
            fy.add(fr * dy);
            fz.add(fr * dz);
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
        }
      }
    }
    if (valid) {
      if (ENERGY) {
        s.ea[i] = (double)e;
        s.wa[i] = (double)w0;
        s.wa[Nc + i] = (double)w1;
        s.wa[2 * Nc + i] = (double)w2;
        s.wa[3 * Nc + i] = (double)w3;
        s.wa[4 * Nc + i] = (double)w4;
        s.wa[5 * Nc + i] = (double)w5;
      }
      epilogue<P, MODE, ENERGY>(s, a, i, inf, fx.getf(), fy.getf(), fz.getf());
    }
  }
}

template <class P, int MODE, bool EN, int SH>
void go(const Sys &s, const LJParams &p, StepArgs a, int block, cudaStream_t st) {
  const int warps = (block > 256 ? 256 : block) / 32;
  const int cells = s.n_cells > 0 ? s.n_cells : 1;
  k_lj_cells<P, MODE, EN, SH><<<(cells + warps - 1) / warps, 32 * warps, 0, st>>>(s, p, a);
}

template <class P, int MODE, bool EN>
void by_shift(const Sys &s, const LJParams &p, StepArgs a, int block, cudaStream_t st) {
  if (p.shift_mode == 2)
    go<P, MODE, EN, 2>(s, p, a, block, st);
  else
    go<P, MODE, EN, 1>(s, p, a, block, st);
}

template <class P, int MODE>
void by_energy(const Sys &s, const LJParams &p, StepArgs a, int block, cudaStream_t st) {
  if (a.energy)
    by_shift<P, MODE, true>(s, p, a, block, st);
  else
    by_shift<P, MODE, false>(s, p, a, block, st);
}

template <class P>
void by_mode(const Sys &s, const LJParams &p, Mode m, StepArgs a, int block, cudaStream_t st) {
  if (m == kForceOnly)
    by_energy<P, kForceOnly>(s, p, a, block, st);
  else if (m == kStep)
    by_energy<P, kStep>(s, p, a, block, st);
  else
    by_energy<P, kFinal>(s, p, a, block, st);
}

}  // namespace

void launch_lj_cells(const Sys &s, const LJParams &p, int precision, Mode mode, StepArgs a,
                     const LaunchCfg &cfg, cudaStream_t st) {
  if (precision == 0)
    by_mode<Fp64>(s, p, mode, a, cfg.block, st);
  else
    by_mode<Mixed>(s, p, mode, a, cfg.block, st);
}

}  // namespace mdk
