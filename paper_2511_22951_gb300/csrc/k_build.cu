// k_build.cu -- Verlet-list rebuild on the GPU (Sec. "Neighbor lists
// construction" of the paper: a virtual Cartesian grid of cells of size
// >= R = r_ns, one bucket-sort pass of the atoms into the cells, then a
// 3x3x3 cell stencil search; Eq. rhrz gives r_ns = (1 + beta) r_cut, here
// rc + skin).
//
// The chain runs every step and every kernel returns at once unless the
// device flag st->rebuild is set, so the whole step stays on the device
// (no host round trip to decide whether to rebuild):
//   k_pre       count steps since the last build; fixed-interval trigger
//   k_bin       wrap periodic coordinates, cell id per atom, cell histogram
//   k_scan_*    exclusive scan of the histogram (3 phases)
//   k_scatter   counting-sort scatter into cell order (atomic slots)
//   k_cell_sort order each cell's atoms by their permanent id (determinism)
//   k_permute   gather every per-atom array into the new order (scratch)
//   k_copyback  scratch -> primary arrays
//   k_build     Verlet lists (full, or half: each pair once): FP32
//               pre-filter on cell-relative offsets,
//               exact FP64 test for the few candidates near r_ns
//   k_finish    clear the flag, count the build
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "mdk_internal.cuh"

namespace mdk {

namespace {

constexpr int kBlk = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ bool flag_on(const Sys &s) {
  return *(volatile int *)&s.st->rebuild != 0;
}
// a full build: re-bin, re-sort and rebuild the (outer) list from the cells;
// with the outer list off every build is full
__device__ __forceinline__ bool full_on(const Sys &s) {
  return flag_on(s) && *(volatile int *)&s.st->full != 0;
}

__global__ void k_pre(Sys s, int count_step, int use_cond, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DevStatus *st = s.st;
  if (st->abort) {  // stepping stopped at an overflowing build: nothing more
    if (use_cond) cudaGraphSetConditional(h, 0u);
    return;
  }
  st->step_build = count_step;
  st->build_ovf = 0;
  if (count_step) {
    st->since_build += 1;
    st->n_steps += 1;  // index of the force evaluation that follows (Langevin noise)
  }
  if (s.rebuild_every > 0 && st->since_build >= s.rebuild_every) st->rebuild = 1;
  // the window acts at builds that stepping triggers, not at explicit builds
  st->win_active = (s.win_on && count_step && st->rebuild) ? 1 : 0;
  // explicit builds, window builds, list-free forces and a missing outer
  // list take a full build; otherwise k_outer_decide checks the budget
  st->full = (st->rebuild && (!s.outer_on || !count_step || st->win_active ||
                              !st->outer_valid || s.half == 2))
                 ? 1
                 : 0;
  st->win_cut = -INFINITY;
  if (st->win_active) {
    st->key_xmax = dkey(-INFINITY);
    st->key_xmin = dkey(INFINITY);
    st->win_cut = -INFINITY;
    st->win_insert = 0;
  }
  if (use_cond) cudaGraphSetConditional(h, st->rebuild ? 1u : 0u);
}

// ---- moving window (Sec. "Moving window simulation"; rules in mdk.h) ----
// Front: bins of width front_bin along x; a bin is shocked when its mean v_x
// exceeds u_p / 2, decided exactly on velocities rounded to multiples of
// 2^-40 Angstrom/fs (integer sums, so the order of the atomics is irrelevant).
// Leading edge = max x.
constexpr double kTwo40 = 1099511627776.0;
constexpr int kFbinSmem = 2048;  // bins privatised in shared memory up to this count

__device__ __forceinline__ int front_bin_of(const Sys &s, double x) {
  const double u = floor(__ddiv_rn(__dsub_rn(x, s.win_xlo), s.front_bin));
  return u < 0.0 ? 0 : (u > (double)(s.n_fbins - 1) ? s.n_fbins - 1 : (int)u);
}

__global__ void __launch_bounds__(kBlk) k_win_stats(Sys s) {
  __shared__ long long sh[2 * kFbinSmem];
  if (!full_on(s) || !s.st->win_active) return;
  const bool priv = s.n_fbins <= kFbinSmem;
  if (priv)
    for (int q = threadIdx.x; q < 2 * s.n_fbins; q += blockDim.x) sh[q] = 0;
  __syncthreads();
  long long *hist = priv ? sh : s.fbin;
  const int N = s.st->N;
  long long xmax = dkey(-INFINITY);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double x = s.x[i], vx = s.v[i];
    const long long k = dkey(x);
    if (k > xmax) xmax = k;
    if (!isfinite(x) || !isfinite(vx)) continue;
    const int b = front_bin_of(s, x);
    atomicAdd((unsigned long long *)&hist[2 * b], (unsigned long long)__double2ll_rn(vx * kTwo40));
    atomicAdd((unsigned long long *)&hist[2 * b + 1], 1ull);
  }
  for (int o = 16; o > 0; o >>= 1) xmax = max(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&s.st->key_xmax, xmax);
  if (priv) {
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * s.n_fbins; q += blockDim.x)
      if (sh[q] != 0) atomicAdd((unsigned long long *)&s.fbin[q], (unsigned long long)sh[q]);
  }
}

// Front, cut and the number of fresh-slab copies to append (capped by the
// box along x and by the capacity).  One block; the bin sums are cleared
// for the next build.
__global__ void __launch_bounds__(kBlk) k_win_plan(Sys s) {
  __shared__ int best;
  if (!full_on(s) || !s.st->win_active) return;
  if (threadIdx.x == 0) best = -1;
  __syncthreads();
  const long long q_up = __double2ll_rn(s.u_p * kTwo40);
  int mine = -1;
  for (int b = threadIdx.x; b < s.n_fbins; b += blockDim.x) {
    const long long sum = s.fbin[2 * b], cnt = s.fbin[2 * b + 1];
    if (cnt > 0 && 2 * sum > cnt * q_up) mine = b;
  }
  if (mine >= 0) atomicMax(&best, mine);
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * s.n_fbins; q += blockDim.x) s.fbin[q] = 0;
  if (threadIdx.x != 0) return;
  DevStatus *st = s.st;
  const double xmax = dkey_inv(st->key_xmax);
  st->win_n_old = st->N;
  st->win_insert = 0;
  st->win_cut = -INFINITY;
  const bool fixed = isfinite(s.fixed_front);
  if (best < 0 && !fixed) return;
  const double front =
      fixed ? s.fixed_front : __dadd_rn(s.win_xlo, __dmul_rn((double)(best + 1), s.front_bin));
  st->win_cut = front - s.L_behind;
  const double need = front + s.L_ahead - xmax;
  long long copies = need > 0.0 ? (long long)ceil(need / s.slab_lx) : 0;
  const double fit = floor(__ddiv_rn(__dsub_rn(__dsub_rn(s.win_xhi, xmax), s.slab_gap), s.slab_lx));
  const long long fit_n = fit > 0.0 ? (long long)fit : 0;
  if (copies > fit_n) copies = fit_n;
  long long add = copies * (long long)s.n_slab;
  const long long room = (long long)s.N_cap - st->N;
  if (add > room) {
    add = room;
    atomicOr(&st->bits, kStCapacity);
  }
  st->win_insert = (int)add;
  st->win_x0 = xmax;
  st->win_id0 = st->next_id;
  st->next_id += (int)add;
  st->N += (int)add;
  st->n_inserted += add;
}

__global__ void __launch_bounds__(kBlk) k_win_insert(Sys s) {
  if (!full_on(s) || !s.st->win_active) return;
  const DevStatus *st = s.st;
  const int add = st->win_insert, n0 = st->win_n_old, id0 = st->win_id0;
  const size_t Nc = s.N_cap;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < add; q += gridDim.x * blockDim.x) {
    const int c = q / s.n_slab, k = q % s.n_slab;
    const double *a = s.slab + 6 * (size_t)k;
    const int i = n0 + q;
    // copy c sits at x offset (x_max + gap) + c * slab_lx, rounded in that order
    const double x0 = __dadd_rn(__dadd_rn(st->win_x0, s.slab_gap), __dmul_rn((double)c, s.slab_lx));
    s.x[i] = __dadd_rn(a[0], x0);
    s.x[Nc + i] = a[1];
    s.x[2 * Nc + i] = a[2];
    for (int d = 0; d < 3; ++d) {
      s.v[d * Nc + i] = a[3 + d];
      s.f[d * Nc + i] = 0.0;
    }
    s.id[i] = id0 + q;
    s.info[i] = s.slab_info;
  }
}

// atoms a window deleted sit in the last bucket, past the kept ones: drop them
__global__ void k_win_trim(Sys s) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || !full_on(s)) return;
  DevStatus *st = s.st;
  const int kept = s.cell_start[s.n_cells];
  st->n_deleted += st->N - kept;
  st->N = kept;
}


__global__ void k_set_flag(Sys s) {
  if (threadIdx.x == 0 && blockIdx.x == 0) s.st->rebuild = 1;
}

__global__ void __launch_bounds__(kBlk) k_bin(Sys s) {
  if (!full_on(s)) return;
  const int N = s.st->N;
  const bool win = s.win_on && s.st->win_active;
  long long xmin = dkey(INFINITY);  // smallest x kept (window: new rear layer)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
  const Grid &g = s.grid[s.info[i] >> 8];
  if (win) {
    const double x = s.x[i];
    if (x < s.st->win_cut) {  // behind the window: to the deletion bucket
      s.cell_of[i] = s.n_cells;
      s.tmpu[i] = 0;
      atomicAdd(&s.cell_cnt[s.n_cells], 1);
      continue;
    }
    xmin = min(xmin, dkey(x));
  }
  int c[3];
  for (int d = 0; d < 3; ++d) {
    double xv = s.x[(size_t)d * s.N_cap + i];
    if (!isfinite(xv)) {
      atomicOr(&s.st->bits, kStNonfinite);
      xv = g.lo[d];
      s.x[(size_t)d * s.N_cap + i] = xv;
    }
    if (g.per[d]) {
      const double lo = g.lo[d], hi = g.hi[d], L = g.L[d];
      if (xv >= hi || xv < lo) {
        // whole box lengths, one at a time (as the definition states);
        // atoms more than 4 boxes away jump by a floor first
        if (fabs(xv - lo) > 4.0 * L) xv = xv - L * floor((xv - lo) / L);
        for (int it = 0; it < 8 && xv >= hi; ++it) xv = xv - L;
        for (int it = 0; it < 8 && xv < lo; ++it) xv = xv + L;
        if (xv >= hi || xv < lo) xv = lo;
        s.x[(size_t)d * s.N_cap + i] = xv;
      }
    }
    int ck = (int)floor((xv - g.lo[d]) * g.inv_h[d]);
    ck = min(max(ck, 0), g.nc[d] - 1);
    c[d] = ck;
  }
  const int cell = g.cell_off + c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
  s.cell_of[i] = cell;
  s.tmpu[i] = pack_cell(c[0], c[1], c[2]);
  atomicAdd(&s.cell_cnt[cell], 1);
  }
  if (win) {  // one atomic per warp, not per atom
    for (int o = 16; o > 0; o >>= 1) xmin = min(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
    if ((threadIdx.x & 31) == 0) atomicMin(&s.st->key_xmin, xmin);
  }
}

// block-wide exclusive scan of one value per thread; returns the prefix and
// writes the block total to *total
__device__ __forceinline__ int block_exscan(int v, int *total) {
  __shared__ int warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    int w = (lane < nw) ? warp_sums[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) warp_sums[lane] = wi - w;
    if (lane == nw - 1) *total = wi;
  }
  __syncthreads();
  const int res = warp_sums[warp] + incl - v;
  __syncthreads();
  return res;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(Sys s) {
  if (!full_on(s)) return;
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int sum = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q)
    if (base + q <= s.n_cells) sum += s.cell_cnt[base + q];
  __shared__ int tot;
  block_exscan(sum, &tot);
  if (threadIdx.x == 0) s.scan_part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(Sys s) {
  if (!full_on(s)) return;
  // n_scan_blocks <= kScanThreads * 8
  constexpr int kPer = 8;
  const int base = threadIdx.x * kPer;
  int loc[kPer];
  int sum = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    loc[q] = (base + q < s.n_scan_blocks) ? s.scan_part[base + q] : 0;
    sum += loc[q];
  }
  __shared__ int tot;
  int pre = block_exscan(sum, &tot);
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    if (base + q < s.n_scan_blocks) s.scan_part[base + q] = pre;
    pre += loc[q];
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(Sys s) {
  if (!full_on(s)) return;
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int loc[kScanItems];
  int sum = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    loc[q] = (base + q <= s.n_cells) ? s.cell_cnt[base + q] : 0;
    sum += loc[q];
  }
  __shared__ int tot;
  int pre = block_exscan(sum, &tot) + s.scan_part[blockIdx.x];
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    const int c = base + q;
    if (c <= s.n_cells) {
      s.cell_start[c] = pre;
      s.cell_fill[c] = pre;
      s.cell_cnt[c] = 0;  // ready for the next build
    }
    pre += loc[q];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1)
    s.cell_start[s.n_cells + 1] = pre;
}

__global__ void __launch_bounds__(kBlk) k_scatter(Sys s) {
  if (!full_on(s)) return;
  const int N = s.st->N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
  const int pos = atomicAdd(&s.cell_fill[dbg_idx(s, s.cell_of[i], s.n_cells + 1)], 1);
  s.order[dbg_idx(s, pos, s.N_cap)] = i;
  }
}

// Order inside each cell by permanent atom id, so the layout does not depend
// on the order of the scatter's atomics: the atom at slot k of its cell takes
// rank = number of atoms of the cell with a smaller id, and lands at
// cell_start + rank of the final order (kept in tmpi, which k_permute reads
// first and overwrites at the same index).  One thread per atom: the
// comparisons of a cell run in parallel, with independent loads.  Atoms a
// window deletes (the last bucket) keep the scatter's order.
__global__ void __launch_bounds__(kBlk) k_cell_sort(Sys s) {
  if (!full_on(s)) return;
  const int N = s.st->N;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const int v = s.order[k];
    const int b = s.cell_of[v];
    const int a = s.cell_start[b], e = s.cell_start[b + 1];
    int rank = k - a;
    if (b < s.n_cells) {
      const int key = s.id[v];
      rank = 0;
#pragma unroll 4
      for (int q = a; q < e; ++q) rank += s.id[s.order[q]] < key ? 1 : 0;
    }
    s.tmpi[dbg_idx(s, a + rank, s.N_cap)] = v;
  }
}

template <class P>
__global__ void __launch_bounds__(kBlk) k_permute(Sys s, typename P::vec4 *pg_target) {
  if (!full_on(s)) return;
  const int N = s.st->N;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
  const size_t Nc = s.N_cap;
  const int o = dbg_idx(s, s.tmpi[k], s.N_cap);  // the cell-sorted order (k_cell_sort)
  double xv[3];
  for (int d = 0; d < 3; ++d) {
    xv[d] = s.x[d * Nc + o];
    s.tmp[d * Nc + k] = xv[d];
    s.tmp[(3 + d) * Nc + k] = s.v[d * Nc + o];
    s.tmp[(6 + d) * Nc + k] = s.f[d * Nc + o];
    s.xref[d * Nc + k] = xv[d];
  }
  s.tmpi[k] = s.id[o];
  const uint32_t cc = s.tmpu[o];
  s.cellc[k] = cc;
  uint32_t inf = s.info[o] & ~kInfoFar;
  if (s.win_on && s.st->win_active && s.st->win_cut > -INFINITY &&
      xv[0] < dkey_inv(s.st->key_xmin) + s.piston_depth)
    inf |= kInfoPiston;
  const Grid &g = s.grid[inf >> 8];
  double p[3];
  bool far = false;
  for (int d = 0; d < 3; ++d) {
    p[d] = xv[d] - cell_center(g, d, cell_coord(cc, d));
    // the FP32 pre-filter bound assumes |p| <= 2h (true for periodic
    // dimensions after wrapping); atoms clamped into an end cell of a free
    // dimension may lie further out and always take the exact test
    if (!(fabs(p[d]) <= 2.0 * g.h[d])) far = true;
  }
  if (far) inf |= kInfoFar;
  s.tmpu[Nc + k] = inf;
  // a far atom's pre-filter offset is NaN: every float r^2 with it is NaN,
  // fails both band tests and so always takes the exact FP64 test
  s.pf[k] = far ? make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, __uint_as_float(inf))
                : Mixed::make(p[0], p[1], p[2], inf);
  pg_target[k] = P::make(p[0], p[1], p[2], inf);
  }
}

__global__ void __launch_bounds__(kBlk) k_copyback(Sys s) {
  if (!full_on(s)) return;
  const int N = s.st->N;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
  const size_t Nc = s.N_cap;
  for (int d = 0; d < 3; ++d) {
    s.x[d * Nc + k] = s.tmp[d * Nc + k];
    s.v[d * Nc + k] = s.tmp[(3 + d) * Nc + k];
    s.f[d * Nc + k] = s.tmp[(6 + d) * Nc + k];
  }
  s.id[k] = s.tmpi[k];
  s.info[k] = s.tmpu[Nc + k];
  }
}

// periodic image crossed when stencil offset sd leaves cell cd of nc cells
__device__ __forceinline__ bool stencil_cell(int cd, int sd, int nc, int per, int *cell,
                                             int *img) {
  int c = cd + sd;
  int n = 0;
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

// Verlet lists (the paper's 3x3x3 cell template), one thread per atom in
// cell order, so the lanes of a warp share most of their stencil cells.
// Accepted entries are staged in shared memory (two groups of 8 per thread,
// written while the other is flushed) and reach HBM as full 32-byte sectors
// of the list layout.  The candidate loop is branch-free: every candidate is
// stored into the next slot and the count advances only when it is accepted.
// Candidates near r_ns, and far atoms (NaN offsets), take the exact FP64 test
// of the definition.
__device__ __forceinline__ int image_of(int c, int sd, int nc, int per) {
  if (!per) return 0;
  const int q = c + sd;
  return q < 0 ? -1 : (q >= nc ? 1 : 0);
}

// The definition, rounded step by step without contraction, for a candidate
// inside the pre-filter band or with a far atom:
// d = (x_j - x_i) + n L,  r^2 = (dx^2 + dy^2) + dz^2 < r_ns^2.
__device__ __noinline__ bool exact_pair(const Sys &s, const Grid &g, int i, uint32_t code, int c0,
                                        int c1, int c2, double rns2) {
  const size_t Nc = s.N_cap;
  const int j = nbr_j(code);
  const int nx = image_of(c0, nbr_s(code, 0), g.nc[0], g.per[0]);
  const int ny = image_of(c1, nbr_s(code, 1), g.nc[1], g.per[1]);
  const int nz = image_of(c2, nbr_s(code, 2), g.nc[2], g.per[2]);
  const double ex = __dadd_rn(__dadd_rn(s.x[j], -s.x[i]), __dmul_rn((double)nx, g.L[0]));
  const double ey = __dadd_rn(__dadd_rn(s.x[Nc + j], -s.x[Nc + i]), __dmul_rn((double)ny, g.L[1]));
  const double ez =
      __dadd_rn(__dadd_rn(s.x[2 * Nc + j], -s.x[2 * Nc + i]), __dmul_rn((double)nz, g.L[2]));
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
  return r2 < rns2;
}

// Half lists keep each unordered pair in one of its two atoms' lists: for
// j != i in the list of the smaller index when i + j is even and of the
// larger when it is odd (so every atom keeps about half of its neighbours,
// whatever its place in the cell order).  (i, j, s) and (j, i, -s) pass the
// same distance test, so the half list is exactly one of each mirror pair.
__device__ __forceinline__ bool half_keep(int i, int j, bool s_pos) {
  if (j == i) return s_pos;
  return (i < j) == (((i ^ j) & 1) == 0);
}

// HALF: the list kind is a template parameter, so a full list's candidate
// loop carries no half-list test
// where a build writes: the Verlet list (s.nbr), or with the outer list on
// the outer list (s.nbr1, radius rc + skin_outer, always full)
struct ListOut {
  uint32_t *nbr;
  int32_t *nnbr;
  int nmax;
  double rns2;
  float lo, hi;
  int *max_seen;
};

template <bool HALF>
__global__ void __launch_bounds__(kBlk) k_build(Sys s, ListOut lo_) {
  __shared__ uint32_t stage[2 * kGroup][kBlk];
  if (!full_on(s) || s.half == 2) return;  // 2: forces straight from the cells, no list
  const int N = s.st->N;
  const size_t Nc = s.N_cap;
  const float lo_thr = lo_.lo, hi_thr = lo_.hi;
  const double rns2 = lo_.rns2;
  const int ngroups = lo_.nmax / kGroup;
  constexpr bool half = HALF;
  const int tx = threadIdx.x;
  for (int i = blockIdx.x * kBlk + tx; i < N; i += gridDim.x * kBlk) {
    const float4 pi = __ldg(s.pf + i);
    const Grid &g = s.grid[__float_as_uint(pi.w) >> 8];
    const uint32_t cc = s.cellc[i];
    const int c0 = cell_coord(cc, 0), c1 = cell_coord(cc, 1), c2 = cell_coord(cc, 2);
    int count = 0;
    auto flush = [&](int grp, int fill) {
      if (grp >= ngroups) return;
      const int h = (grp & 1) * kGroup;
      const uint32_t pad = pad_entry(Nc);
      uint32_t w[kGroup];
#pragma unroll
      for (int q = 0; q < kGroup; ++q) w[q] = q < fill ? stage[h + q][tx] : pad;
      uint4 *o = reinterpret_cast<uint4 *>(lo_.nbr) + ((size_t)grp * Nc + i) * 2;
      // lists are written once per build and read by the next pass from
      // HBM: evict-first stores keep L2 for the records the builds gather
      __stcs(o, make_uint4(w[0], w[1], w[2], w[3]));
      __stcs(o + 1, make_uint4(w[4], w[5], w[6], w[7]));
    };
    for (int t = 0; t < 27; ++t) {
      const int sx = t % 3 - 1, sy = (t / 3) % 3 - 1, sz = t / 9 - 1;
      int cx, cy, cz, nx, ny, nz;
      if (!stencil_cell(c0, sx, g.nc[0], g.per[0], &cx, &nx) ||
          !stencil_cell(c1, sy, g.nc[1], g.per[1], &cy, &ny) ||
          !stencil_cell(c2, sz, g.nc[2], g.per[2], &cz, &nz))
        continue;
      const int cj = dbg_idx(s, g.cell_off + cx + g.nc[0] * (cy + g.nc[1] * cz), s.n_cells);
      const int a = s.cell_start[cj], b = dbg_idx(s, s.cell_start[cj + 1], s.N_cap + 1, a);
      // d = p_j - q with q = p_i - s h (the shifted own offset, once per cell)
      const float qx = pi.x - (float)sx * g.hf[0];
      const float qy = pi.y - (float)sy * g.hf[1];
      const float qz = pi.z - (float)sz * g.hf[2];
      const int self = (nx == 0 && ny == 0 && nz == 0) ? i : -1;
      const uint32_t code = pack_nbr(0, sx, sy, sz);
      // half lists: an image of i itself is kept for the lexicographically
      // positive stencil offset only (its mirror has the negative one)
      const bool s_pos = sz > 0 || (sz == 0 && (sy > 0 || (sy == 0 && sx > 0)));
      // blocks of four candidates; FULL: all four inside the cell's range
      const float2 mqx = make_float2(-qx, -qx), mqy = make_float2(-qy, -qy),
                   mqz = make_float2(-qz, -qz);
      auto block4 = [&](const int j0, auto full) {
        constexpr bool FULL = decltype(full)::value;
        const int before = count;
        float4 pj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) pj[u] = __ldg(s.pf + (FULL ? j0 + u : min(j0 + u, b - 1)));
        // r^2 of two candidates per packed FP32 instruction
        float r2v[4];
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
          const float4 &qa = pj[2 * pr], &qb = pj[2 * pr + 1];
          const float2 dx = __fadd2_rn(make_float2(qa.x, qb.x), mqx);
          const float2 dy = __fadd2_rn(make_float2(qa.y, qb.y), mqy);
          const float2 dz = __fadd2_rn(make_float2(qa.z, qb.z), mqz);
          const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
          r2v[2 * pr] = r2.x;
          r2v[2 * pr + 1] = r2.y;
        }
        bool band = false;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u;
          const float r2f = r2v[u];
          const bool ok = (FULL || j < b) && j != self && (!half || half_keep(i, j, s_pos));
          const bool acc = ok && r2f < lo_thr;
          band = band || (ok && !acc && !(r2f > hi_thr));
          stage[count & 15][tx] = code | ((uint32_t)j << 6);  // kept only if accepted
          count += acc ? 1 : 0;
        }
        if (band) {
          // rare: redo this block of four with the exact test where needed
          count = before;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = j0 + u;
            const float r2f = r2v[u];
            const bool ok = (FULL || j < b) && j != self && (!half || half_keep(i, j, s_pos));
            bool acc = ok && r2f < lo_thr;
            if (ok && !acc && !(r2f > hi_thr))
              acc = exact_pair(s, g, i, code | ((uint32_t)j << 6), c0, c1, c2, rns2);
            stage[count & 15][tx] = code | ((uint32_t)j << 6);
            count += acc ? 1 : 0;
          }
        }
        // a group of 8 completed in this block: write it out
        if ((before >> 3) != (count >> 3)) flush(before >> 3, kGroup);
      };
      int j0 = a;
      for (; j0 + 4 <= b; j0 += 4) block4(j0, std::true_type());
      if (j0 < b) block4(j0, std::false_type());
    }
    if (count & 7) flush(count >> 3, count & 7);
    lo_.nnbr[i] = count;
    if (count > lo_.nmax) {
      atomicOr(&s.st->bits, kStOverflow);
      atomicMax(lo_.max_seen, count);
      s.st->build_ovf = 1;
    }
  }
}

// ---- two-level lists: the Verlet list filtered from the outer list ----------
// Every build measures d, the largest displacement of an atom since the last
// full build (x_full: positions right after that build).  A pair closer than
// rc + skin now was closer than rc + skin + 2 d then, so while
// d <= (skin_outer - skin) / 2 the outer list holds every pair within
// rc + skin, and filtering it gives the exact Verlet list.
__global__ void __launch_bounds__(kBlk) k_outer_disp(Sys s) {
  if (!flag_on(s) || !s.outer_on || s.st->full) return;
  const int N = s.st->N;
  const size_t Nc = s.N_cap;
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double dx = s.x[i] - s.xfull[i], dy = s.x[Nc + i] - s.xfull[Nc + i],
                 dz = s.x[2 * Nc + i] - s.xfull[2 * Nc + i];
    const double d2 = dx * dx + dy * dy + dz * dz;
    // a non-finite position forces a full build (whose binning reports it)
    m = d2 == d2 ? fmax(m, d2) : INFINITY;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  // non-negative doubles order like their bit patterns
  if ((threadIdx.x & 31) == 0) atomicMax(&s.st->dmax_key, __double_as_longlong(m));
}

__global__ void k_outer_decide(Sys s) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || !flag_on(s) || !s.outer_on) return;
  DevStatus *st = s.st;
  if (!st->full) {
    // sqrt rounded up by one part in 2^40: the bound stays a bound
    const double d = sqrt(__longlong_as_double(st->dmax_key)) * (1.0 + 0x1p-40);
    st->d_acc = d;
    if (!(d <= s.outer_budget)) st->full = 1;
  }
  if (st->full) {
    st->d_acc = 0.0;
    st->outer_valid = 1;  // the chain below rebuilds the outer list
    st->n_full_builds += 1;
  }
  st->dmax_key = 0;
}

// full builds: x_full = x (after the re-sort); filter builds: the trigger's
// reference positions (FP64 x_ref and the FP32 cell-relative record the
// pre-filter reads) move to the current positions; atoms keep their cells,
// so the outer list's stencil codes stay exact
__global__ void __launch_bounds__(kBlk) k_outer_refresh(Sys s) {
  if (!flag_on(s) || !s.outer_on) return;
  const int N = s.st->N;
  const size_t Nc = s.N_cap;
  if (s.st->full) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
      for (int d = 0; d < 3; ++d) s.xfull[d * Nc + i] = s.x[d * Nc + i];
    return;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double p[3];
    const uint32_t cc = s.cellc[i];
    const uint32_t inf = s.info[i];
    const Grid &g = s.grid[inf >> 8];
    for (int d = 0; d < 3; ++d) {
      const double xv = s.x[d * Nc + i];
      s.xref[d * Nc + i] = xv;
      p[d] = xv - cell_center(g, d, cell_coord(cc, d));
    }
    if (!(inf & kInfoFar)) s.pf[i] = Mixed::make(p[0], p[1], p[2], inf);
  }
}

// the Verlet list (full or half) from the outer list: the same FP32
// pre-filter, band and exact FP64 test as k_build, on the outer list's
// candidates in their order (so the list equals a build from the cells)
template <bool HALF>
__global__ void __launch_bounds__(kBlk) k_build_filter(Sys s) {
  __shared__ uint32_t stage[2 * kGroup][kBlk];
  if (!flag_on(s) || !s.outer_on || s.half == 2) return;
  const int N = s.st->N;
  const size_t Nc = s.N_cap;
  const float lo_thr = s.filt_lo, hi_thr = s.filt_hi;
  const double rns2 = s.rns2;
  const int ngroups = s.nmax / kGroup;
  const int tx = threadIdx.x;
  for (int i = blockIdx.x * kBlk + tx; i < N; i += gridDim.x * kBlk) {
    const float4 pi = __ldg(s.pf + i);
    const Grid &g = s.grid[__float_as_uint(pi.w) >> 8];
    const uint32_t cc = s.cellc[i];
    const int c0 = cell_coord(cc, 0), c1 = cell_coord(cc, 1), c2 = cell_coord(cc, 2);
    const int n1 = min(s.nnbr1[i], s.nmax1);
    int count = 0;
    auto flush = [&](int grp, int fill) {
      if (grp >= ngroups) return;
      const int h = (grp & 1) * kGroup;
      const uint32_t pad = pad_entry(Nc);
      uint32_t w[kGroup];
#pragma unroll
      for (int q = 0; q < kGroup; ++q) w[q] = q < fill ? stage[h + q][tx] : pad;
      uint4 *o = reinterpret_cast<uint4 *>(s.nbr) + ((size_t)grp * Nc + i) * 2;
      // lists are written once per build and read by the next pass from
      // HBM: evict-first stores keep L2 for the records the builds gather
      __stcs(o, make_uint4(w[0], w[1], w[2], w[3]));
      __stcs(o + 1, make_uint4(w[4], w[5], w[6], w[7]));
    };
    const uint4 *row = reinterpret_cast<const uint4 *>(s.nbr1) + (size_t)i * 2;
    // r^2 (FP32) of two candidates at once with the packed FP32 instructions:
    // d = (p_j - p_i) + s h, the stencil shifts s 4^d from the entries' codes
    // (cell size pre-scaled by 4^-d)
    const float2 mpx = make_float2(-pi.x, -pi.x), mpy = make_float2(-pi.y, -pi.y),
                 mpz = make_float2(-pi.z, -pi.z);
    const float2 hx2 = make_float2(g.hf[0], g.hf[0]),
                 hy2 = make_float2(0.25f * g.hf[1], 0.25f * g.hf[1]),
                 hz2 = make_float2(0.0625f * g.hf[2], 0.0625f * g.hf[2]);
    auto r2pair = [&](uint32_t ea, uint32_t eb, const float4 &qa, const float4 &qb) {
      const float2 sx = __fadd2_rn(make_float2(__uint_as_float((ea & 3u) | 0x4B000000u),
                                               __uint_as_float((eb & 3u) | 0x4B000000u)),
                                   make_float2(-8388609.0f, -8388609.0f));
      const float2 sy = __fadd2_rn(make_float2(__uint_as_float((ea & 12u) | 0x4B000000u),
                                               __uint_as_float((eb & 12u) | 0x4B000000u)),
                                   make_float2(-8388612.0f, -8388612.0f));
      const float2 sz = __fadd2_rn(make_float2(__uint_as_float((ea & 48u) | 0x4B000000u),
                                               __uint_as_float((eb & 48u) | 0x4B000000u)),
                                   make_float2(-8388624.0f, -8388624.0f));
      const float2 dx = __ffma2_rn(sx, hx2, __fadd2_rn(make_float2(qa.x, qb.x), mpx));
      const float2 dy = __ffma2_rn(sy, hy2, __fadd2_rn(make_float2(qa.y, qb.y), mpy));
      const float2 dz = __ffma2_rn(sz, hz2, __fadd2_rn(make_float2(qa.z, qb.z), mpz));
      return __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    };
    // four candidates at a time (as k_build's blocks of four)
    auto block4 = [&](const uint32_t *e) {
      const int before = count;
      // whole groups: slots past n1 hold pad_entry, whose record (pf[N_cap])
      // lies 1e18 A away and fails the pre-filter outright
      float4 pj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) pj[u] = __ldg(s.pf + dbg_idx(s, nbr_j(e[u]), Nc + 1, i));
      const float2 r01 = r2pair(e[0], e[1], pj[0], pj[1]);
      const float2 r23 = r2pair(e[2], e[3], pj[2], pj[3]);
      const float r2v[4] = {r01.x, r01.y, r23.x, r23.y};
      bool band = false;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t code = e[u];
        const float r2f = r2v[u];
        // lexicographically positive stencil offset <=> 6-bit code > 21
        const bool ok = !HALF || half_keep(i, nbr_j(code), (code & 63u) > 21u);
        const bool acc = ok && r2f < lo_thr;
        band = band || (ok && !acc && !(r2f > hi_thr));
        stage[count & 15][tx] = code;  // kept only if accepted
        count += acc ? 1 : 0;
      }
      if (band) {
        count = before;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t code = e[u];
          const float r2f = r2v[u];
          const bool ok = !HALF || half_keep(i, nbr_j(code), (code & 63u) > 21u);
          bool acc = ok && r2f < lo_thr;
          if (ok && !acc && !(r2f > hi_thr)) acc = exact_pair(s, g, i, code, c0, c1, c2, rns2);
          stage[count & 15][tx] = code;
          count += acc ? 1 : 0;
        }
      }
      if ((before >> 3) != (count >> 3)) flush(before >> 3, kGroup);
    };
    // the next group's entries are loaded while this group runs (their HBM
    // latency overlaps the candidate gathers)
    uint4 na = make_uint4(0, 0, 0, 0), nb = na;
    if (n1 > 0) {
      ld_group(row, na, nb);
    }
    for (int k0 = 0; k0 < n1; k0 += kGroup) {
      const uint4 a = na, b = nb;
      row += Nc * 2;
      if (k0 + kGroup < n1) {
        ld_group(row, na, nb);
      }
      const uint32_t ea[4] = {a.x, a.y, a.z, a.w};
      const uint32_t eb[4] = {b.x, b.y, b.z, b.w};
      block4(ea);
      block4(eb);
    }
    if (count & 7) flush(count >> 3, count & 7);
    s.nnbr[i] = count;
    if (count > s.nmax) {
      atomicOr(&s.st->bits, kStOverflow);
      atomicMax(&s.st->max_nnbr, count);
      s.st->build_ovf = 1;
    }
  }
}

// A build that stepping triggered and whose list outgrew its capacity stops
// the stepping (st->abort): the lists are truncated, so no force pass may use
// them; the host regrows the workspace, carries the state over and resumes.
__global__ void k_finish(Sys s, int from_graph) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DevStatus *st = s.st;
  if (st->rebuild) {
    st->rebuild = 0;
    st->n_builds += 1;
    if (from_graph) st->n_graph_builds += 1;
    st->since_build = 0;
    if (st->step_build && st->build_ovf) st->abort = 1;
  }
}

// Replay of a filter build (checkpoint restore with two-level lists): the
// Verlet list is filtered from the outer list of the full build just
// replayed, at the positions now in x, as a stepping build would.
__global__ void k_replay_filter_head(Sys s) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DevStatus *st = s.st;
  st->rebuild = 1;
  st->full = 0;
  st->win_active = 0;
  st->win_cut = -INFINITY;
  st->step_build = 0;
  st->build_ovf = 0;
  st->outer_valid = 1;
}

// gather copy of the positions in x with the cells of the last build (the
// expression of the step epilogue)
template <class P>
__global__ void __launch_bounds__(kBlk) k_regather(Sys s, typename P::vec4 *out) {
  const int N = s.st->N;
  const size_t Nc = s.N_cap;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const uint32_t inf = s.info[i];
    const Grid &g = s.grid[inf >> 8];
    const uint32_t cc = s.cellc[i];
    out[i] = P::make(s.x[i] - cell_center(g, 0, cell_coord(cc, 0)),
                     s.x[Nc + i] - cell_center(g, 1, cell_coord(cc, 1)),
                     s.x[2 * Nc + i] - cell_center(g, 2, cell_coord(cc, 2)), inf);
  }
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_set_rebuild_flag(const Sys &s, cudaStream_t st) { k_set_flag<<<1, 32, 0, st>>>(s); }

// The chain is enqueued every step and usually has nothing to do: a grid of
// N/256 blocks that all exit at once still costs ~0.1 ms of block
// scheduling, so every kernel of the chain runs on a persistent grid (a few
// blocks per SM) with grid-stride loops; a skipped rebuild costs a few us.
int persistent_blocks(const void *fn, int threads, int smem) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess ||
      occ <= 0)
    occ = 1;
  return sms * occ;
}

void launch_rebuild_head(const Sys &s, int count_step, cudaGraphConditionalHandle h,
                         cudaStream_t st) {
  k_pre<<<1, 32, 0, st>>>(s, count_step, 1, h);
}

int rebuild_chain_kernels(const Sys &s) { return 11 + (s.win_on ? 4 : 0) + (s.outer_on ? 4 : 0); }

int launch_rebuild_body(const Sys &s, int target_pg, int precision, int from_graph,
                        cudaStream_t st) {
  static int g_atom = 0, g_build = 0, g_cells = 0, g_filter = 0;
  if (g_atom == 0) {
    g_atom = persistent_blocks((const void *)k_bin, kBlk, 0);
    g_build = persistent_blocks((const void *)k_build<false>, kBlk, 0);
    g_cells = persistent_blocks((const void *)k_cell_sort, kBlk, 0);
    g_filter = persistent_blocks((const void *)k_build_filter<false>, kBlk, 0);
  }
  const int gN = std::min(g_atom, nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk));
  const int gC = std::min(g_cells, nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk));
  const int gB = std::min(g_build, nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk));
  const int gF = std::min(g_filter, nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk));
  if (s.outer_on) {
    k_outer_disp<<<gN, kBlk, 0, st>>>(s);
    k_outer_decide<<<1, 32, 0, st>>>(s);
  }
  if (s.win_on) {
    k_win_stats<<<gN, kBlk, 0, st>>>(s);
    k_win_plan<<<1, kBlk, 0, st>>>(s);
    k_win_insert<<<gN, kBlk, 0, st>>>(s);
  }
  k_bin<<<gN, kBlk, 0, st>>>(s);
  k_scan_reduce<<<s.n_scan_blocks, kScanThreads, 0, st>>>(s);
  k_scan_top<<<1, kScanThreads, 0, st>>>(s);
  k_scan_apply<<<s.n_scan_blocks, kScanThreads, 0, st>>>(s);
  k_scatter<<<gN, kBlk, 0, st>>>(s);
  k_cell_sort<<<gC, kBlk, 0, st>>>(s);
  if (precision == 0)
    k_permute<Fp64><<<gN, kBlk, 0, st>>>(s, (dvec4 *)s.pg[target_pg]);
  else
    k_permute<Mixed><<<gN, kBlk, 0, st>>>(s, (float4 *)s.pg[target_pg]);
  k_copyback<<<gN, kBlk, 0, st>>>(s);
  if (s.win_on) k_win_trim<<<1, 32, 0, st>>>(s);
  if (!s.outer_on) {
    const ListOut lo{s.nbr, s.nnbr, s.nmax, s.rns2, s.filt_lo, s.filt_hi, &s.st->max_nnbr};
    if (s.half == 1)
      k_build<true><<<gB, kBlk, 0, st>>>(s, lo);
    else
      k_build<false><<<gB, kBlk, 0, st>>>(s, lo);
  } else {
    const ListOut lo{s.nbr1, s.nnbr1, s.nmax1, s.rns2_1, s.filt1_lo, s.filt1_hi, &s.st->max_nnbr1};
    k_build<false><<<gB, kBlk, 0, st>>>(s, lo);
    k_outer_refresh<<<gN, kBlk, 0, st>>>(s);
    if (s.half == 1)
      k_build_filter<true><<<gF, kBlk, 0, st>>>(s);
    else
      k_build_filter<false><<<gF, kBlk, 0, st>>>(s);
  }
  k_finish<<<1, 32, 0, st>>>(s, from_graph);
  return rebuild_chain_kernels(s) - 1;
}

void launch_rebuild(const Sys &s, int target_pg, int precision, int count_step, cudaStream_t st) {
  k_pre<<<1, 32, 0, st>>>(s, count_step, 0, 0);
  launch_rebuild_body(s, target_pg, precision, 0, st);
}

void launch_replay_filter(const Sys &s, int target_pg, int precision, cudaStream_t st) {
  k_replay_filter_head<<<1, 32, 0, st>>>(s);
  launch_rebuild_body(s, target_pg, precision, 0, st);
}

void launch_regather(const Sys &s, int target_pg, int precision, cudaStream_t st) {
  const int g = std::min(1024, nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk));
  if (precision == 0)
    k_regather<Fp64><<<g, kBlk, 0, st>>>(s, (dvec4 *)s.pg[target_pg]);
  else
    k_regather<Mixed><<<g, kBlk, 0, st>>>(s, (float4 *)s.pg[target_pg]);
}

int scan_blocks_for(int n_buckets) { return (n_buckets + kScanTile - 1) / kScanTile; }

namespace {
__global__ void k_set_piston(Sys s, const uint8_t *flags, int64_t n_flags) {
  const int N = s.st->N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int o = s.id[i];
    const uint32_t pbit = (flags && o < n_flags && flags[o]) ? kInfoPiston : 0u;
    s.info[i] = (s.info[i] & ~kInfoPiston) | pbit;
    if (o < s.N_cap) s.info0[o] = (s.info0[o] & ~kInfoPiston) | pbit;
  }
}
}  // namespace

void launch_set_piston(const Sys &s, const uint8_t *flags, int64_t n_flags, cudaStream_t st) {
  const int g = std::min(1024, nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk));
  k_set_piston<<<g, kBlk, 0, st>>>(s, flags, n_flags);
}

}  // namespace mdk
