// mdk_noalloc.cu -- mdk_lj_compute_noalloc: LJ energy and forces with no
// device allocation and no workspace (declared in include/mdk.h).
//
// Some callers cannot allocate device memory: their device memory belongs to
// another allocator (a framework's caching pool, an arena reserved at
// start-up), or their host loop cannot afford an allocation and the device
// synchronisation that freeing implies.  For them this variant of the force
// kernel keeps its scratch -- cell histogram, cell starts, atoms sorted by
// cell, wrapped positions and per-atom energies -- in one fixed-size
// file-scope __device__ array instead of a caller-supplied workspace, and walks
// the 27-cell stencil directly (no Verlet list, pairs with r < rc).
//
// The array lives in every GPU that loads the library until the process
// exits.  Host code cannot use its name as a device address (there it is a
// host-side shadow), so the first call on each device looks its address up
// with cudaGetSymbolAddress while that device is current, and passes the
// pointer to the kernels.  Every call shares the array: each call zeroes the
// histogram it accumulates into, and calls whose work overlaps on a GPU race.
//
// An atom with a non-finite coordinate goes to a bucket past the real cells:
// no pair includes it, and its force row and the energy come out NaN (the
// call does not synchronise, so the results are its only status channel).
#include <math.h>

#include <mutex>

#include "mdk.h"
#include "mdk_internal.cuh"

namespace mdk {
namespace {

constexpr int kMaxAtoms = MDK_NOALLOC_MAX_ATOMS;
constexpr int kMaxCells = MDK_NOALLOC_MAX_CELLS;
constexpr int kMaxDevices = 64;
constexpr int kBlk = 256;

// scratch layout (bytes), every part 256-byte aligned; the cell arrays hold
// n_cells + 1 buckets (the last one for atoms with a non-finite coordinate)
constexpr size_t kBuckets = (size_t)kMaxCells + 64;
constexpr size_t kOffCount = 0;
constexpr size_t kOffStart = kOffCount + 4 * kBuckets;
constexpr size_t kOffFill = kOffStart + 4 * kBuckets;
constexpr size_t kOffCellOf = kOffFill + 4 * kBuckets;
constexpr size_t kOffOrder = kOffCellOf + 4 * (size_t)kMaxAtoms;
constexpr size_t kOffSorted = kOffOrder + 4 * (size_t)kMaxAtoms;
constexpr size_t kOffE = kOffSorted + 4 * (size_t)kMaxAtoms;
constexpr size_t kOffX = kOffE + 8 * (size_t)kMaxAtoms;
constexpr size_t kScratchBytes = kOffX + 24 * (size_t)kMaxAtoms;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct NaScratch {
  int *count, *start, *fill, *cell_of, *order, *sorted;
  double *e, *xw;  // xw: wrapped positions [3][kMaxAtoms]
};

struct NaParams {
  int N;
  int nc[3], per[3];
  int n_cells;
  double lo[3], hi[3], L[3], inv_h[3];
  double eps4, eps24, sig2, rc2, u_shift, du_rc, rc;
  int shift_mode;
};

__host__ __device__ inline NaScratch carve(unsigned char *base) {
  NaScratch s;
  s.count = reinterpret_cast<int *>(base + kOffCount);
  s.start = reinterpret_cast<int *>(base + kOffStart);
  s.fill = reinterpret_cast<int *>(base + kOffFill);
  s.cell_of = reinterpret_cast<int *>(base + kOffCellOf);
  s.order = reinterpret_cast<int *>(base + kOffOrder);
  s.sorted = reinterpret_cast<int *>(base + kOffSorted);
  s.e = reinterpret_cast<double *>(base + kOffE);
  s.xw = reinterpret_cast<double *>(base + kOffX);
  return s;
}

__global__ void k_na_zero(NaParams p, unsigned char *base) {
  NaScratch s = carve(base);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= p.n_cells; c += gridDim.x * blockDim.x)
    s.count[c] = 0;
}

// wrap (periodic dimensions, by whole box lengths as in the list build),
// cell id, histogram; a non-finite coordinate sends the atom to bucket n_cells
__global__ void k_na_bin(NaParams p, const double *x, unsigned char *base) {
  NaScratch s = carve(base);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.N) return;
  const double x0 = x[3 * (size_t)i], x1 = x[3 * (size_t)i + 1], x2 = x[3 * (size_t)i + 2];
  if (!(isfinite(x0) && isfinite(x1) && isfinite(x2))) {
    for (int d = 0; d < 3; ++d) s.xw[(size_t)d * kMaxAtoms + i] = NAN;
    s.cell_of[i] = p.n_cells;
    atomicAdd(&s.count[p.n_cells], 1);
    return;
  }
  int c[3];
  for (int d = 0; d < 3; ++d) {
    double v = d == 0 ? x0 : (d == 1 ? x1 : x2);
    if (p.per[d] && (v >= p.hi[d] || v < p.lo[d])) {
      if (fabs(v - p.lo[d]) > 4.0 * p.L[d]) v = v - p.L[d] * floor((v - p.lo[d]) / p.L[d]);
      for (int it = 0; it < 8 && v >= p.hi[d]; ++it) v = v - p.L[d];
      for (int it = 0; it < 8 && v < p.lo[d]; ++it) v = v + p.L[d];
      if (v >= p.hi[d] || v < p.lo[d]) v = p.lo[d];
    }
    s.xw[(size_t)d * kMaxAtoms + i] = v;
    int ck = (int)floor((v - p.lo[d]) * p.inv_h[d]);
    c[d] = min(max(ck, 0), p.nc[d] - 1);
  }
  const int cell = c[0] + p.nc[0] * (c[1] + p.nc[1] * c[2]);
  s.cell_of[i] = cell;
  atomicAdd(&s.count[cell], 1);
}

// exclusive scan of the n_cells + 1 bucket counts, one block
// (n_cells + 1 <= 1024 * kPer)
__global__ void __launch_bounds__(1024) k_na_scan(NaParams p, unsigned char *base) {
  NaScratch s = carve(base);
  constexpr int kPer = kMaxCells / 1024 + 1;
  const int nb = p.n_cells + 1;
  __shared__ int warp_tot[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int loc[kPer];
  int sum = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int c = t * kPer + q;
    loc[q] = c < nb ? s.count[c] : 0;
    sum += loc[q];
  }
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int v0 = warp_tot[lane];
    int vi = v0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += v;
    }
    warp_tot[lane] = vi - v0;
  }
  __syncthreads();
  int pre = warp_tot[w] + incl - sum;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int c = t * kPer + q;
    if (c < nb) {
      s.start[c] = pre;
      s.fill[c] = pre;
    }
    pre += loc[q];
  }
  if (t == 1023) s.start[nb] = pre;
}

__global__ void k_na_scatter(NaParams p, unsigned char *base) {
  NaScratch s = carve(base);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.N) return;
  s.order[atomicAdd(&s.fill[s.cell_of[i]], 1)] = i;
}

// atoms of a cell in increasing index order, so results do not depend on
// the order of the atomic slots: the atom in slot k takes rank = number of
// atoms of its bucket with a smaller index (one thread per atom, the
// comparisons of a bucket run in parallel)
__global__ void k_na_rank(NaParams p, unsigned char *base) {
  NaScratch s = carve(base);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p.N) return;
  const int v = s.order[k];
  const int b = s.cell_of[v];
  const int a = s.start[b], e = s.start[b + 1];
  int rank = 0;
  for (int q = a; q < e; ++q) rank += s.order[q] < v ? 1 : 0;
  s.sorted[a + rank] = v;
}

// the force kernel's variant: 27-cell stencil, each stencil position one
// periodic image, d = (x_j - x_i) + n L, pairs with r^2 < rc^2, FP64
__global__ void __launch_bounds__(kBlk) k_na_force(NaParams p, unsigned char *base, double *F) {
  NaScratch s = carve(base);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.N) return;
  const double *X = s.xw, *Y = s.xw + kMaxAtoms, *Z = s.xw + 2 * kMaxAtoms;
  const double xi = X[i], yi = Y[i], zi = Z[i];
  const int cell = s.cell_of[i];
  if (cell == p.n_cells) {  // non-finite input: in no pair, NaN results
    F[3 * (size_t)i + 0] = NAN;
    F[3 * (size_t)i + 1] = NAN;
    F[3 * (size_t)i + 2] = NAN;
    s.e[i] = NAN;
    return;
  }
  const int c0 = cell % p.nc[0], c1 = (cell / p.nc[0]) % p.nc[1], c2 = cell / (p.nc[0] * p.nc[1]);
  double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0;
  for (int sz = -1; sz <= 1; ++sz) {
    int cz = c2 + sz, nz = 0;
    if (p.per[2]) {
      if (cz < 0) { cz += p.nc[2]; nz = -1; } else if (cz >= p.nc[2]) { cz -= p.nc[2]; nz = 1; }
    } else if (cz < 0 || cz >= p.nc[2]) {
      continue;
    }
    for (int sy = -1; sy <= 1; ++sy) {
      int cy = c1 + sy, ny = 0;
      if (p.per[1]) {
        if (cy < 0) { cy += p.nc[1]; ny = -1; } else if (cy >= p.nc[1]) { cy -= p.nc[1]; ny = 1; }
      } else if (cy < 0 || cy >= p.nc[1]) {
        continue;
      }
      for (int sx = -1; sx <= 1; ++sx) {
        int cx = c0 + sx, nx = 0;
        if (p.per[0]) {
          if (cx < 0) { cx += p.nc[0]; nx = -1; } else if (cx >= p.nc[0]) { cx -= p.nc[0]; nx = 1; }
        } else if (cx < 0 || cx >= p.nc[0]) {
          continue;
        }
        const int cj = cx + p.nc[0] * (cy + p.nc[1] * cz);
        const bool self_img = nx == 0 && ny == 0 && nz == 0;
        for (int q = s.start[cj]; q < s.start[cj + 1]; ++q) {
          const int j = s.sorted[q];
          if (j == i && self_img) continue;
          const double dx = (X[j] - xi) + (double)nx * p.L[0];
          const double dy = (Y[j] - yi) + (double)ny * p.L[1];
          const double dz = (Z[j] - zi) + (double)nz * p.L[2];
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (!(r2 < p.rc2)) continue;
          const double inv = 1.0 / r2;
          const double s2 = p.sig2 * inv, s6 = s2 * s2 * s2;
          double fr = -p.eps24 * (2.0 * s6 * s6 - s6) * inv;
          double v = p.eps4 * (s6 * s6 - s6) - p.u_shift;
          if (p.shift_mode == 2) {
            const double r = sqrt(r2);
            fr -= p.du_rc / r;
            v -= (r - p.rc) * p.du_rc;
          }
          fx += fr * dx;
          fy += fr * dy;
          fz += fr * dz;
          e += 0.5 * v;
        }
      }
    }
  }
  F[3 * (size_t)i + 0] = fx;
  F[3 * (size_t)i + 1] = fy;
  F[3 * (size_t)i + 2] = fz;
  s.e[i] = e;
}

// fixed-order energy sum (deterministic)
__global__ void __launch_bounds__(1024) k_na_energy(NaParams p, unsigned char *base, double *E) {
  NaScratch s = carve(base);
  __shared__ double sh[1024];
  double acc = 0.0;
  for (int i = threadIdx.x; i < p.N; i += 1024) acc += s.e[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) E[0] = sh[0];
}

std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

// device address of the scratch array on the current device (looked up once)
int scratch_address(unsigned char **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MDK_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return MDK_ERR_CUDA;
    g_addr[dev] = static_cast<unsigned char *>(ptr);
  }
  *out = g_addr[dev];
  return MDK_OK;
}

}  // namespace
}  // namespace mdk

using namespace mdk;

extern "C" int mdk_lj_compute_noalloc(const double *x, int64_t N, const double box_lo[3],
                                      const double box_hi[3], const int periodic[3], double eps,
                                      double sigma, double rc, int shift_mode, double *F,
                                      double *E, void *cuda_stream) {
  if (N < 0 || !box_lo || !box_hi || !periodic || !E || (N > 0 && (!x || !F)))
    return MDK_ERR_BAD_ARG;
  if (!(eps > 0.0) || !(sigma > 0.0) || !(rc > 0.0) || shift_mode < 0 || shift_mode > 2)
    return MDK_ERR_BAD_ARG;
  if (N > kMaxAtoms) return MDK_ERR_TOO_LARGE;
  NaParams p{};
  p.N = (int)N;
  long long cells = 1;
  for (int d = 0; d < 3; ++d) {
    const double L = box_hi[d] - box_lo[d];
    if (!(L > 0.0)) return MDK_ERR_BAD_ARG;
    if (periodic[d] && L < rc) return MDK_ERR_BOX_TOO_SMALL;
    int nc = (int)floor(L / (rc * (1.0 + 1e-10)));
    if (nc < 1) nc = 1;
    if (nc > kMaxCells) return MDK_ERR_TOO_LARGE;
    p.nc[d] = nc;
    p.per[d] = periodic[d] ? 1 : 0;
    p.lo[d] = box_lo[d];
    p.hi[d] = box_hi[d];
    p.L[d] = L;
    p.inv_h[d] = 1.0 / (L / nc);
    cells *= nc;
  }
  if (cells > kMaxCells) return MDK_ERR_TOO_LARGE;
  p.n_cells = (int)cells;
  const double sr = sigma / rc, s6 = sr * sr * sr * sr * sr * sr;
  p.eps4 = 4.0 * eps;
  p.eps24 = 24.0 * eps;
  p.sig2 = sigma * sigma;
  p.rc = rc;
  p.rc2 = rc * rc;
  p.u_shift = shift_mode >= 1 ? 4.0 * eps * (s6 * s6 - s6) : 0.0;
  p.du_rc = shift_mode == 2 ? -24.0 * eps * (2.0 * s6 * s6 - s6) / rc : 0.0;
  p.shift_mode = shift_mode;
  unsigned char *base = nullptr;
  int r = scratch_address(&base);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int gN = (int)((N + kBlk - 1) / kBlk);
  const int gC = (p.n_cells + 1 + kBlk - 1) / kBlk;
  k_na_zero<<<gC, kBlk, 0, st>>>(p, base);
  if (N > 0) k_na_bin<<<gN, kBlk, 0, st>>>(p, x, base);
  k_na_scan<<<1, 1024, 0, st>>>(p, base);
  if (N > 0) {
    k_na_scatter<<<gN, kBlk, 0, st>>>(p, base);
    k_na_rank<<<gN, kBlk, 0, st>>>(p, base);
    k_na_force<<<gN, kBlk, 0, st>>>(p, base, F);
  }
  k_na_energy<<<1, 1024, 0, st>>>(p, base, E);
  return cudaPeekAtLastError() == cudaSuccess ? MDK_OK : MDK_ERR_CUDA;
}
