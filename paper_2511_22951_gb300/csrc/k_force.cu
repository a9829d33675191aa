// k_force.cu -- per-atom kernels around the force loop (GB300, sm_103a): the
// first half-kick and drift of a step from stored forces, the deterministic
// per-replica sums of energies and virials, and the state / force / per-atom
// copies between the internal cell order and the caller's order.
#include "k_pair.cuh"

namespace mdk {

namespace {

using namespace pair;

constexpr int kBlk = 256;

// ---- first half-kick + drift from the stored forces ---------------------------------
// The same arithmetic as the second half of the fused step epilogue of the
// force pass in use (FP64 forces: the kick c F and drift_publish; FP32 forces
// of the mixed full-list kernels, a.f32: the FP32 kick increment of the FP32
// force the last pass stored exactly, and drift32), so a run split over
// several mdk_step calls is bitwise the run in one call.
template <class P>
__global__ void __launch_bounds__(kBlk) k_kick_drift(Sys s, StepArgs a) {
  const int N = run_n(s.st);
  const int i = blockIdx.x * kBlk + threadIdx.x;
  if (i >= N) return;
  const size_t Nc = s.N_cap;
  const uint32_t inf = s.info[i];
  const int type = inf & 15u;
  double vx = s.v[i], vy = s.v[Nc + i], vz = s.v[2 * Nc + i];
  const bool mixed = sizeof(typename G<P>::R) == 4 && a.f32;
  if (inf & kInfoPiston) {
    vx = s.u_p;
    vy = 0.0;
    vz = 0.0;
  } else if (mixed) {
    vx += kick32(s, a, type, (float)s.f[i]);
    vy += kick32(s, a, type, (float)s.f[Nc + i]);
    vz += kick32(s, a, type, (float)s.f[2 * Nc + i]);
  } else {
    const double c = 0.5 * a.dt * s.acc_over_m[type];
    vx += c * s.f[i];
    vy += c * s.f[Nc + i];
    vz += c * s.f[2 * Nc + i];
  }
  if (mixed)
    drift32(s, a, i, inf, vx, vy, vz);
  else
    drift_publish<P>(s, a, i, inf, vx, vy, vz);
}

// ---- deterministic per-replica sums (fixed order, no atomics) -----------------------
// Two passes: every block sums one chunk of kRedChunk atoms of one replica
// (a fixed partition, so the result does not depend on the launch), then one
// block per replica sums its chunks' partials in chunk order.  All SMs share
// the first pass, so the sums of an 8.4M-atom system take a fraction of a
// millisecond instead of one SM's tens of milliseconds.
constexpr int kRedThreads = 256;
constexpr int kRedTop = 1024;

// the block's sums of acc[0..7] (fixed shuffle tree, then warps in order);
// value c ends in thread c (c < 8)
template <int NT>
__device__ __forceinline__ double block_sum8(double (&acc)[8]) {
  __shared__ double sh[8][NT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    double v = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[c][wid] = v;
  }
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 8)
    for (int w = 0; w < NT / 32; ++w) t += sh[threadIdx.x][w];
  return t;
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_chunks(Sys s, int with_ke) {
  const int r = blockIdx.x;
  const Grid &g = s.grid[r];
  const int n = (s.n_rep == 1) ? s.st->N : g.n_atoms;
  const size_t Nc = s.N_cap;
  for (int k = blockIdx.y; k < s.red_chunks; k += gridDim.y) {
    const int q1 = min(n, (k + 1) * kRedChunk);
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.0;
    for (int q = k * kRedChunk + threadIdx.x; q < q1; q += kRedThreads) {
      const int i = g.atom_off + q;
      acc[0] += with_ke ? s.ka[i] : 0.0;
      acc[1] += s.ea[i];
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[2 + c] += s.wa[c * Nc + i];
    }
    const double t = block_sum8<kRedThreads>(acc);
    if (threadIdx.x < 8) s.red_part[((size_t)r * s.red_chunks + k) * 8 + threadIdx.x] = t;
    __syncthreads();  // block_sum8's shared slots are reused by the next chunk
  }
}

__global__ void __launch_bounds__(kRedTop) k_reduce_top(Sys s) {
  const int r = blockIdx.x;
  double acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0.0;
  const double *p = s.red_part + (size_t)r * s.red_chunks * 8;
  for (int k = threadIdx.x; k < s.red_chunks; k += kRedTop) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] += p[(size_t)k * 8 + c];
  }
  const double t = block_sum8<kRedTop>(acc);
  if (threadIdx.x < 8) s.red[r * 9 + threadIdx.x] = t;
  if (threadIdx.x == 0) s.red[r * 9 + 8] = (double)((s.n_rep == 1) ? s.st->N : s.grid[r].n_atoms);
}

// ---- state in / out in the caller's order -------------------------------------------
template <class P>
__global__ void __launch_bounds__(kBlk) k_load_state(Sys s, const double *x, const double *v,
                                                     int target_pg) {
  const int N = s.st->N;
  const int i = blockIdx.x * kBlk + threadIdx.x;
  if (i >= N) return;
  const size_t Nc = s.N_cap;
  for (int d = 0; d < 3; ++d) {
    s.x[d * Nc + i] = x[3 * (size_t)i + d];
    s.v[d * Nc + i] = v ? v[3 * (size_t)i + d] : 0.0;
    s.f[d * Nc + i] = 0.0;
  }
  s.id[i] = i;
  s.info[i] = s.info0[i];
}

__global__ void __launch_bounds__(kBlk) k_store_state(Sys s, double *x, double *v) {
  const int N = s.st->N;
  const int i = blockIdx.x * kBlk + threadIdx.x;
  if (i >= N) return;
  const size_t Nc = s.N_cap;
  const size_t o = (size_t)s.id[i];
  for (int d = 0; d < 3; ++d) {
    if (x) x[3 * o + d] = s.x[d * Nc + i];
    if (v) v[3 * o + d] = s.v[d * Nc + i];
  }
}

__global__ void __launch_bounds__(kBlk) k_store_forces(Sys s, double *f) {
  const int N = s.st->N;
  const int i = blockIdx.x * kBlk + threadIdx.x;
  if (i >= N) return;
  const size_t Nc = s.N_cap;
  const size_t o = (size_t)s.id[i];
  for (int d = 0; d < 3; ++d) f[3 * o + d] = s.f[d * Nc + i];
}

__global__ void __launch_bounds__(kBlk) k_store_per_atom(Sys s, double *ua, double *wa) {
  const int N = s.st->N;
  const int i = blockIdx.x * kBlk + threadIdx.x;
  if (i >= N) return;
  const size_t Nc = s.N_cap;
  const size_t o = (size_t)s.id[i];
  if (ua) ua[o] = s.ea[i];
  if (wa)
    for (int c = 0; c < 6; ++c) wa[6 * o + c] = s.wa[c * Nc + i];
}



inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace





void launch_kick_drift(const Sys &s, int precision, StepArgs a, cudaStream_t st) {
  const int g = nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk);
  if (precision == 0)
    k_kick_drift<Fp64><<<g, kBlk, 0, st>>>(s, a);
  else
    k_kick_drift<Mixed><<<g, kBlk, 0, st>>>(s, a);
}

int launch_reduce(const Sys &s, int with_ke, cudaStream_t st) {
  k_reduce_chunks<<<dim3(s.n_rep, std::min(s.red_chunks, 65535)), kRedThreads, 0, st>>>(s,
                                                                                      with_ke);
  k_reduce_top<<<s.n_rep, kRedTop, 0, st>>>(s);
  return 2;
}


namespace {
template <class P>
__global__ void k_init_far(Sys s) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const size_t Nc = s.N_cap;
  for (int b = 0; b < 2; ++b)
    reinterpret_cast<typename P::vec4 *>(s.pg[b])[Nc] = P::make(1e18, 1e18, 1e18, 0u);
  s.pf[Nc] = make_float4(1e18f, 1e18f, 1e18f, 0.0f);
}
}  // namespace

void launch_init_far(const Sys &s, int precision, cudaStream_t st) {
  if (precision == 0)
    k_init_far<Fp64><<<1, 32, 0, st>>>(s);
  else
    k_init_far<Mixed><<<1, 32, 0, st>>>(s);
}

void launch_load_state(const Sys &s, const double *x, const double *v, int precision,
                       int target_pg, cudaStream_t st) {
  const int g = nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk);
  if (precision == 0)
    k_load_state<Fp64><<<g, kBlk, 0, st>>>(s, x, v, target_pg);
  else
    k_load_state<Mixed><<<g, kBlk, 0, st>>>(s, x, v, target_pg);
}

void launch_store_state(const Sys &s, double *x, double *v, cudaStream_t st) {
  k_store_state<<<nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk), kBlk, 0, st>>>(s, x, v);
}

void launch_store_forces(const Sys &s, double *f, cudaStream_t st) {
  k_store_forces<<<nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk), kBlk, 0, st>>>(s, f);
}

void launch_store_per_atom(const Sys &s, double *ua, double *wa, cudaStream_t st) {
  k_store_per_atom<<<nblk(s.N_cap > 0 ? s.N_cap : 1, kBlk), kBlk, 0, st>>>(s, ua, wa);
}



}  // namespace mdk
