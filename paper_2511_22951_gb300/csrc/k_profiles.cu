// k_profiles.cu -- per-bin statistics of the paper's Appendix ("Analysis of
// MD simulation results") on the GPU.
//
// For bins of width w along one axis: N_l atoms, mass M_l, centre-of-mass
// velocity u_l, temperature per degree of freedom T^a = sum m (v^a - u^a)^2 /
// (k_B N_l), potential energy sum U_i, and pressure tensor
// P^{ab} = [sum m (v^a - u^a)(v^b - u^b) + sum W_i^{ab}] / V_l with the
// per-atom virial W_i = 1/2 sum_j r_ij (x) f_ij (the Appendix's virial sum,
// read with the pair force).  Two passes over the atoms: sums that need only
// the atom (count, mass, momentum, U, W), then the peculiar kinetic tensor
// about the bin's COM velocity.  Bin sums use FP64 atomics (the order of the
// additions is not fixed; results agree with a sequential sum to ~1e-15).
#include <math.h>

#include "mdk_internal.cuh"

namespace mdk {
namespace {

constexpr int kBlk = 256;
constexpr double kBoltzmann = 8.617333262e-5;  // eV/K
// accumulator slots per bin
constexpr int kN = 0, kM = 1, kP = 2, kU = 5, kW = 6, kT = 12, kUl = 18;

struct ProfArgs {
  int axis, nbins;
  double origin, w, volume;
  double *acc;  // nbins * kProfWidth
  double *out;  // nbins * kProfOut
};

__device__ __forceinline__ int bin_of(const Sys &s, const ProfArgs &p, int i) {
  const double u = (s.x[(size_t)p.axis * s.N_cap + i] - p.origin) / p.w;
  const double l = floor(u);
  return (l >= 0.0 && l < (double)p.nbins) ? (int)l : -1;
}

__global__ void k_prof_zero(ProfArgs p) {
  const int n = p.nbins * kProfWidth;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
    p.acc[q] = 0.0;
}

__global__ void __launch_bounds__(kBlk) k_prof_a(Sys s, ProfArgs p) {
  const int N = s.st->N;
  const size_t Nc = s.N_cap;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int l = bin_of(s, p, i);
    if (l < 0) continue;
    const double m = s.mass[s.info[i] & 15u];
    double *a = p.acc + (size_t)l * kProfWidth;
    atomicAdd(a + kN, 1.0);
    atomicAdd(a + kM, m);
    for (int d = 0; d < 3; ++d) atomicAdd(a + kP + d, m * s.v[d * Nc + i]);
    atomicAdd(a + kU, s.ea[i]);
    for (int c = 0; c < 6; ++c) atomicAdd(a + kW + c, s.wa[c * Nc + i]);
  }
}

__global__ void k_prof_com(ProfArgs p) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < p.nbins; l += gridDim.x * blockDim.x) {
    double *a = p.acc + (size_t)l * kProfWidth;
    for (int d = 0; d < 3; ++d) a[kUl + d] = a[kM] > 0.0 ? a[kP + d] / a[kM] : 0.0;
  }
}

__global__ void __launch_bounds__(kBlk) k_prof_b(Sys s, ProfArgs p) {
  const int N = s.st->N;
  const size_t Nc = s.N_cap;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int l = bin_of(s, p, i);
    if (l < 0) continue;
    double *a = p.acc + (size_t)l * kProfWidth;
    const double mk = 2.0 * s.ke_m[s.info[i] & 15u];  // m / (eV per u A^2/fs^2)
    const double dx = s.v[i] - a[kUl], dy = s.v[Nc + i] - a[kUl + 1],
                 dz = s.v[2 * Nc + i] - a[kUl + 2];
    atomicAdd(a + kT + 0, mk * dx * dx);
    atomicAdd(a + kT + 1, mk * dy * dy);
    atomicAdd(a + kT + 2, mk * dz * dz);
    atomicAdd(a + kT + 3, mk * dx * dy);
    atomicAdd(a + kT + 4, mk * dx * dz);
    atomicAdd(a + kT + 5, mk * dy * dz);
  }
}

// out per bin: N, M, u[3], T[3], E_pot, P[6] (xx yy zz xy xz yz), E_kin, V
__global__ void k_prof_fin(ProfArgs p) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < p.nbins; l += gridDim.x * blockDim.x) {
    const double *a = p.acc + (size_t)l * kProfWidth;
    double *o = p.out + (size_t)l * kProfOut;
    const double n = a[kN];
    o[0] = n;
    o[1] = a[kM];
    for (int d = 0; d < 3; ++d) o[2 + d] = a[kUl + d];
    for (int d = 0; d < 3; ++d) o[5 + d] = n > 0.0 ? a[kT + d] / (kBoltzmann * n) : 0.0;
    o[8] = a[kU];
    for (int c = 0; c < 6; ++c) o[9 + c] = (a[kT + c] + a[kW + c]) / p.volume;
    o[15] = 0.5 * (a[kT] + a[kT + 1] + a[kT + 2]);
    o[16] = p.volume;
  }
}

}  // namespace

void launch_profiles(const Sys &s, int axis, double origin, double bin_w, int nbins,
                     double cross_area, double *acc, cudaStream_t st) {
  ProfArgs p;
  p.axis = axis;
  p.nbins = nbins;
  p.origin = origin;
  p.w = bin_w;
  p.volume = bin_w * cross_area;
  p.acc = acc;
  p.out = acc + (size_t)nbins * kProfWidth;
  const int gb = (nbins + kBlk - 1) / kBlk;
  const int ga = (int)((s.N_cap + kBlk - 1) / kBlk) > 0 ? (int)((s.N_cap + kBlk - 1) / kBlk) : 1;
  k_prof_zero<<<(nbins * kProfWidth + kBlk - 1) / kBlk, kBlk, 0, st>>>(p);
  k_prof_a<<<ga, kBlk, 0, st>>>(s, p);
  k_prof_com<<<gb, kBlk, 0, st>>>(p);
  k_prof_b<<<ga, kBlk, 0, st>>>(s, p);
  k_prof_fin<<<gb, kBlk, 0, st>>>(p);
}

}  // namespace mdk
