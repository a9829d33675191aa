// mdk_internal.cuh -- device-side data layout shared by the CUDA sources of
// libmdk.so (GB300, sm_103a).  Nothing here is visible through the C ABI.
//
// Layout in HBM (all inside the caller's workspace, atoms in cell order):
//   x, v, f, xref : FP64 SoA, component c of atom i at [c * N_cap + i]
//   pf            : float4 per atom, position relative to its cell centre
//                   with the info word in .w; written at each list build,
//                   used by the build's FP32 pre-filter (NaN for far atoms)
//   pg[2]         : per-step gather copy, double-buffered; float4 (mixed) or
//                   32-byte FP64 vector of x - centre(cell), info in .w
//   info          : type (bits 0-3) | piston (bit 4) | far (bit 5) |
//                   replica (bits 8-31)
//   cell buckets  : n_cells real cells + 1 bucket for atoms a moving window
//                   deletes (the counting sort moves them past the kept atoms)
//   nbr           : Verlet lists in groups of 8 entries per atom (ell_index),
//                   packed (s_x+1) | (s_y+1) << 2 | (s_z+1) << 4 | j << 6,
//                   s = stencil offset of j's cell; each 2-bit code sits in
//                   place, so one AND with a constant exponent turns it
//                   into a float (s_scaled)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mdk {

// 1 eV/(Angstrom u) in Angstrom/fs^2 (elementary charge / atomic mass unit,
// 1e-10 m, 1e-30 s^2).
constexpr double kAcc = 9.648533212331e-3;
// fixed-point unit of the mixed path's half-list accumulators: 2^-40
// (eV/A, eV); an atom's total must stay below 2^23 in magnitude
constexpr double kHalfScale = 1099511627776.0;

constexpr int kMaxTypes = 16;
constexpr int kMaxLang = 8;  // Langevin regions
constexpr uint32_t kInfoPiston = 1u << 4;
constexpr uint32_t kInfoFar = 1u << 5;

// device status bits
enum : unsigned {
  kStOverflow = 1u,
  kStNonfinite = 2u,
  kStRhoRange = 4u,
  kStAtomLost = 8u,
  kStTimeout = 16u,
  kStCapacity = 32u,  // a window append did not fit the capacity
  kStBounds = 64u,    // debug builds: an index outside its array was caught
};

struct DevStatus {
  int N;                 // atoms present
  int abort;             // != 0: a list build during stepping overflowed; every
                         // later kernel of the stepping chain does nothing, so
                         // the state stays that of the moment of the build
                         // (positions drifted, velocities at the half step)
  int rebuild;           // != 0: rebuild the lists before the next force pass
  unsigned bits;         // kSt* raised since the host last cleared them
  int max_nnbr;          // longest list seen at a build
  long long n_builds;
  long long n_graph_builds;  // builds run inside a captured step's conditional node
  long long n_steps;
  int since_build;       // steps since the last build
  int next_id;           // id of the next atom a moving window appends
  // moving window (order-preserving integer keys of doubles, for atomics)
  long long key_xmax, key_xmin;
  double win_cut;        // atoms with x below are deleted at this build
  double win_x0;         // x offset of the first appended slab copy
  int win_insert;        // atoms appended at this build
  int win_n_old;         // atom count before the append
  int win_id0;           // id of the first appended atom
  int win_active;        // the window acts at this build (builds during steps)
  long long n_inserted, n_deleted;
  // outer list (two-level lists; Sys.outer_on)
  int full;              // this build re-bins and rebuilds the outer list (else:
                         // the Verlet list is filtered from the outer list)
  int outer_valid;       // the outer list holds the pairs of the last full build
  int max_nnbr1;         // longest outer list seen at a build
  long long dmax_key;    // max |x - x_full|^2 at this build (bits of a double >= 0)
  double d_acc;          // the largest displacement since the last full build
  long long n_full_builds;
  int step_build;        // this build was triggered by stepping (k_pre, count_step)
  int build_ovf;         // a list of this build outgrew its capacity
};

// atoms a force or integration kernel works on: none once stepping aborted
__device__ __forceinline__ int run_n(const DevStatus *st) {
  return st->abort ? 0 : st->N;
}

// one replica's box and cell grid
struct Grid {
  double lo[3], hi[3], L[3], h[3], inv_h[3];
  double lo_c[3];  // lo + h/2: the centre of cell 0
  float hf[3];
  int nc[3];
  int per[3];
  int cell_off;   // first global cell id of this replica
  int atom_off;   // first atom of this replica (atoms stay grouped by replica)
  int n_atoms;
  // cell centres along each dimension, fma(c, h, lo_c) for c < nc (device
  // memory in the workspace, filled when the workspace is set)
  const double *ctr[3];
};

struct Sys {
  // sizes
  int N_cap;
  int nmax;
  int n_rep;
  int n_cells;           // real cells; bucket n_cells holds atoms a window deletes
  int n_scan_blocks;     // scan blocks over n_cells + 1 buckets
  // per-atom arrays
  double *x, *v, *f, *xref;
  double *tmp;              // 9 * N_cap doubles of sort scratch
  uint32_t *info, *cellc, *tmpu, *info0;
  int32_t *id, *tmpi;
  float4 *pf;
  void *pg[2];
  void *pgF;                // EAM: gather copy with F'(rho_j) in .w (density pass)
  int32_t *nnbr;
  uint32_t *nbr;
  int half;                 // list kind: 0 full, 1 half (each pair once), 2 none (LJ
                            // forces straight from the build's cells)
  // half-list accumulators, [10][N_cap] 8-byte words: F_x, F_y, F_z, U_i,
  // W_i[6]; int64 fixed point (kHalfScale) in the mixed path, double in the
  // FP64 path; zero between force passes
  long long *hacc;
  double *ea, *ka, *wa;     // per-atom U_i, K_i, W_i[6] (SoA)
  double *rho;
  void *fp;                 // F'(rho_i): double (FP64) or float (mixed)
  // cell sort scratch
  int32_t *cell_cnt, *cell_start, *cell_fill, *cell_of, *order, *scan_part;
  Grid *grid;
  DevStatus *st;
  double *red;              // reductions: per replica [K, U, W0..W5, N]
  double *red_part;         // per replica and chunk of kRedChunk atoms: the 8 partial sums
  int red_chunks;           // chunks per replica (ceil of its largest atom count / kRedChunk)
  // list parameters
  double rns2;              // (rc + skin)^2
  float filt_lo, filt_hi;   // FP32 pre-filter band around rns2
  // outer list (two-level lists, outer_on != 0): every pair within
  // rc + skin_outer of the last full build, full kind; the Verlet list above is
  // filtered from it while every atom has moved less than outer_budget =
  // (skin_outer - skin) / 2 since that build (positions then: xfull)
  int outer_on;
  double *xfull;
  int nmax1;
  int32_t *nnbr1;
  uint32_t *nbr1;
  double rns2_1;            // (rc + skin_outer)^2
  float filt1_lo, filt1_hi;
  double outer_budget;
  double half_skin2;        // (skin/2)^2
  int rebuild_every;
  // integration
  double mass[kMaxTypes];         // m of each type (u)
  double acc_over_m[kMaxTypes];   // kAcc / m for each type
  float acc_over_mf[kMaxTypes];   // the same in FP32 (mixed-path kicks)
  float half_skin2f;              // (skin/2)^2 in FP32 (mixed-path displacement test)
  double ke_m[kMaxTypes];         // m / (2 kAcc): K in eV from v^2
  double u_p;                     // piston speed
  // moving window along x (off when win_on == 0)
  int win_on;
  int n_slab;
  double L_behind, L_ahead, slab_lx, slab_gap, piston_depth;
  const double *slab;             // fresh slab: [n_slab][6] = x, y, z, vx, vy, vz
  uint32_t slab_info;             // info word of appended atoms
  // Langevin thermostat regions along x (n_lang = 0: off): x in
  // [lang_xlo, lang_xhi), target mean velocity, and per (region, type) the
  // friction factor g = -beta m / A and the noise amplitude
  // sigma = sqrt(24 beta m k_B T / (dt A)) of the current dt
  int n_lang;
  double lang_xlo[kMaxLang], lang_xhi[kMaxLang];
  double lang_u[kMaxLang][3];
  double lang_g[kMaxLang][kMaxTypes], lang_sig[kMaxLang][kMaxTypes];
  unsigned long long lang_seed;
  // per-replica thermostats (batched contexts; target mean velocity 0):
  // lang_rep[(replica * kMaxTypes + type) * 2 + {0, 1}] = (g, sigma)
  int lang_rep_on;
  const double *lang_rep;
  double win_xlo, win_xhi;        // the box along x
  double front_bin;               // width of the bins that locate the front
  double fixed_front;             // finite: the front's x, fixed (stationary window)
  int n_fbins;                    // bins over [win_xlo, win_xhi)
  long long *fbin;                // [2 n_fbins]: sum of q(v_x), atom count per bin
};

// Debug builds (compiled with MDK_DEBUG): an index about to be read or
// written is checked against its array's extent n; a bad one raises
// kStBounds in the status word and is replaced by `safe` (in range), so the
// kernel finishes without touching memory it does not own and the call
// reports MDK_ERR_BOUNDS.  Release builds compile the check away.
__device__ __forceinline__ uint32_t dbg_idx(const Sys &s, uint32_t j, uint32_t n,
                                            uint32_t safe = 0) {
#ifdef MDK_DEBUG
  if (j >= n) {
    atomicOr(&s.st->bits, kStBounds);
    return safe;
  }
#endif
  (void)s;
  (void)n;
  (void)safe;
  return j;
}

// order-preserving map of a double onto a signed 64-bit key (for atomicMax/Min)
__device__ __forceinline__ long long dkey(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : b ^ 0x7FFFFFFFFFFFFFFFLL;
}
__device__ __forceinline__ double dkey_inv(long long k) {
  return __longlong_as_double(k >= 0 ? k : k ^ 0x7FFFFFFFFFFFFFFFLL);
}

struct LJParams {
  double eps4, eps24, sig2, rc2, u_shift, du_rc, rc;
  float eps4f, eps24f, sig2f, rc2f, u_shiftf, du_rcf, rcf;
  int shift_mode;
};

// 32-byte FP64 gather-copy element (x, y, z, info bits in w)
struct alignas(32) dvec4 {
  double x, y, z, w;
};

struct EAMParams {
  int nr, nrho;
  double rc, rc2, inv_dr, dr, rho_max, inv_drho, drho;
  float rc2f, inv_drf;
  // FP64 knot tables (value, h * slope) per knot
  const double2 *phi64, *rho64, *F64;
  // FP32 tables of the mixed path, rounded from FP64 quantities so that no
  // FP32 subtraction of neighbouring knot values is needed:
  //   rho_i32[k] = (y_k, y_{k+1} - y_k, h m_k, h m_{k+1})   (pass 1, rho value)
  //   rho_d32[k] = (rho_{k+1} - rho_k, h m_k)                (adjoint, slopes)
  //   phi_v32[k] = y_k                                         (pass 2 energy)
  const float4 *rho_i32;
  const float2 *rho_d32;
  const float *phi_v32;
  // force pass: phi and rho interleaved per knot, so one pair of loads
  // serves both derivatives
  //   pr32[k] = (phi_{k+1} - phi_k, h m^phi_k, rho_{k+1} - rho_k, h m^rho_k)
  //   pr64[k] = (phi_k, h m^phi_k, rho_k, h m^rho_k)
  const float4 *pr32;
  const dvec4 *pr64;
  // the full-list mixed force pass: one 32-byte record per interval k, read
  // with one 256-bit load per pair:
  //   pr8[2k] = pr32[k],  pr8[2k + 1] = (phi_k, h m^phi_{k+1}, 0, h m^rho_{k+1})
  const float4 *pr8;
};

// Behler-Parrinello model: symmetry-function parameters by value (read as
// constant operands inside the triplet loops), network weights in the
// workspace (staged into shared memory per block).  The angular functions
// sit on a fixed grid of slots, slot = (p * kBpZ + z) * 2 + (lambda < 0):
// p the (eta, kind) group, z the zeta group; so every accumulator has a
// compile-time register index.  The device network input is [kBpRad radial
// values, kBpSlots slot values] (kBpIn); unused inputs have zero weights.
constexpr int kBpRad = 8;                  // radial functions (G1, G2, G3)
constexpr int kBpY = 8;                    // (eta, kind) groups of angular functions
constexpr int kBpZ = 4;                    // zeta groups
constexpr int kBpSlots = 2 * kBpY * kBpZ;  // angular slots
constexpr int kBpIn = kBpRad + kBpSlots;   // device network inputs
constexpr int kBpH = 32;                   // units per hidden layer
// words of the packed weight area (largest network)
constexpr int kBpWords = kBpIn * kBpH + kBpH + kBpH * kBpH + 2 * kBpH;
struct BPParams {
  int n_rad, nY, nZ, H1, H2, any4;
  unsigned long long slot_mask;            // slots holding a function
  double rc, b3;
  float rcf, b3f;
  int rad_kind[kBpRad];
  double rad_p0[kBpRad], rad_p1[kBpRad];
  float rad_p0f[kBpRad], rad_p1f[kBpRad];
  double y_eta[kBpY];
  float y_etaf[kBpY];
  int y_kind[kBpY];                        // 4: with the R_jk factors, 5: without
  int zset;                                // 1: the zetas are among {1, 2, 4, 16}, group z
                                           // holding zeta = 1, 2, 4, 16; 0: any integers
  int z_pow[kBpZ];                         // zeta - 1 (a non-negative integer)
  double z_zeta[kBpZ], z_coef[kBpZ];       // zeta, 2^(1 - zeta)
  float z_zetaf[kBpZ], z_coeff[kBpZ];
  // packed weights: W01 [kBpIn][H1], b1 [H1], W12 [H1][H2], b2 [H2], w23 [H2]
  const double *w64;
  const float *w32;
};

// writable view of the device tables filled by launch_eam_prepare
struct EAMTablesDev {
  double2 *phi64, *rho64, *F64;
  float4 *rho_i32;
  float2 *rho_d32;
  float *phi_v32;
  float4 *pr32;
  dvec4 *pr64;
  float4 *pr8;
};

// Centre of cell c along d, fma(c, h, lo_c), read from the grid's table
// (GB300's FP64 pipe is slow; a cached load replaces the conversion and the
// FMA).  Gather copies hold x - centre, so |p| <= h/2 right after a build
// (h/2 + skin/2 later); the build and every step read the same table, so the
// offsets of one list lifetime are consistent.
__device__ __forceinline__ double cell_center(const Grid &g, int d, int c) {
  return __ldg(g.ctr[d] + c);
}

// Verlet-list layout: entries in groups of 8 per atom; group g of atom i is
// the 32-byte sector starting at word (g * N_cap + i) * 8.  A thread reads 8
// entries with two 16-byte loads, a warp reads 1 KB contiguous, and the build
// writes whole sectors (no partial-sector read-modify-write in L2).
constexpr int kGroup = 8;
// atoms per block of the first pass of the per-replica sums
constexpr int kRedChunk = 8192;
__host__ __device__ __forceinline__ size_t ell_index(int k, int i, size_t Nc) {
  return ((size_t)(k >> 3) * Nc + (size_t)i) * kGroup + (size_t)(k & 7);
}

__host__ __device__ __forceinline__ uint32_t pack_nbr(int j, int sx, int sy, int sz) {
  return ((uint32_t)j << 6) | (uint32_t)(sx + 1) | ((uint32_t)(sy + 1) << 2) |
         ((uint32_t)(sz + 1) << 4);
}
__host__ __device__ __forceinline__ int nbr_j(uint32_t e) { return (int)(e >> 6); }

// The slots of a list's last group past its length hold this entry: atom
// index N_cap (a record of the gather copies kept 1e18 A away, past the last
// atom) with a zero stencil offset, so a walk can read whole groups without
// bounds tests; no pair with it is ever inside a cutoff.
__host__ __device__ __forceinline__ uint32_t pad_entry(size_t n_cap) {
  return 21u | ((uint32_t)n_cap << 6);
}

#ifdef __CUDACC__
// One ELL8 group (8 entries, a 32-byte sector) with one 256-bit streaming
// load (new with sm_100): a warp's 32 groups are 1 KB contiguous, read as
// whole sectors by one instruction instead of two 16-byte halves.
__device__ __forceinline__ void ld_group(const uint4 *p, uint4 &a, uint4 &b) {
  asm("ld.global.cs.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
      : "l"(p));
}
#endif
__host__ __device__ __forceinline__ int nbr_s(uint32_t e, int d) {
  return (int)((e >> (2 * d)) & 3u) - 1;
}
__host__ __device__ __forceinline__ uint32_t pack_cell(int cx, int cy, int cz) {
  return (uint32_t)cx | ((uint32_t)cy << 10) | ((uint32_t)cz << 20);
}
__host__ __device__ __forceinline__ int cell_coord(uint32_t c, int d) {
  return (int)((c >> (10 * d)) & 1023u);
}


// precision traits of the per-step gather copy
struct Fp64 {
  using real = double;
  using vec4 = dvec4;
  static __device__ __forceinline__ uint32_t info(const dvec4 &p) {
    return (uint32_t)__double_as_longlong(p.w);
  }
  static __device__ __forceinline__ dvec4 make(double a, double b, double c, uint32_t w) {
    dvec4 r;
    r.x = a;
    r.y = b;
    r.z = c;
    r.w = __longlong_as_double((long long)w);
    return r;
  }
};
struct Mixed {
  using real = float;
  using vec4 = float4;
  static __device__ __forceinline__ uint32_t info(const float4 &p) {
    return __float_as_uint(p.w);
  }
  static __device__ __forceinline__ float4 make(double a, double b, double c, uint32_t w) {
    return make_float4((float)a, (float)b, (float)c, __uint_as_float(w));
  }
};

// a per-atom sum: plain in FP64; Kahan-compensated in FP32
template <class R>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double get() const { return s; }
  __device__ __forceinline__ double getf() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
  // the compensated sum rounded to FP32 (the pair terms are FP32)
  __device__ __forceinline__ float getf() const { return s - c; }
};

// launch helpers implemented in the .cu files --------------------------------
enum Mode { kForceOnly = 0, kStep = 1, kFinal = 2 };

struct StepArgs {
  double dt;
  int cur;              // gather copy read this step (pg[cur]); pg[cur^1] written
  int energy;           // compute per-atom energies / virials this step
  float hdtf;           // dt / 2 in FP32 (mixed-path kicks)
  int f32;              // k_kick_drift: the force pass in use ends its steps with
                        // FP32 forces (the mixed full-list kernels), so the first
                        // kick takes the FP32 increment of the stored force
};

void launch_rebuild(const Sys &s, int target_pg, int precision, int count_step, cudaStream_t st);
// checkpoint restore: a filter build (two-level lists) at the positions in x,
// and the gather copy pg[target_pg] of x with the cells of the last build
void launch_replay_filter(const Sys &s, int target_pg, int precision, cudaStream_t st);
void launch_regather(const Sys &s, int target_pg, int precision, cudaStream_t st);
// The same chain in two parts for a captured step: the head decides whether
// to rebuild and sets the conditional node's value; the body (run by that
// node only when the value is 1) rebuilds.  Returns the kernels of the body.
void launch_rebuild_head(const Sys &s, int count_step, cudaGraphConditionalHandle h,
                         cudaStream_t st);
int launch_rebuild_body(const Sys &s, int target_pg, int precision, int from_graph,
                        cudaStream_t st);
int rebuild_chain_kernels(const Sys &s);
void launch_set_piston(const Sys &s, const uint8_t *flags, int64_t n_flags, cudaStream_t st);
int scan_blocks_for(int n_cells);
void launch_set_rebuild_flag(const Sys &s, cudaStream_t st);
// launch shape of the pair kernels, picked by the autotuner
struct LaunchCfg {
  int tpa = 1;      // threads per atom: 1, 2 or 4
  int block = 256;  // threads per block: 128, 256 or 512
  int half = 0;     // list kind: 1 = half lists with accumulating atomics (tpa 1),
                    // 2 = LJ from the cells, one warp per cell (no list)
};

void launch_lj(const Sys &s, const LJParams &p, int precision, Mode mode, StepArgs a,
               const LaunchCfg &cfg, cudaStream_t st);
// the per-atom pass that finishes a step from the accumulators in s.hacc
void launch_half_fin(const Sys &s, int precision, Mode mode, StepArgs a, cudaStream_t st);
// Behler-Parrinello forces into s.hacc (full lists), then launch_half_fin
void launch_bpnn(const Sys &s, const BPParams &p, int precision, Mode mode, StepArgs a,
                 cudaStream_t st);
size_t bpnn_smem_bytes(const BPParams &p, int precision, int nmax, int *warps);
int configure_bpnn_smem(size_t bytes, int precision);
// LJ from the build's cells, one warp per cell, neighbour cells tiled in
// shared memory (list kind 2)
void launch_lj_cells(const Sys &s, const LJParams &p, int precision, Mode mode, StepArgs a,
                     const LaunchCfg &cfg, cudaStream_t st);
// half lists: the pair pass with accumulating atomics, then the per-atom pass
void launch_lj_half(const Sys &s, const LJParams &p, int precision, Mode mode, StepArgs a,
                    const LaunchCfg &cfg, cudaStream_t st);
void launch_eam(const Sys &s, const EAMParams &p, int precision, Mode mode, StepArgs a,
                const LaunchCfg &cfg, cudaStream_t st);
void launch_kick_drift(const Sys &s, int precision, StepArgs a, cudaStream_t st);
// returns the number of kernels launched
int launch_reduce(const Sys &s, int with_ke, cudaStream_t st);
void launch_eam_prepare(const EAMParams &p, const double *phi, const double *rho,
                        const double *F, EAMTablesDev out, cudaStream_t st);
// the far records at index N_cap of both gather copies (see pad_entry)
void launch_init_far(const Sys &s, int precision, cudaStream_t st);
void launch_load_state(const Sys &s, const double *x_aos, const double *v_aos,
                       int precision, int target_pg, cudaStream_t st);
void launch_store_state(const Sys &s, double *x_aos, double *v_aos, cudaStream_t st);
void launch_store_forces(const Sys &s, double *f_aos, cudaStream_t st);
void launch_store_per_atom(const Sys &s, double *ua, double *wa, cudaStream_t st);
// Appendix profiles: kProfOut outputs per bin (see mdk_profiles), computed in
// an accumulator of kProfWidth doubles per bin
constexpr int kProfOut = 17;
constexpr int kProfWidth = 24;
void launch_profiles(const Sys &s, int axis, double origin, double bin_w, int nbins,
                     double cross_area, double *acc, cudaStream_t st);
int eam_smem_bytes(const EAMParams &p, int precision, int pass);
int configure_eam_smem(int bytes_pass1, int bytes_pass2, int precision);
int configure_eam_half_smem(int bytes_pass1, int bytes_pass2, int precision);
// half lists: density pass, embedding, force pass with accumulating atomics,
// then launch_half_fin
void launch_eam_half(const Sys &s, const EAMParams &p, int precision, Mode mode, StepArgs a,
                     const LaunchCfg &cfg, cudaStream_t st);
// pass 1 of the EAM force loop alone (rho_i and F'(rho_i) of the current positions)
void launch_eam_rho(const Sys &s, const EAMParams &p, int precision, StepArgs a,
                    const LaunchCfg &cfg, cudaStream_t st);

// EAM adjoint (k_adjoint.cu): gradient of sum_r gE_r E_r + sum_i gF_i . F_i with
// respect to the phi, rho and F knot values
struct AdjArgs {
  int cur;                           // gather copy of the current positions
  int f_in_smem;                     // F histogram privatised in shared memory
  const double *gE;                  // [n_rep] energy weights
  void *gint;                        // [N_cap] gF in internal order (gather-copy type)
  double *lam;                       // [N_cap] lambda_i = gE F'(rho_i) + c_i F''(rho_i)
  longlong2 *acc_phi, *acc_rho;      // per knot: (d/dy, d/dM), fixed point (units 1/S)
  double2 *acc_F;                    // per knot: (d/dy, d/dM), FP64
  long long *aux;                    // [0..3] bounds (bits of max |gE|, |gF_i|, |lambda|,
                                     // |F'|), [4] the fixed-point scale S (bits of a double)
  double *out;                       // [2 nr + nrho] knot gradients (phi | rho | F)
};
int adjoint_smem_bytes(const EAMParams &ep, int precision, int pass);
int adjoint_f_in_smem(const EAMParams &ep, int precision);
int launch_eam_adjoint(const Sys &s, const EAMParams &ep, int precision, const double *gF,
                       const AdjArgs &a, int64_t n_atoms, cudaStream_t st);

}  // namespace mdk
