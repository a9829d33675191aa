// mdk_api.cu -- the C ABI of libmdk.so (declared in include/mdk.h).
//
// Host code only marshals arguments, lays the caller's workspace out and
// enqueues kernels on the context's stream; every step of the MD path
// (binning, list build, forces, integration, reductions) runs in the
// kernels of k_build.cu and k_force.cu.  No device memory is allocated here.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mdk.h"
#include "mdk_internal.cuh"

using namespace mdk;

namespace {
// NVTX range over a C-ABI call (visible in Nsight timelines; a no-op when no
// tool is attached)
struct Nvtx {
  explicit Nvtx(const char *name) { nvtxRangePushA(name); }
  ~Nvtx() { nvtxRangePop(); }
  Nvtx(const Nvtx &) = delete;
  Nvtx &operator=(const Nvtx &) = delete;
};
}  // namespace

struct mdk_ctx {
  cudaStream_t stream = nullptr;
  int precision = MDK_FP64;
  int n_rep = 1;
  std::vector<double> lo, hi;
  std::vector<int> per;
  std::vector<int64_t> n_atoms;
  int64_t N = 0, N_cap = 0;
  std::vector<uint32_t> info0;
  int n_types = 0;
  double type_mass[kMaxTypes] = {0};
  // potential
  int pot = 0;  // 0 none, 1 LJ, 2 EAM, 3 BPNN
  LJParams lj{};
  EAMParams eam{};
  std::vector<double> eam_phi, eam_rho, eam_F;
  BPParams bp{};
  std::vector<double> bp_w64;  // packed device-order weights (kBpWords)
  std::vector<float> bp_w32;
  double *bp_w64_dev = nullptr;
  float *bp_w32_dev = nullptr;
  // neighbour plan
  bool planned = false;
  double rc_list = 0.0, skin = 0.3;
  int nmax_req = 0, rebuild_every = 0;
  int nmax = 0;
  int nmax_grow = 0;      // capacity wanted after an overflow
  // outer list (two-level lists): skin of the outer list, 0 = off; it takes
  // effect when it exceeds the Verlet skin
  double skin_outer = 0.0;
  int nmax1 = 0, nmax1_grow = 0;
  bool need_ws = false;   // the current workspace no longer fits the plan
  int n_cells = 0;
  std::vector<Grid> grids;
  // workspace
  char *ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_ok = false;
  Sys sys{};
  char *eam_base = nullptr;
  EAMTablesDev eam_dev{};
  double2 *adj_acc = nullptr;  // adjoint histograms: phi, rho (nr each), F (nrho)
  long long *adj_aux = nullptr;  // adjoint bounds and fixed-point scale
  double *adj_out = nullptr;   // [2 nr + nrho] knot gradients
  double *adj_gE = nullptr;    // [n_rep] energy weights
  double *thermo_ring = nullptr;
  int cur = 0;
  bool state_set = false, list_built = false, forces_valid = false;
  bool per_atom_valid = false;  // ea/wa hold U_i, W_i of the current order
  double u_p = 0.0;
  int thermo_every = 0, thermo_cap = 0;
  int64_t thermo_written = 0, thermo_read = 0;
  int64_t steps_done = 0;
  // steps_done - (device step counter) while no step is pending: the device
  // counter restarts at mdk_set_state and is carried by checkpoints
  int64_t steps_base = 0;
  // a stepping build overflowed: the state is mid-step (positions drifted,
  // velocities at the half step); the next mdk_step starts with the force
  // pass of that step
  bool pending = false;
  LaunchCfg cfg;  // pair-kernel launch shape (mdk_autotune)
  // CUDA graphs of two plain steps, one per parity of the gather copy
  bool graphs_on = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  uint64_t gkey[2] = {0, 0};
  cudaStream_t body_stream = nullptr;  // captures the conditional rebuild bodies
  int64_t graph_kernels = 0;  // kernels of one graph that run at every replay
  double *ctr_dev = nullptr;     // cell-centre tables in the workspace
  std::vector<double> ctr_host;  // their values (kept until the upload completes)
  int64_t body_kernels = 0;   // kernels of one conditional rebuild body
  long long graph_builds0 = 0;  // device count of in-graph builds at mdk_profile
  // moving window
  bool win_on = false;
  double win_L_behind = 0.0, win_L_ahead = 0.0, win_slab_lx = 0.0, win_gap = 0.0,
         win_depth = 0.0;
  uint32_t win_info = 0;
  std::vector<double> win_slab;  // [n][6]
  int64_t win_slab_cap = 0;      // slab atoms the workspace has room for
  double *win_slab_dev = nullptr;
  double win_front_bin = 1.0;
  double win_fixed_front = NAN;
  // Langevin regions (mdk_set_langevin)
  int lang_n = 0;
  double lang_xlo[kMaxLang] = {0}, lang_xhi[kMaxLang] = {0}, lang_kT[kMaxLang] = {0},
         lang_beta[kMaxLang] = {0}, lang_u[kMaxLang][3] = {{0}};
  unsigned long long lang_seed = 0;
  double lang_dt = 1.0;  // time step the noise amplitudes were computed for
  bool lang_rep_on = false;             // per-replica thermostats (mdk_set_langevin_replicas)
  std::vector<double> lang_rep_T, lang_rep_beta;
  std::vector<double> lang_rep_host;    // (g, sigma) per replica and type, as uploaded
  double *lang_rep_dev = nullptr;
  int win_nbins = 1;             // front bins over the box along x
  int win_nbins_cap = 0;         // bins the workspace has room for
  long long *win_fbin = nullptr;
  // measurement (mdk_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, int>> ev_force, ev_chain, ev_kick;  // (start, end) indices
  int64_t launches = 0;
};

namespace {

#define MDK_CK(call)                                                   \
  do {                                                                 \
    cudaError_t _e = (call);                                           \
    if (_e != cudaSuccess) {                                           \
      fprintf(stderr, "mdk: %s failed: %s\n", #call, cudaGetErrorString(_e)); \
      return MDK_ERR_CUDA;                                             \
    }                                                                  \
  } while (0)

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Carver {
  char *base;
  size_t off = 0;
  template <class T>
  T *take(size_t count) {
    off = align256(off);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += sizeof(T) * (count > 0 ? count : 1);
    return p;
  }
};

// Lay the workspace out (base == nullptr only measures).
size_t layout(mdk_ctx *c, char *base) {
  Carver cv{base};
  Sys &s = c->sys;
  const size_t Nc = (size_t)std::max<int64_t>(c->N_cap, 1);
  s.x = cv.take<double>(3 * Nc);
  s.v = cv.take<double>(3 * Nc);
  s.f = cv.take<double>(3 * Nc);
  s.xref = cv.take<double>(3 * Nc);
  s.tmp = cv.take<double>(9 * Nc);
  s.info = cv.take<uint32_t>(Nc);
  s.info0 = cv.take<uint32_t>(Nc);
  s.cellc = cv.take<uint32_t>(Nc);
  s.tmpu = cv.take<uint32_t>(2 * Nc);
  s.id = cv.take<int32_t>(Nc);
  s.tmpi = cv.take<int32_t>(Nc);
  s.pf = cv.take<float4>(Nc + 1);  // + the far record (pad_entry)
  const size_t gsz = c->precision == MDK_FP64 ? 32 : 16;
  s.pg[0] = cv.take<char>(gsz * (Nc + 1));  // + the far record (pad_entry)
  s.pg[1] = cv.take<char>(gsz * (Nc + 1));
  s.pgF = cv.take<char>(gsz * (c->pot == 2 ? Nc : 1));
  s.nnbr = cv.take<int32_t>(Nc);
  s.nbr = cv.take<uint32_t>((size_t)std::max(c->nmax, c->nmax_grow) * Nc);
  s.nnbr1 = cv.take<int32_t>(c->nmax1 > 0 ? Nc : 1);
  s.xfull = cv.take<double>(c->nmax1 > 0 ? 3 * Nc : 1);
  s.nbr1 = cv.take<uint32_t>(c->nmax1 > 0 ? (size_t)std::max(c->nmax1, c->nmax1_grow) * Nc : 1);
  s.hacc = cv.take<long long>(10 * Nc);
  s.ea = cv.take<double>(Nc);
  s.ka = cv.take<double>(Nc);
  s.wa = cv.take<double>(6 * Nc);
  s.rho = cv.take<double>(Nc);
  s.fp = cv.take<double>(Nc);
  s.cell_cnt = cv.take<int32_t>((size_t)c->n_cells + 1);
  s.cell_start = cv.take<int32_t>((size_t)c->n_cells + 2);
  s.cell_fill = cv.take<int32_t>((size_t)c->n_cells + 1);
  s.scan_part = cv.take<int32_t>(scan_blocks_for(c->n_cells + 1));
  c->win_slab_cap = (int64_t)(c->win_slab.size() / 6);
  c->win_slab_dev = cv.take<double>(c->win_slab.size());
  c->win_nbins_cap = c->win_nbins;
  c->win_fbin = cv.take<long long>(2 * (size_t)c->win_nbins);
  s.cell_of = cv.take<int32_t>(Nc);
  s.order = cv.take<int32_t>(Nc);
  s.grid = cv.take<Grid>(c->n_rep);
  {
    // cell-centre tables: per replica, nc[0] + nc[1] + nc[2] doubles
    size_t n_ctr = 0;
    for (const Grid &g : c->grids) n_ctr += (size_t)g.nc[0] + g.nc[1] + g.nc[2];
    double *ctr = cv.take<double>(std::max<size_t>(n_ctr, 1));
    c->ctr_dev = ctr;
    if (base) {
      size_t off = 0;
      for (Grid &g : c->grids)
        for (int d = 0; d < 3; ++d) {
          g.ctr[d] = ctr + off;
          off += (size_t)g.nc[d];
        }
    }
  }
  s.st = cv.take<DevStatus>(1);
  s.red = cv.take<double>((size_t)9 * c->n_rep);
  {
    // chunks per replica for the first pass of the sums: a single replica
    // may grow to N_cap atoms (window appends), batched replicas keep theirs
    int64_t per = c->n_rep == 1 ? (int64_t)Nc : 1;
    if (c->n_rep > 1)
      for (const Grid &g : c->grids) per = std::max<int64_t>(per, g.n_atoms);
    s.red_chunks = (int)std::max<int64_t>(1, (per + kRedChunk - 1) / kRedChunk);
    s.red_part = cv.take<double>((size_t)8 * c->n_rep * s.red_chunks);
  }
  c->thermo_ring = cv.take<double>((size_t)std::max(c->thermo_cap, 1) * c->n_rep * 10);
  // EAM tables: raw knots, (y, h m) FP64 and FP32 copies
  const int nr = c->pot == 2 ? c->eam.nr : 1, nrho = c->pot == 2 ? c->eam.nrho : 1;
  double *kn = cv.take<double>((size_t)2 * nr + nrho);
  EAMTablesDev &t = c->eam_dev;
  t.phi64 = cv.take<double2>(nr);
  t.rho64 = cv.take<double2>(nr);
  t.F64 = cv.take<double2>(nrho);
  t.rho_i32 = cv.take<float4>(nr);
  t.rho_d32 = cv.take<float2>(nr);
  t.phi_v32 = cv.take<float>(nr);
  t.pr32 = cv.take<float4>(nr);
  t.pr64 = cv.take<dvec4>(nr);
  t.pr8 = cv.take<float4>((size_t)2 * nr);
  c->adj_acc = cv.take<double2>((size_t)2 * nr + nrho);
  c->adj_out = cv.take<double>((size_t)2 * nr + nrho);
  c->adj_gE = cv.take<double>(c->n_rep);
  c->adj_aux = cv.take<long long>(8);
  c->lang_rep_dev = cv.take<double>((size_t)c->n_rep * kMaxTypes * 2);
  c->bp_w64_dev = cv.take<double>(kBpWords);
  c->bp_w32_dev = cv.take<float>(kBpWords);
  c->eam_base = reinterpret_cast<char *>(kn);
  c->eam.phi64 = t.phi64;
  c->eam.rho64 = t.rho64;
  c->eam.F64 = t.F64;
  c->eam.rho_i32 = t.rho_i32;
  c->eam.rho_d32 = t.rho_d32;
  c->eam.phi_v32 = t.phi_v32;
  c->eam.pr32 = t.pr32;
  c->eam.pr64 = t.pr64;
  c->eam.pr8 = t.pr8;
  return align256(cv.off);
}

int check_ctx(const mdk_ctx *c) { return c ? MDK_OK : MDK_ERR_BAD_ARG; }

int plan(mdk_ctx *c, double rc, double skin, int max_neighbors, int rebuild_every) {
  if (!(rc > 0.0) || !(skin >= 0.0) || max_neighbors < 0 || rebuild_every < 0)
    return MDK_ERR_BAD_ARG;
  const double rns_v = rc + skin;
  // with the outer list on, cells (and the outer list) span rc + skin_outer
  const bool outer = c->skin_outer > skin;
  const double rns = outer ? rc + c->skin_outer : rns_v;
  std::vector<Grid> gs((size_t)c->n_rep);
  int cells = 0;
  double max_density = 0.0;
  int64_t atom_off = 0;
  for (int r = 0; r < c->n_rep; ++r) {
    Grid &g = gs[(size_t)r];
    memset(&g, 0, sizeof(g));
    double vol = 1.0;
    for (int d = 0; d < 3; ++d) {
      const double lo = c->lo[3 * r + d], hi = c->hi[3 * r + d];
      const double L = hi - lo;
      if (!(L > 0.0)) return MDK_ERR_BAD_ARG;
      if (c->per[3 * r + d] && L < rns) return MDK_ERR_BOX_TOO_SMALL;
      // cells of size h = L/nc strictly above r_ns (see the cell-list search)
      int nc = (int)floor(L / (rns * (1.0 + 1e-10)));
      nc = std::max(1, std::min(nc, 1023));
      g.lo[d] = lo;
      g.hi[d] = hi;
      g.L[d] = L;
      g.nc[d] = nc;
      g.h[d] = L / nc;
      g.lo_c[d] = lo + 0.5 * g.h[d];
      g.inv_h[d] = 1.0 / g.h[d];
      g.hf[d] = (float)g.h[d];
      g.per[d] = c->per[3 * r + d] ? 1 : 0;
      vol *= L;
    }
    g.cell_off = cells;
    g.atom_off = (int)atom_off;
    g.n_atoms = (int)c->n_atoms[(size_t)r];
    atom_off += c->n_atoms[(size_t)r];
    const long long nc3 = (long long)g.nc[0] * g.nc[1] * g.nc[2];
    if ((long long)cells + nc3 > (1LL << 30)) return MDK_ERR_BAD_ARG;
    cells += (int)nc3;
    max_density = std::max(max_density, (double)c->n_atoms[(size_t)r] / vol);
  }
  if (scan_blocks_for(cells + 1) > 8192) return MDK_ERR_BAD_ARG;
  int nmax = (max_neighbors + kGroup - 1) / kGroup * kGroup;
  if (nmax == 0) {
    const double est = 4.0 / 3.0 * M_PI * rns_v * rns_v * rns_v * max_density;
    nmax = (int)ceil(1.6 * est + 24.0);
    nmax = (nmax + kGroup - 1) / kGroup * kGroup;
  }
  int nmax1 = 0;
  if (outer) {
    const double est1 = 4.0 / 3.0 * M_PI * rns * rns * rns * max_density;
    nmax1 = std::max((int)ceil(1.6 * est1 + 24.0), nmax);
    nmax1 = (nmax1 + kGroup - 1) / kGroup * kGroup;
  }
  c->grids = gs;
  c->n_cells = cells;
  c->nmax = nmax;
  c->nmax1 = std::max(nmax1, outer ? c->nmax1_grow : 0);
  c->rc_list = rc;
  c->skin = skin;
  c->nmax_req = max_neighbors;
  c->rebuild_every = rebuild_every;
  c->planned = true;
  return MDK_OK;
}

double pot_rc(const mdk_ctx *c) {
  if (c->pot == 1) return c->lj.rc;
  if (c->pot == 2) return c->eam.rc;
  if (c->pot == 3) return c->bp.rc;
  return 0.0;
}

// switch between full and half lists; the next call that needs the list
// rebuilds it
void use_list_kind(mdk_ctx *c, int kind) {
  if (c->cfg.half == kind) return;
  c->cfg.half = kind;
  c->sys.half = kind;
  c->list_built = false;
}

void fill_sys_params(mdk_ctx *c) {
  Sys &s = c->sys;
  s.N_cap = (int)c->N_cap;
  s.nmax = c->nmax;
  s.n_rep = c->n_rep;
  s.n_cells = c->n_cells;
  s.n_scan_blocks = scan_blocks_for(c->n_cells + 1);
  s.half = (c->pot == 1 || (c->pot == 2 && c->cfg.half == 1)) ? c->cfg.half : 0;
  const double rns = c->rc_list + c->skin;
  s.rns2 = rns * rns;
  // FP32 pre-filter band: cell-relative offsets have |p| <= 2h at a full
  // build (atoms beyond are flagged far and always take the exact test), and
  // with two-level lists at most (skin_outer - skin)/2 more at a filter build
  // (the displacement budget); each offset carries <= ulp(|p|)/2 of
  // rounding, so the float r^2 of a candidate near r_ns is within
  // ~2 r_ns (2 ulp(2h) + ulp(r_ns)) + 3 ulp(r_ns^2) of the exact one:
  // ~5e-7 r_ns^2 even for cells of rc + 1.5 A; 1e-4 leaves a wide margin, and
  // candidates inside the band take the FP64 test
  s.filt_lo = (float)(s.rns2 * (1.0 - 1e-4));
  s.filt_hi = (float)(s.rns2 * (1.0 + 1e-4));
  s.outer_on = c->nmax1 > 0 ? 1 : 0;
  s.nmax1 = c->nmax1;
  {
    const double r1 = c->rc_list + (s.outer_on ? c->skin_outer : c->skin);
    s.rns2_1 = r1 * r1;
    s.filt1_lo = (float)(s.rns2_1 * (1.0 - 1e-4));
    s.filt1_hi = (float)(s.rns2_1 * (1.0 + 1e-4));
    s.outer_budget = s.outer_on ? 0.5 * (c->skin_outer - c->skin) : 0.0;
  }
  s.half_skin2 = 0.25 * c->skin * c->skin;
  s.half_skin2f = (float)s.half_skin2;
  s.rebuild_every = c->rebuild_every;
  for (int t = 0; t < kMaxTypes; ++t) {
    const double m = t < c->n_types ? c->type_mass[t] : 1.0;
    s.mass[t] = m;
    s.acc_over_m[t] = kAcc / m;
    s.acc_over_mf[t] = (float)(kAcc / m);
    s.ke_m[t] = 0.5 * m / kAcc;
  }
  s.u_p = c->u_p;
  s.win_on = c->win_on ? 1 : 0;
  s.n_slab = (int)(c->win_slab.size() / 6);
  s.L_behind = c->win_L_behind;
  s.L_ahead = c->win_L_ahead;
  s.slab_lx = c->win_slab_lx;
  s.slab_gap = c->win_gap;
  s.piston_depth = c->win_depth;
  s.slab = c->win_slab_dev;
  s.slab_info = c->win_info;
  s.win_xlo = c->lo[0];
  s.win_xhi = c->hi[0];
  s.front_bin = c->win_front_bin;
  s.fixed_front = c->win_fixed_front;
  s.n_lang = c->lang_n;
  for (int q = 0; q < kMaxLang; ++q) {
    s.lang_xlo[q] = c->lang_xlo[q];
    s.lang_xhi[q] = c->lang_xhi[q];
    for (int d = 0; d < 3; ++d) s.lang_u[q][d] = c->lang_u[q][d];
    for (int t = 0; t < kMaxTypes; ++t) {
      // friction factor g = -beta m / A and noise amplitude
      // sigma = sqrt(24 beta m k_B T / (dt A)), once per region and type
      const double m = s.mass[t], beta = c->lang_beta[q];
      const double g = q < c->lang_n ? (-beta * m) / kAcc : 0.0;
      const double sig =
          q < c->lang_n ? sqrt((((24.0 * beta) * m) * c->lang_kT[q]) / (c->lang_dt * kAcc)) : 0.0;
      s.lang_g[q][t] = g;
      s.lang_sig[q][t] = sig;
    }
  }
  s.lang_seed = c->lang_seed;
  s.lang_rep_on = c->lang_rep_on ? 1 : 0;
  s.lang_rep = c->lang_rep_dev;
  s.n_fbins = c->win_nbins;
  s.fbin = c->win_fbin;
}

// (g, sigma) of every replica and atom type for the current dt, copied into
// the workspace
int upload_lang_rep(mdk_ctx *c) {
  if (!c->lang_rep_on || !c->ws_ok) return MDK_OK;
  const double kB = 8.617333262e-5;  // eV/K
  c->lang_rep_host.assign((size_t)c->n_rep * kMaxTypes * 2, 0.0);
  for (int r = 0; r < c->n_rep; ++r)
    for (int t = 0; t < kMaxTypes; ++t) {
      const double m = t < c->n_types ? c->type_mass[t] : 1.0, beta = c->lang_rep_beta[r];
      const double kT = kB * c->lang_rep_T[r];
      c->lang_rep_host[((size_t)r * kMaxTypes + t) * 2] = (-beta * m) / kAcc;
      c->lang_rep_host[((size_t)r * kMaxTypes + t) * 2 + 1] =
          sqrt((((24.0 * beta) * m) * kT) / (c->lang_dt * kAcc));
    }
  MDK_CK(cudaMemcpyAsync(c->lang_rep_dev, c->lang_rep_host.data(),
                         sizeof(double) * c->lang_rep_host.size(), cudaMemcpyHostToDevice,
                         c->stream));
  MDK_CK(cudaStreamSynchronize(c->stream));
  return MDK_OK;
}

int read_status(mdk_ctx *c, DevStatus *out) {
  MDK_CK(cudaMemcpyAsync(out, c->sys.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
  MDK_CK(cudaStreamSynchronize(c->stream));
  if (out->abort && !c->pending && c->state_set) {
    // stepping stopped at an overflowing build: n_steps counts the pending
    // step's force evaluation, the steps before it are complete
    c->pending = true;
    c->steps_done = c->steps_base + (out->n_steps - 1);
    c->forces_valid = false;
    c->per_atom_valid = false;
  }
  return MDK_OK;
}

int status_from_bits(unsigned bits) {
  if (bits & kStBounds) return MDK_ERR_BOUNDS;
  if (bits & kStNonfinite) return MDK_ERR_NONFINITE;
  if (bits & kStOverflow) return MDK_ERR_NEIGH_OVERFLOW;
  if (bits & kStAtomLost) return MDK_ERR_ATOM_LOST;
  if (bits & kStTimeout) return MDK_ERR_TIMEOUT;
  if (bits & kStCapacity) return MDK_ERR_CAPACITY;
  if (bits & kStRhoRange) return MDK_ERR_RHO_RANGE;
  return MDK_OK;
}

__global__ void k_init_status(Sys s, int N) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    DevStatus *st = s.st;
    st->N = N;
    st->abort = 0;
    st->step_build = 0;
    st->build_ovf = 0;
    st->rebuild = 1;
    st->bits = 0;
    st->max_nnbr = 0;
    st->since_build = 0;
    st->next_id = N;
    st->n_inserted = 0;
    st->n_deleted = 0;
    st->n_steps = 0;
  }
}

__global__ void k_clear_bits(Sys s) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    s.st->bits = 0;
    s.st->max_nnbr = 0;
  }
}

// a sample of a step that did not run (stepping aborted) carries step = NaN
// and is skipped by mdk_get_thermo
__global__ void k_thermo_store(Sys s, double *ring, int slot, double step) {
  const int r = threadIdx.x;
  if (r >= s.n_rep) return;
  double *o = ring + ((size_t)slot * s.n_rep + r) * 10;
  const double *q = s.red + 9 * r;
  o[0] = s.st->abort ? NAN : step;
  o[1] = q[0];
  o[2] = q[1];
  o[3] = q[8];
  for (int c = 0; c < 6; ++c) o[4 + c] = q[2 + c];
}


// checkpoint restore: the status of a loaded state before the replayed
// builds, then the saved counters after them
__global__ void k_ckpt_begin(Sys s, int N) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DevStatus *st = s.st;
  memset(st, 0, sizeof(DevStatus));
  st->N = N;
  st->win_cut = -INFINITY;
}

struct CkptCounters {
  long long n_steps, n_builds, n_graph_builds, n_full_builds, n_inserted, n_deleted;
  int since_build, next_id, outer_valid;
};

__global__ void k_ckpt_end(Sys s, CkptCounters k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DevStatus *st = s.st;
  st->n_steps = k.n_steps;
  st->n_builds = k.n_builds;
  st->n_graph_builds = k.n_graph_builds;
  st->n_full_builds = k.n_full_builds;
  st->n_inserted = k.n_inserted;
  st->n_deleted = k.n_deleted;
  st->since_build = k.since_build;
  st->next_id = k.next_id;
  st->outer_valid = k.outer_valid;
  st->rebuild = 0;
}

// next free event of the measurement pool (created on first use)
int take_event(mdk_ctx *c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    c->ev_pool.push_back(e);
  }
  return (int)c->ev_used++;
}

// record an event pair around what `launch` enqueues when profiling
template <class F>
int timed(mdk_ctx *c, std::vector<std::pair<int, int>> &log, int n_kernels, F launch) {
  int a = -1, b = -1;
  if (c->prof) {
    a = take_event(c);
    if (a >= 0) cudaEventRecord(c->ev_pool[(size_t)a], c->stream);
  }
  launch();
  c->launches += n_kernels;
  if (c->prof && a >= 0) {
    b = take_event(c);
    if (b >= 0) {
      cudaEventRecord(c->ev_pool[(size_t)b], c->stream);
      log.emplace_back(a, b);
    }
  }
  return cudaPeekAtLastError() == cudaSuccess ? MDK_OK : MDK_ERR_CUDA;
}

int force_pass(mdk_ctx *c, Mode mode, int energy, double dt) {
  StepArgs a{dt, c->cur, energy, (float)(0.5 * dt)};
  const bool cells = c->pot == 1 && c->cfg.half == 2;
  const bool half = (c->pot == 1 || c->pot == 2) && c->cfg.half == 1;
  const int nk = c->pot == 1 ? (half ? 2 : 1) : (c->pot == 2 && half ? 4 : 2);
  return timed(c, c->ev_force, nk, [&] {
    if (c->pot == 3)
      launch_bpnn(c->sys, c->bp, c->precision, mode, a, c->stream);
    else if (cells)
      launch_lj_cells(c->sys, c->lj, c->precision, mode, a, c->cfg, c->stream);
    else if (half && c->pot == 2)
      launch_eam_half(c->sys, c->eam, c->precision, mode, a, c->cfg, c->stream);
    else if (half)
      launch_lj_half(c->sys, c->lj, c->precision, mode, a, c->cfg, c->stream);
    else if (c->pot == 1)
      launch_lj(c->sys, c->lj, c->precision, mode, a, c->cfg, c->stream);
    else
      launch_eam(c->sys, c->eam, c->precision, mode, a, c->cfg, c->stream);
  });
}


int rebuild_chain(mdk_ctx *c, int count_step) {
  return timed(c, c->ev_chain, rebuild_chain_kernels(c->sys), [&] {
    launch_rebuild(c->sys, c->cur, c->precision, count_step, c->stream);
  });
}

int ensure_ready(mdk_ctx *c) {
  if (!c->ws_ok || c->need_ws) return MDK_ERR_WORKSPACE;
  if (!c->state_set) return MDK_ERR_ORDER;
  if (c->pot == 0) return MDK_ERR_ORDER;
  if (pot_rc(c) > c->rc_list) return MDK_ERR_ORDER;
  return MDK_OK;
}

// capacities wanted after a list overflow (Verlet list, outer list)
void note_overflow(mdk_ctx *c, const DevStatus &st) {
  if (st.max_nnbr > c->nmax)
    c->nmax_grow = ((int)ceil(st.max_nnbr * 1.25) + 8 + kGroup - 1) / kGroup * kGroup;
  if (c->nmax1 > 0 && st.max_nnbr1 > c->nmax1)
    c->nmax1_grow = ((int)ceil(st.max_nnbr1 * 1.25) + 8 + kGroup - 1) / kGroup * kGroup;
}

int build_now(mdk_ctx *c) {
  Nvtx range("mdk list build");
  launch_set_rebuild_flag(c->sys, c->stream);
  int rr = rebuild_chain(c, 0);
  if (rr) return rr;
  DevStatus st;
  int rc = read_status(c, &st);
  if (rc) return rc;
  if (st.bits & kStOverflow) {
    note_overflow(c, st);
    c->need_ws = true;
    c->list_built = false;
    return MDK_ERR_NEIGH_OVERFLOW;
  }
  if (st.bits & kStNonfinite) return MDK_ERR_NONFINITE;
  c->list_built = true;
  return MDK_OK;
}

// Atoms present: the host count, or the device's once a window can change it.
int device_n(mdk_ctx *c, int64_t *n) {
  if (!c->win_on) {
    *n = c->N;
    return MDK_OK;
  }
  DevStatus st;
  int r = read_status(c, &st);
  if (r) return r;
  c->N = st.N;
  *n = st.N;
  return MDK_OK;
}

// Internal index of the atom of rank r in ascending-id order (the caller's
// order once a window has appended or deleted atoms).
int caller_order(mdk_ctx *c, int64_t n, std::vector<int32_t> &ord, std::vector<int32_t> &id) {
  id.resize((size_t)n);
  ord.resize((size_t)n);
  if (n > 0) {
    MDK_CK(cudaMemcpyAsync(id.data(), c->sys.id, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                           c->stream));
    MDK_CK(cudaStreamSynchronize(c->stream));
  }
  for (int64_t r = 0; r < n; ++r) ord[(size_t)r] = (int32_t)r;
  std::sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return id[(size_t)a] < id[(size_t)b]; });
  return MDK_OK;
}

// comp doubles per atom of the SoA array src (component stride N_cap) in the
// caller's order into out (host, or device when on_device).
int gather_by_id(mdk_ctx *c, int64_t n, const double *src, int comp, double *out, int on_device) {
  std::vector<int32_t> ord, id;
  int r = caller_order(c, n, ord, id);
  if (r) return r;
  std::vector<double> buf((size_t)n * comp), res((size_t)n * comp);
  for (int k = 0; k < comp && n > 0; ++k)
    MDK_CK(cudaMemcpyAsync(buf.data() + (size_t)k * n, src + (size_t)k * c->N_cap,
                           sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  MDK_CK(cudaStreamSynchronize(c->stream));
  for (int64_t q = 0; q < n; ++q)
    for (int k = 0; k < comp; ++k) res[(size_t)q * comp + k] = buf[(size_t)k * n + ord[(size_t)q]];
  if (n == 0) return MDK_OK;
  if (on_device) {
    MDK_CK(cudaMemcpyAsync(out, res.data(), sizeof(double) * res.size(), cudaMemcpyHostToDevice,
                           c->stream));
    MDK_CK(cudaStreamSynchronize(c->stream));
  } else {
    memcpy(out, res.data(), sizeof(double) * res.size());
  }
  return MDK_OK;
}

// Fingerprint of everything a captured step bakes into its kernel
// parameters (FNV-1a over the parameter structs and dt).
uint64_t fnv(uint64_t h, const void *p, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t q = 0; q < n; ++q) {
    h ^= b[q];
    h *= 1099511628211ull;
  }
  return h;
}

uint64_t graph_key(const mdk_ctx *c, double dt) {
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, &c->sys, sizeof(Sys));
  h = fnv(h, &c->lj, sizeof(LJParams));
  h = fnv(h, &c->eam, sizeof(EAMParams));
  h = fnv(h, &c->cfg, sizeof(LaunchCfg));
  h = fnv(h, &c->pot, sizeof(int));
  h = fnv(h, &c->bp, sizeof(BPParams));
  h = fnv(h, &c->precision, sizeof(int));
  h = fnv(h, &dt, sizeof(double));
  return h;
}

// The rebuild chain of a captured step: the head kernel (k_pre) decides and
// sets the value of an IF conditional node whose body holds the rest of the
// chain, so a step without a rebuild runs two kernels, not the whole chain.
int capture_conditional_chain(mdk_ctx *c) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  MDK_CK(cudaStreamGetCaptureInfo(c->cap_stream, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle h;
  MDK_CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  launch_rebuild_head(c->sys, 1, h, c->cap_stream);
  c->launches += 1;
  MDK_CK(cudaPeekAtLastError());
  MDK_CK(cudaStreamGetCaptureInfo(c->cap_stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  MDK_CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
  MDK_CK(cudaStreamUpdateCaptureDependencies(c->cap_stream, &node, nullptr, 1,
                                             cudaStreamSetCaptureDependencies));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  MDK_CK(cudaStreamBeginCaptureToGraph(c->body_stream, body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal));
  c->body_kernels = launch_rebuild_body(c->sys, c->cur, c->precision, 1, c->body_stream);
  const cudaError_t e = cudaPeekAtLastError();
  cudaGraph_t out = nullptr;
  MDK_CK(cudaStreamEndCapture(c->body_stream, &out));
  return e == cudaSuccess ? MDK_OK : MDK_ERR_CUDA;
}

// Capture two plain steps (force pass + rebuild chain, twice) starting from
// gather-copy parity `parity`; the graph ends at the same parity.
int capture_two_steps(mdk_ctx *c, int parity, double dt, uint64_t key) {
  if (!c->cap_stream) MDK_CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  if (!c->body_stream) MDK_CK(cudaStreamCreateWithFlags(&c->body_stream, cudaStreamNonBlocking));
  const cudaStream_t keep_stream = c->stream;
  const int keep_cur = c->cur;
  const bool keep_prof = c->prof;
  const int64_t keep_launches = c->launches;
  MDK_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  c->stream = c->cap_stream;
  c->cur = parity;
  c->prof = false;
  int r = MDK_OK;
  for (int h = 0; h < 2 && !r; ++h) {
    r = force_pass(c, kStep, 0, dt);
    c->cur ^= 1;
    if (!r) r = capture_conditional_chain(c);
  }
  c->stream = keep_stream;
  c->cur = keep_cur;
  c->prof = keep_prof;
  c->graph_kernels = c->launches - keep_launches;
  c->launches = keep_launches;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (r || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return r ? r : MDK_ERR_CUDA;
  }
  if (c->gexec[parity]) cudaGraphExecDestroy(c->gexec[parity]);
  c->gexec[parity] = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&c->gexec[parity], g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return MDK_ERR_CUDA;
  c->gkey[parity] = key;
  return MDK_OK;
}

}  // namespace

extern "C" {

const char *mdk_status_string(int s) {
  switch (s) {
    case MDK_OK: return "ok";
    case MDK_ERR_BAD_ARG: return "bad argument";
    case MDK_ERR_BOX_TOO_SMALL: return "periodic box shorter than rc + skin";
    case MDK_ERR_NEIGH_OVERFLOW: return "neighbour list overflow (capacity raised; resize the workspace)";
    case MDK_ERR_ATOM_LOST: return "atom moved more than one cell between builds";
    case MDK_ERR_NONFINITE: return "non-finite position or force";
    case MDK_ERR_TIMEOUT: return "device wait timed out";
    case MDK_ERR_CUDA: return "CUDA runtime error";
    case MDK_ERR_WORKSPACE: return "workspace missing or too small";
    case MDK_ERR_ORDER: return "call made before a required call";
    case MDK_ERR_RHO_RANGE: return "EAM density above the F table (extrapolated)";
    case MDK_ERR_TOO_LARGE: return "size above the fixed maximum of the allocation-free entry point";
    case MDK_ERR_CAPACITY: return "atom capacity full: the moving window could not append all atoms";
    case MDK_ERR_BOUNDS: return "index out of range caught by a debug-build check (results invalid)";
    default: return "unknown status";
  }
}

int mdk_create_batch(mdk_ctx **out, int n_rep, const double *box_lo, const double *box_hi,
                     const int *periodic, const int64_t *n_atoms, const double *masses,
                     int precision, void *cuda_stream) {
  if (!out || n_rep < 1 || n_rep > (1 << 20) || !box_lo || !box_hi || !periodic || !n_atoms)
    return MDK_ERR_BAD_ARG;
  if (precision != MDK_FP64 && precision != MDK_MIXED) return MDK_ERR_BAD_ARG;
  int64_t total = 0;
  for (int r = 0; r < n_rep; ++r) {
    if (n_atoms[r] < 0) return MDK_ERR_BAD_ARG;
    total += n_atoms[r];
  }
  if (total >= ((int64_t)1 << 26)) return MDK_ERR_BAD_ARG;
  if (total > 0 && !masses) return MDK_ERR_BAD_ARG;
  mdk_ctx *c = new (std::nothrow) mdk_ctx();
  if (!c) return MDK_ERR_BAD_ARG;
  c->stream = (cudaStream_t)cuda_stream;
  c->precision = precision;
  c->n_rep = n_rep;
  c->lo.assign(box_lo, box_lo + 3 * n_rep);
  c->hi.assign(box_hi, box_hi + 3 * n_rep);
  c->per.assign(periodic, periodic + 3 * n_rep);
  c->n_atoms.assign(n_atoms, n_atoms + n_rep);
  c->N = total;
  c->N_cap = total;
  c->info0.resize((size_t)total);
  int64_t i = 0;
  for (int r = 0; r < n_rep; ++r)
    for (int64_t q = 0; q < n_atoms[r]; ++q, ++i) {
      const double m = masses[i];
      if (!(m > 0.0)) {
        delete c;
        return MDK_ERR_BAD_ARG;
      }
      int t = 0;
      while (t < c->n_types && c->type_mass[t] != m) ++t;
      if (t == c->n_types) {
        if (c->n_types == kMaxTypes) {
          delete c;
          return MDK_ERR_BAD_ARG;
        }
        c->type_mass[c->n_types++] = m;
      }
      c->info0[(size_t)i] = (uint32_t)t | ((uint32_t)r << 8);
    }
  *out = c;
  return MDK_OK;
}

int mdk_create(mdk_ctx **out, const double box_lo[3], const double box_hi[3],
               const int periodic[3], int64_t N, const double *masses, int precision,
               void *cuda_stream) {
  return mdk_create_batch(out, 1, box_lo, box_hi, periodic, &N, masses, precision,
                          cuda_stream);
}

int mdk_destroy(mdk_ctx *c) {
  if (!c) return MDK_ERR_BAD_ARG;
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (int q = 0; q < 2; ++q)
    if (c->gexec[q]) cudaGraphExecDestroy(c->gexec[q]);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->body_stream) cudaStreamDestroy(c->body_stream);
  delete c;
  return MDK_OK;
}

int mdk_set_capacity(mdk_ctx *c, int64_t max_atoms) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (max_atoms < c->N || max_atoms >= ((int64_t)1 << 26)) return MDK_ERR_BAD_ARG;
  if (c->n_rep != 1 && max_atoms != c->N) return MDK_ERR_BAD_ARG;
  c->N_cap = max_atoms;
  c->ws_ok = false;
  return MDK_OK;
}

int mdk_set_potential_lj(mdk_ctx *c, double eps, double sigma, double rc, int shift_mode) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (!(eps > 0.0) || !(sigma > 0.0) || !(rc > 0.0) || shift_mode < 0 || shift_mode > 2)
    return MDK_ERR_BAD_ARG;
  LJParams &p = c->lj;
  const double sr = sigma / rc, s6 = sr * sr * sr * sr * sr * sr;
  const double u_rc = 4.0 * eps * (s6 * s6 - s6);
  const double du_rc = -24.0 * eps * (2.0 * s6 * s6 - s6) / rc;
  p.eps4 = 4.0 * eps;
  p.eps24 = 24.0 * eps;
  p.sig2 = sigma * sigma;
  p.rc = rc;
  p.rc2 = rc * rc;
  p.u_shift = shift_mode >= 1 ? u_rc : 0.0;
  p.du_rc = shift_mode == 2 ? du_rc : 0.0;
  p.eps4f = (float)p.eps4;
  p.eps24f = (float)p.eps24;
  p.sig2f = (float)p.sig2;
  p.rc2f = (float)p.rc2;
  p.rcf = (float)rc;
  p.u_shiftf = (float)p.u_shift;
  p.du_rcf = (float)p.du_rc;
  p.shift_mode = shift_mode;
  c->pot = 1;
  if (!c->planned) plan(c, rc, 0.3, 0, 0);
  return MDK_OK;
}

int mdk_set_potential_eam(mdk_ctx *c, int nr, double rc, const double *phi, const double *rho,
                          int nrho, double rho_max, const double *F) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  // FP64 tables of phi and rho must fit shared memory together (16 B per knot)
  if (nr < 3 || nr > 7168 || nrho < 3 || nrho > 65536 || !(rc > 0.0) || !(rho_max > 0.0) ||
      !phi || !rho || !F)
    return MDK_ERR_BAD_ARG;
  const bool resized = c->pot != 2 || c->eam.nr != nr || c->eam.nrho != nrho;
  EAMParams &e = c->eam;
  e.nr = nr;
  e.nrho = nrho;
  e.rc = rc;
  e.rc2 = rc * rc;
  e.dr = rc / (nr - 1);
  e.inv_dr = 1.0 / e.dr;
  e.rho_max = rho_max;
  e.drho = rho_max / (nrho - 1);
  e.inv_drho = 1.0 / e.drho;
  e.rc2f = (float)e.rc2;
  e.inv_drf = (float)e.inv_dr;
  c->eam_phi.assign(phi, phi + nr);
  c->eam_rho.assign(rho, rho + nr);
  c->eam_F.assign(F, F + nrho);
  c->pot = 2;
  if (c->cfg.half == MDK_LIST_CELLS) use_list_kind(c, MDK_LIST_FULL);  // LJ only
  if (!c->planned) plan(c, rc, 0.3, 0, 0);
  if (resized) {
    c->ws_ok = false;  // table area changes size: a new workspace is needed
    return MDK_OK;
  }
  if (c->ws_ok) {
    // same table sizes: upload into the existing workspace
    double *kn = reinterpret_cast<double *>(c->eam_base);
    MDK_CK(cudaMemcpyAsync(kn, phi, sizeof(double) * nr, cudaMemcpyHostToDevice, c->stream));
    MDK_CK(cudaMemcpyAsync(kn + nr, rho, sizeof(double) * nr, cudaMemcpyHostToDevice, c->stream));
    MDK_CK(cudaMemcpyAsync(kn + 2 * nr, F, sizeof(double) * nrho, cudaMemcpyHostToDevice,
                           c->stream));
    launch_eam_prepare(e, kn, kn + nr, kn + 2 * nr, c->eam_dev, c->stream);
    MDK_CK(cudaPeekAtLastError());
    c->forces_valid = false;
  }
  return MDK_OK;
}

// weights of the BPNN model into the workspace, shared-memory limit of its kernel
int upload_bpnn(mdk_ctx *c) {
  if (!c->bp_w64_dev || c->bp_w64.empty()) return MDK_ERR_ORDER;
  MDK_CK(cudaMemcpyAsync(c->bp_w64_dev, c->bp_w64.data(), sizeof(double) * kBpWords,
                         cudaMemcpyHostToDevice, c->stream));
  MDK_CK(cudaMemcpyAsync(c->bp_w32_dev, c->bp_w32.data(), sizeof(float) * kBpWords,
                         cudaMemcpyHostToDevice, c->stream));
  c->bp.w64 = c->bp_w64_dev;
  c->bp.w32 = c->bp_w32_dev;
  if (configure_bpnn_smem(bpnn_smem_bytes(c->bp, c->precision, c->nmax, nullptr), c->precision))
    return MDK_ERR_CUDA;
  return MDK_OK;
}

int mdk_set_potential_bpnn(mdk_ctx *c, double rc, int n_rad, const int *rad_kind,
                           const double *rad_par, int n_ang, const int *ang_kind,
                           const double *ang_par, int H1, int H2, const double *W01,
                           const double *b1, const double *W12, const double *b2,
                           const double *w23, double b3) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (!(rc > 0.0) || !std::isfinite(rc) || n_rad < 0 || n_rad > kBpRad || n_ang < 0 ||
      n_ang > kBpSlots || n_rad + n_ang < 1 || H1 < 1 || H1 > kBpH || H2 < 1 || H2 > kBpH ||
      (n_rad > 0 && (!rad_kind || !rad_par)) || (n_ang > 0 && (!ang_kind || !ang_par)) || !W01 ||
      !b1 || !W12 || !b2 || !w23 || !std::isfinite(b3))
    return MDK_ERR_BAD_ARG;
  BPParams p{};
  p.n_rad = n_rad;
  p.H1 = H1;
  p.H2 = H2;
  p.rc = rc;
  p.rcf = (float)rc;
  p.b3 = b3;
  p.b3f = (float)b3;
  for (int m = 0; m < n_rad; ++m) {
    const int k = rad_kind[m];
    const double p0 = rad_par[2 * m], p1 = rad_par[2 * m + 1];
    if ((k != 1 && k != 2 && k != 3) || !std::isfinite(p0) || !std::isfinite(p1))
      return MDK_ERR_BAD_ARG;
    p.rad_kind[m] = k;
    p.rad_p0[m] = p0;
    p.rad_p1[m] = p1;
    p.rad_p0f[m] = (float)p0;
    p.rad_p1f[m] = (float)p1;
  }
  // angular functions onto the slot grid.  When every zeta is 1, 2, 4 or 16
  // the zeta groups are those four, in that order (the kernel's compiled
  // power ladder); otherwise groups are numbered in order of appearance.
  static const double kZetaSet[kBpZ] = {1.0, 2.0, 4.0, 16.0};
  p.zset = 1;
  for (int m = 0; m < n_ang; ++m) {
    const double zeta = ang_par[3 * m];
    bool in = false;
    for (int q = 0; q < kBpZ; ++q) in = in || zeta == kZetaSet[q];
    if (!in) p.zset = 0;
  }
  if (p.zset == 1) {
    p.nZ = kBpZ;
    for (int q = 0; q < kBpZ; ++q) {
      p.z_zeta[q] = kZetaSet[q];
      p.z_zetaf[q] = (float)kZetaSet[q];
      p.z_pow[q] = (int)kZetaSet[q] - 1;
      p.z_coef[q] = ldexp(1.0, 1 - (int)kZetaSet[q]);
      p.z_coeff[q] = (float)p.z_coef[q];
    }
  }
  std::vector<int> slot_of((size_t)n_ang);
  for (int m = 0; m < n_ang; ++m) {
    const int k = ang_kind[m];
    const double zeta = ang_par[3 * m], lam = ang_par[3 * m + 1], eta = ang_par[3 * m + 2];
    if ((k != 4 && k != 5) || !(zeta >= 1.0 && zeta <= 64.0) || zeta != floor(zeta) ||
        (lam != 1.0 && lam != -1.0) || !std::isfinite(eta))
      return MDK_ERR_BAD_ARG;
    int y = -1, z = -1;
    for (int q = 0; q < p.nY; ++q)
      if (p.y_eta[q] == eta && p.y_kind[q] == k) y = q;
    if (y < 0) {
      if (p.nY == kBpY) return MDK_ERR_BAD_ARG;
      y = p.nY++;
      p.y_eta[y] = eta;
      p.y_etaf[y] = (float)eta;
      p.y_kind[y] = k;
      if (k == 4) p.any4 = 1;
    }
    for (int q = 0; q < p.nZ; ++q)
      if (p.z_zeta[q] == zeta) z = q;
    if (z < 0) {
      if (p.nZ == kBpZ) return MDK_ERR_BAD_ARG;
      z = p.nZ++;
      p.z_zeta[z] = zeta;
      p.z_zetaf[z] = (float)zeta;
      p.z_pow[z] = (int)zeta - 1;
      p.z_coef[z] = ldexp(1.0, 1 - (int)zeta);
      p.z_coeff[z] = (float)p.z_coef[z];
    }
    const int slot = (y * kBpZ + z) * 2 + (lam < 0.0 ? 1 : 0);
    if ((p.slot_mask >> slot) & 1ull) return MDK_ERR_BAD_ARG;  // the same function twice
    p.slot_mask |= 1ull << slot;
    slot_of[(size_t)m] = slot;
  }
  // weights in device order: rows [radial 0..kBpRad), [slots 0..kBpSlots)
  std::vector<double> w((size_t)kBpWords, 0.0);
  const int G = n_rad + n_ang;
  for (int q = 0; q < G * H1; ++q)
    if (!std::isfinite(W01[q])) return MDK_ERR_BAD_ARG;
  for (int m = 0; m < G; ++m) {
    const int row = m < n_rad ? m : kBpRad + slot_of[(size_t)(m - n_rad)];
    for (int j = 0; j < H1; ++j) w[(size_t)row * H1 + j] = W01[(size_t)m * H1 + j];
  }
  size_t o = (size_t)kBpIn * H1;
  for (int j = 0; j < H1; ++j) w[o + j] = b1[j];
  o += H1;
  for (int q = 0; q < H1 * H2; ++q) w[o + q] = W12[q];
  o += (size_t)H1 * H2;
  for (int k = 0; k < H2; ++k) w[o + k] = b2[k];
  o += H2;
  for (int k = 0; k < H2; ++k) w[o + k] = w23[k];
  for (double v : w)
    if (!std::isfinite(v)) return MDK_ERR_BAD_ARG;
  c->bp_w64 = w;
  c->bp_w32.assign(w.begin(), w.end());
  p.w64 = c->bp_w64_dev;
  p.w32 = c->bp_w32_dev;
  c->bp = p;
  c->pot = 3;
  use_list_kind(c, MDK_LIST_FULL);  // the BPNN pass reads full lists
  c->forces_valid = false;
  if (!c->planned) plan(c, rc, 0.3, 0, 0);
  if (c->ws_ok) {
    const int r = upload_bpnn(c);
    if (r) return r;
  }
  return MDK_OK;
}

int mdk_plan_neighbors(mdk_ctx *c, double rc, double skin, int max_neighbors, int rebuild_every) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  const int old_nmax = c->nmax, old_cells = c->n_cells, old_nmax1 = c->nmax1;
  int rc_ = plan(c, rc, skin, max_neighbors, rebuild_every);
  if (rc_) return rc_;
  if (c->nmax != old_nmax || c->n_cells != old_cells || c->nmax1 != old_nmax1) c->need_ws = true;
  c->list_built = false;
  return MDK_OK;
}

int mdk_workspace_size(const mdk_ctx *cc, size_t *bytes) {
  if (!cc || !bytes) return MDK_ERR_BAD_ARG;
  mdk_ctx *c = const_cast<mdk_ctx *>(cc);
  if (!c->planned) {
    if (c->pot == 0) return MDK_ERR_ORDER;
    int r = plan(c, pot_rc(c), 0.3, 0, 0);
    if (r) return r;
  }
  Sys keep = c->sys;
  EAMParams ekeep = c->eam;
  EAMTablesDev tkeep = c->eam_dev;
  char *kb = c->eam_base;
  double *tr = c->thermo_ring;
  *bytes = layout(c, nullptr);
  c->sys = keep;
  c->eam = ekeep;
  c->eam_dev = tkeep;
  c->eam_base = kb;
  c->thermo_ring = tr;
  return MDK_OK;
}

int mdk_set_workspace(mdk_ctx *c, void *dev_ptr, size_t bytes) {
  if (check_ctx(c) || !dev_ptr || ((uintptr_t)dev_ptr & 255)) return MDK_ERR_BAD_ARG;
  size_t need = 0;
  int r = mdk_workspace_size(c, &need);
  if (r) return r;
  if (bytes < need) return MDK_ERR_WORKSPACE;
  c->ws = (char *)dev_ptr;
  c->ws_bytes = bytes;
  c->nmax = std::max(c->nmax, c->nmax_grow);
  c->nmax_grow = 0;
  if (c->nmax1 > 0) c->nmax1 = std::max(c->nmax1, c->nmax1_grow);
  c->nmax1_grow = 0;
  c->need_ws = false;
  layout(c, c->ws);
  fill_sys_params(c);
  Sys &s = c->sys;
  MDK_CK(cudaMemsetAsync(s.st, 0, sizeof(DevStatus), c->stream));
  launch_init_far(s, c->precision, c->stream);
  MDK_CK(cudaMemsetAsync(s.cell_cnt, 0, sizeof(int32_t) * (c->n_cells + 1), c->stream));
  MDK_CK(cudaMemsetAsync(s.hacc, 0, sizeof(long long) * 10 * (size_t)std::max<int64_t>(c->N_cap, 1),
                         c->stream));
  MDK_CK(cudaMemsetAsync(c->win_fbin, 0, sizeof(long long) * 2 * c->win_nbins, c->stream));
  if (!c->win_slab.empty())
    MDK_CK(cudaMemcpyAsync(c->win_slab_dev, c->win_slab.data(), sizeof(double) * c->win_slab.size(),
                           cudaMemcpyHostToDevice, c->stream));
  MDK_CK(cudaMemcpyAsync(s.grid, c->grids.data(), sizeof(Grid) * c->n_rep,
                         cudaMemcpyHostToDevice, c->stream));
  {
    // the cell centres, with the expression the kernels used to evaluate
    c->ctr_host.clear();
    for (const Grid &g : c->grids)
      for (int d = 0; d < 3; ++d)
        for (int q = 0; q < g.nc[d]; ++q) c->ctr_host.push_back(std::fma((double)q, g.h[d], g.lo_c[d]));
    if (!c->ctr_host.empty())
      MDK_CK(cudaMemcpyAsync(c->ctr_dev, c->ctr_host.data(), sizeof(double) * c->ctr_host.size(),
                             cudaMemcpyHostToDevice, c->stream));
  }
  if (c->N > 0)
    MDK_CK(cudaMemcpyAsync(s.info0, c->info0.data(), sizeof(uint32_t) * c->N,
                           cudaMemcpyHostToDevice, c->stream));
  if (c->pot == 3) {
    if (upload_bpnn(c)) return MDK_ERR_CUDA;
  }
  if (c->pot == 2) {
    EAMParams &e = c->eam;
    double *kn = reinterpret_cast<double *>(c->eam_base);
    MDK_CK(cudaMemcpyAsync(kn, c->eam_phi.data(), sizeof(double) * e.nr, cudaMemcpyHostToDevice,
                           c->stream));
    MDK_CK(cudaMemcpyAsync(kn + e.nr, c->eam_rho.data(), sizeof(double) * e.nr,
                           cudaMemcpyHostToDevice, c->stream));
    MDK_CK(cudaMemcpyAsync(kn + 2 * e.nr, c->eam_F.data(), sizeof(double) * e.nrho,
                           cudaMemcpyHostToDevice, c->stream));
    launch_eam_prepare(e, kn, kn + e.nr, kn + 2 * e.nr, c->eam_dev, c->stream);
    MDK_CK(cudaPeekAtLastError());
    if (configure_eam_smem(eam_smem_bytes(e, c->precision, 1), eam_smem_bytes(e, c->precision, 2),
                           c->precision) ||
        configure_eam_half_smem(eam_smem_bytes(e, c->precision, 1),
                                eam_smem_bytes(e, c->precision, 2), c->precision))
      return MDK_ERR_CUDA;
  }
  MDK_CK(cudaStreamSynchronize(c->stream));
  c->ws_ok = true;
  c->state_set = false;
  c->pending = false;
  c->list_built = false;
  c->forces_valid = false;
  c->cur = 0;
  c->thermo_written = c->thermo_read = 0;
  return upload_lang_rep(c);
}

int mdk_set_state(mdk_ctx *c, const double *x, const double *v, int on_device) {
  if (check_ctx(c) || (!x && c->N > 0)) return MDK_ERR_BAD_ARG;
  if (!c->ws_ok) return MDK_ERR_WORKSPACE;
  Sys &s = c->sys;
  const double *xd = x, *vd = v;
  if (!on_device && c->N > 0) {
    double *stage = s.tmp;
    MDK_CK(cudaMemcpyAsync(stage, x, sizeof(double) * 3 * c->N, cudaMemcpyHostToDevice, c->stream));
    xd = stage;
    vd = nullptr;
    if (v) {
      MDK_CK(cudaMemcpyAsync(stage + 3 * c->N, v, sizeof(double) * 3 * c->N,
                             cudaMemcpyHostToDevice, c->stream));
      vd = stage + 3 * c->N;
    }
  }
  k_init_status<<<1, 32, 0, c->stream>>>(s, (int)c->N);
  launch_load_state(s, xd, vd, c->precision, c->cur, c->stream);
  MDK_CK(cudaPeekAtLastError());
  c->pending = false;
  c->steps_base = c->steps_done;
  c->state_set = true;
  c->list_built = false;
  c->forces_valid = false;
  return MDK_OK;
}

int mdk_get_state(mdk_ctx *c, double *x, double *v, int on_device) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (!c->ws_ok || !c->state_set) return MDK_ERR_ORDER;
  Sys &s = c->sys;
  if (c->win_on) {
    int64_t n = 0;
    int r = device_n(c, &n);
    if (!r && x) r = gather_by_id(c, n, s.x, 3, x, on_device);
    if (!r && v) r = gather_by_id(c, n, s.v, 3, v, on_device);
    return r;
  }
  if (c->N == 0) return MDK_OK;
  if (on_device) {
    launch_store_state(s, x, v, c->stream);
    MDK_CK(cudaPeekAtLastError());
    return MDK_OK;
  }
  double *stage = s.tmp;
  launch_store_state(s, x ? stage : nullptr, v ? stage + 3 * c->N : nullptr, c->stream);
  if (x)
    MDK_CK(cudaMemcpyAsync(x, stage, sizeof(double) * 3 * c->N, cudaMemcpyDeviceToHost, c->stream));
  if (v)
    MDK_CK(cudaMemcpyAsync(v, stage + 3 * c->N, sizeof(double) * 3 * c->N, cudaMemcpyDeviceToHost,
                           c->stream));
  MDK_CK(cudaStreamSynchronize(c->stream));
  return MDK_OK;
}

int mdk_get_natoms(mdk_ctx *c, int64_t *n) {
  if (!c || !n) return MDK_ERR_BAD_ARG;
  if (c->win_on && c->ws_ok && c->state_set) return device_n(c, n);
  *n = c->N;
  return MDK_OK;
}

}  // extern "C"

namespace {

// ---- checkpoints ---------------------------------------------------------------
// Layout of a checkpoint (host bytes): the header, then per atom in the saving
// context's internal order, component-major: x[3][N], v[3][N], f[3][N],
// x_ref[3][N] (positions of the last list build), x_full[3][N] (two-level
// lists only: positions of the last full build), id[N] (int32), info[N]
// (uint32: type, piston flag, replica).
constexpr char kCkptMagic[8] = {'M', 'D', 'K', 'C', 'K', 'P', 'T', '1'};
enum : int32_t {
  kCkList = 1,        // a list existed: x_ref (and x_full) are meaningful
  kCkForces = 2,      // f holds the forces of x
  kCkPending = 4,     // mid-step: v at the half step, the force pass pending
  kCkOuter = 8,       // x_full present (two-level lists)
  kCkOuterValid = 16  // the outer list of x_full was built
};

struct CkptHeader {
  char magic[8];
  int32_t version, precision, n_rep, flags;
  int64_t N, steps_done;
  int64_t n_steps, n_builds, n_graph_builds, n_full_builds, n_inserted, n_deleted;
  int32_t since_build, next_id;
  double u_p;
  int64_t reserved[4];
};

size_t ckpt_bytes(int64_t N, bool outer) {
  return sizeof(CkptHeader) + (size_t)N * (sizeof(double) * (outer ? 15 : 12) + 8);
}

}  // namespace

extern "C" {

int mdk_checkpoint_size(mdk_ctx *c, size_t *bytes) {
  if (check_ctx(c) || !bytes) return MDK_ERR_BAD_ARG;
  if (!c->ws || !c->state_set) return MDK_ERR_ORDER;
  DevStatus st;
  int r = read_status(c, &st);
  if (r) return r;
  *bytes = ckpt_bytes(st.N, c->sys.outer_on != 0);
  return MDK_OK;
}

int mdk_save_checkpoint(mdk_ctx *c, void *buf, size_t bytes) {
  Nvtx range("mdk_save_checkpoint");
  if (check_ctx(c) || !buf) return MDK_ERR_BAD_ARG;
  if (!c->ws || !c->state_set) return MDK_ERR_ORDER;
  DevStatus st;
  int r = read_status(c, &st);
  if (r) return r;
  const int64_t N = st.N;
  const bool outer = c->sys.outer_on != 0;
  if (bytes < ckpt_bytes(N, outer)) return MDK_ERR_BAD_ARG;
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kCkptMagic, 8);
  h.version = 1;
  h.precision = c->precision;
  h.n_rep = c->n_rep;
  const bool list = c->list_built || c->pending;
  h.flags = (list ? kCkList : 0) | (c->forces_valid && !c->pending ? kCkForces : 0) |
            (c->pending ? kCkPending : 0) | (outer ? kCkOuter : 0) |
            (outer && st.outer_valid ? kCkOuterValid : 0);
  h.N = N;
  h.steps_done = c->steps_done;
  h.n_steps = st.n_steps;
  h.n_builds = st.n_builds;
  h.n_graph_builds = st.n_graph_builds;
  h.n_full_builds = st.n_full_builds;
  h.n_inserted = st.n_inserted;
  h.n_deleted = st.n_deleted;
  h.since_build = st.since_build;
  h.next_id = st.next_id;
  h.u_p = c->u_p;
  char *o = static_cast<char *>(buf);
  memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  const Sys &s = c->sys;
  const size_t Nc = (size_t)c->N_cap;
  const double *arrs[5] = {s.x, s.v, s.f, s.xref, s.xfull};
  for (int a = 0; a < (outer ? 5 : 4); ++a)
    for (int d = 0; d < 3; ++d) {
      if (N > 0)
        MDK_CK(cudaMemcpyAsync(o, arrs[a] + d * Nc, sizeof(double) * N, cudaMemcpyDeviceToHost,
                               c->stream));
      o += sizeof(double) * N;
    }
  if (N > 0) {
    MDK_CK(cudaMemcpyAsync(o, s.id, 4 * N, cudaMemcpyDeviceToHost, c->stream));
    MDK_CK(cudaMemcpyAsync(o + 4 * N, s.info, 4 * N, cudaMemcpyDeviceToHost, c->stream));
  }
  MDK_CK(cudaStreamSynchronize(c->stream));
  return MDK_OK;
}

int mdk_load_checkpoint(mdk_ctx *c, const void *buf, size_t bytes) {
  Nvtx range("mdk_load_checkpoint");
  if (check_ctx(c) || !buf || bytes < sizeof(CkptHeader)) return MDK_ERR_BAD_ARG;
  CkptHeader h;
  memcpy(&h, buf, sizeof(h));
  if (memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1) return MDK_ERR_BAD_ARG;
  const bool outer = (h.flags & kCkOuter) != 0;
  if (h.precision != c->precision || h.n_rep != c->n_rep || h.N < 0 || h.N > c->N_cap ||
      bytes < ckpt_bytes(h.N, outer) || h.steps_done < 0 || h.n_steps < 0)
    return MDK_ERR_BAD_ARG;
  if (c->n_rep > 1 && h.N != c->N) return MDK_ERR_BAD_ARG;
  if (!c->ws_ok || c->need_ws) return MDK_ERR_WORKSPACE;
  const bool pending = (h.flags & kCkPending) != 0;
  const bool list = (h.flags & kCkList) != 0;
  if (pending && !list) return MDK_ERR_BAD_ARG;
  const int64_t N = h.N;
  const size_t Nc = (size_t)c->N_cap;
  Sys &s = c->sys;
  const char *base = static_cast<const char *>(buf) + sizeof(CkptHeader);
  auto arr = [&](int a) {  // array a (x, v, f, x_ref, x_full) of the checkpoint
    return reinterpret_cast<const double *>(base + (size_t)a * 3 * sizeof(double) * N);
  };
  const int n_arr = outer ? 5 : 4;
  const int32_t *ids = reinterpret_cast<const int32_t *>(base + (size_t)n_arr * 3 * 8 * N);
  const uint32_t *info = reinterpret_cast<const uint32_t *>(ids + N);
  // upload array a in the order ord (ord[k]: checkpoint index of internal slot k;
  // empty: the checkpoint's order) into dst
  std::vector<double> stage;
  auto upload = [&](int a, const std::vector<int64_t> &ord, double *dst) -> int {
    const double *src = arr(a);
    for (int d = 0; d < 3 && N > 0; ++d) {
      const double *col = src + (size_t)d * N;
      if (!ord.empty()) {
        stage.resize((size_t)N);
        for (int64_t k = 0; k < N; ++k) stage[(size_t)k] = col[ord[(size_t)k]];
        col = stage.data();
      }
      MDK_CK(cudaMemcpyAsync(dst + d * Nc, col, sizeof(double) * N, cudaMemcpyHostToDevice,
                             c->stream));
      if (!ord.empty()) MDK_CK(cudaStreamSynchronize(c->stream));  // stage is reused
    }
    return MDK_OK;
  };
  c->N = N;
  c->u_p = h.u_p;
  fill_sys_params(c);
  if (N > 0) {
    MDK_CK(cudaMemcpyAsync(s.id, ids, 4 * N, cudaMemcpyHostToDevice, c->stream));
    MDK_CK(cudaMemcpyAsync(s.info, info, 4 * N, cudaMemcpyHostToDevice, c->stream));
  }
  k_ckpt_begin<<<1, 32, 0, c->stream>>>(s, (int)N);
  MDK_CK(cudaPeekAtLastError());
  const std::vector<int64_t> none;
  int r = MDK_OK;
  const bool replay_outer = outer && (h.flags & kCkOuterValid) && s.outer_on;
  if (list) {
    // replay the last builds exactly: a full build at the positions it was
    // made at (x_full with two-level lists, else x_ref), then with two-level
    // lists the filter build at x_ref; cells, order and lists then equal the
    // saved run's
    r = upload(replay_outer ? 4 : 3, none, s.x);
    if (r) return r;
    launch_set_rebuild_flag(s, c->stream);
    launch_rebuild(s, 0, c->precision, 0, c->stream);
    c->launches += rebuild_chain_kernels(s) + 1;
    // the new order: internal slot k holds the atom of id new_id[k]
    std::vector<int32_t> new_id((size_t)N);
    if (N > 0)
      MDK_CK(cudaMemcpyAsync(new_id.data(), s.id, 4 * N, cudaMemcpyDeviceToHost, c->stream));
    MDK_CK(cudaStreamSynchronize(c->stream));
    std::vector<std::pair<int32_t, int64_t>> by_id((size_t)N);
    for (int64_t q = 0; q < N; ++q) by_id[(size_t)q] = {ids[q], q};
    std::sort(by_id.begin(), by_id.end());
    std::vector<int64_t> ord((size_t)N);
    for (int64_t k = 0; k < N; ++k) {
      auto it = std::lower_bound(by_id.begin(), by_id.end(),
                                 std::make_pair(new_id[(size_t)k], (int64_t)-1));
      if (it == by_id.end() || it->first != new_id[(size_t)k]) return MDK_ERR_BAD_ARG;
      ord[(size_t)k] = it->second;
    }
    if (replay_outer) {
      r = upload(3, ord, s.x);
      if (r) return r;
      launch_replay_filter(s, 0, c->precision, c->stream);
      c->launches += rebuild_chain_kernels(s);
    }
    if (!r) r = upload(0, ord, s.x);
    if (!r) r = upload(1, ord, s.v);
    if (!r) r = upload(2, ord, s.f);
    if (!r) r = upload(3, ord, s.xref);
    if (!r && replay_outer) r = upload(4, ord, s.xfull);
    if (r) return r;
    launch_regather(s, 0, c->precision, c->stream);
    c->launches += 1;
  } else {
    r = upload(0, none, s.x);
    if (!r) r = upload(1, none, s.v);
    if (!r) r = upload(2, none, s.f);
    if (r) return r;
  }
  CkptCounters k{h.n_steps, h.n_builds, h.n_graph_builds, h.n_full_builds, h.n_inserted,
                 h.n_deleted, h.since_build, h.next_id, (list && s.outer_on) ? 1 : 0};
  k_ckpt_end<<<1, 32, 0, c->stream>>>(s, k);
  MDK_CK(cudaPeekAtLastError());
  c->cur = 0;
  c->state_set = true;
  c->pending = false;
  DevStatus st;
  r = read_status(c, &st);
  if (r) return r;
  if (st.bits & kStOverflow) {  // the replayed lists outgrow this context's capacity
    note_overflow(c, st);
    c->need_ws = true;
    c->list_built = false;
    return MDK_ERR_NEIGH_OVERFLOW;
  }
  c->list_built = list;
  c->pending = pending;
  c->forces_valid = (h.flags & kCkForces) != 0 && !pending;
  c->per_atom_valid = false;
  c->steps_done = h.steps_done;
  c->steps_base = h.steps_done - (h.n_steps - (pending ? 1 : 0));
  return status_from_bits(st.bits);
}

int mdk_build_neighbors(mdk_ctx *c, double rc, double skin) {
  Nvtx range("mdk_build_neighbors");
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (!c->planned || rc != c->rc_list || skin != c->skin) {
    const int old_nmax = c->nmax, old_cells = c->n_cells;
    int r = plan(c, rc, skin, c->nmax_req, c->rebuild_every);
    if (r) return r;
    if (c->nmax > old_nmax || c->n_cells != old_cells) {
      c->need_ws = true;
      return MDK_ERR_WORKSPACE;
    }
    c->nmax = old_nmax;
    fill_sys_params(c);
  }
  int r = ensure_ready(c);
  if (r) return r;
  return build_now(c);
}

int mdk_neighbor_count(mdk_ctx *c, int64_t *total) {
  if (check_ctx(c) || !total) return MDK_ERR_BAD_ARG;
  if (!c->list_built || c->win_on || c->cfg.half == MDK_LIST_CELLS) return MDK_ERR_ORDER;
  std::vector<int32_t> nn((size_t)c->N);
  if (c->N > 0) {
    MDK_CK(cudaMemcpyAsync(nn.data(), c->sys.nnbr, sizeof(int32_t) * c->N, cudaMemcpyDeviceToHost,
                           c->stream));
    MDK_CK(cudaStreamSynchronize(c->stream));
  }
  int64_t t = 0;
  for (int32_t q : nn) t += std::min(q, c->nmax);
  *total = t;
  return MDK_OK;
}

int mdk_get_neighbors(mdk_ctx *c, int64_t *offsets, int32_t *jout, int32_t *img) {
  if (check_ctx(c) || !offsets) return MDK_ERR_BAD_ARG;
  if (!c->list_built || c->win_on || c->cfg.half == MDK_LIST_CELLS) return MDK_ERR_ORDER;
  const int64_t N = c->N;
  const size_t Nc = (size_t)c->N_cap;
  Sys &s = c->sys;
  std::vector<int32_t> nn((size_t)N), id((size_t)N);
  std::vector<uint32_t> cellc((size_t)N), info((size_t)N);
  if (N > 0) {
    MDK_CK(cudaMemcpyAsync(nn.data(), s.nnbr, 4 * N, cudaMemcpyDeviceToHost, c->stream));
    MDK_CK(cudaMemcpyAsync(id.data(), s.id, 4 * N, cudaMemcpyDeviceToHost, c->stream));
    MDK_CK(cudaMemcpyAsync(cellc.data(), s.cellc, 4 * N, cudaMemcpyDeviceToHost, c->stream));
    MDK_CK(cudaMemcpyAsync(info.data(), s.info, 4 * N, cudaMemcpyDeviceToHost, c->stream));
    MDK_CK(cudaStreamSynchronize(c->stream));
  }
  std::vector<int64_t> cnt((size_t)N, 0);
  for (int64_t i = 0; i < N; ++i) cnt[(size_t)id[(size_t)i]] = std::min(nn[(size_t)i], c->nmax);
  offsets[0] = 0;
  for (int64_t i = 0; i < N; ++i) offsets[i + 1] = offsets[i] + cnt[(size_t)i];
  if (!jout && !img) return MDK_OK;
  // copy the list groups of a chunk of atoms at a time and decode on the host
  const int64_t chunk = 1 << 16;
  std::vector<uint32_t> buf;
  for (int64_t a = 0; a < N; a += chunk) {
    const int64_t b = std::min(N, a + chunk);
    int width = 0;
    for (int64_t i = a; i < b; ++i) width = std::max(width, std::min(nn[(size_t)i], c->nmax));
    if (width == 0) continue;
    const int groups = (width + kGroup - 1) / kGroup;
    const size_t row = (size_t)(b - a) * kGroup;  // words of one group row
    buf.assign(row * groups, 0);
    MDK_CK(cudaMemcpy2DAsync(buf.data(), sizeof(uint32_t) * row, s.nbr + (size_t)a * kGroup,
                             sizeof(uint32_t) * Nc * kGroup, sizeof(uint32_t) * row, groups,
                             cudaMemcpyDeviceToHost, c->stream));
    MDK_CK(cudaStreamSynchronize(c->stream));
    for (int64_t i = a; i < b; ++i) {
      const int64_t base = offsets[id[(size_t)i]];
      const int k_n = std::min(nn[(size_t)i], c->nmax);
      const Grid &g = c->grids[info[(size_t)i] >> 8];
      for (int k = 0; k < k_n; ++k) {
        const uint32_t e = buf[(size_t)(k / kGroup) * row + (size_t)(i - a) * kGroup + k % kGroup];
        const int j = nbr_j(e);
        if (jout) jout[base + k] = id[(size_t)j];
        if (img)
          for (int d = 0; d < 3; ++d) {
            const int sd = nbr_s(e, d);
            const int cd = cell_coord(cellc[(size_t)i], d) + sd;
            int n = 0;
            if (g.per[d]) n = cd < 0 ? -1 : (cd >= g.nc[d] ? 1 : 0);
            img[3 * (base + k) + d] = n;
          }
      }
    }
  }
  return MDK_OK;
}

int mdk_compute(mdk_ctx *c, double *E, double *F, double *virial, int on_device) {
  Nvtx range("mdk_compute");
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  int r = ensure_ready(c);
  if (r) return r;
  if (!c->list_built) {
    r = build_now(c);
    if (r) return r;
  }
  Sys &s = c->sys;
  r = force_pass(c, kForceOnly, 1, 0.0);
  if (r) return r;
  c->launches += launch_reduce(s, 0, c->stream);
  MDK_CK(cudaPeekAtLastError());
  c->forces_valid = true;
  c->per_atom_valid = true;
  const int R = c->n_rep;
  if (c->win_on && F) {
    int64_t n = 0;
    r = device_n(c, &n);
    if (!r) r = gather_by_id(c, n, s.f, 3, F, on_device);
    if (r) return r;
    F = nullptr;  // written
  }
  if (on_device) {
    if (F) launch_store_forces(s, F, c->stream);
    for (int q = 0; q < R; ++q) {
      if (E) MDK_CK(cudaMemcpyAsync(E + q, s.red + 9 * q + 1, sizeof(double),
                                    cudaMemcpyDeviceToDevice, c->stream));
      if (virial) MDK_CK(cudaMemcpyAsync(virial + 6 * q, s.red + 9 * q + 2, 6 * sizeof(double),
                                         cudaMemcpyDeviceToDevice, c->stream));
    }
    MDK_CK(cudaPeekAtLastError());
    return MDK_OK;
  }
  std::vector<double> red((size_t)9 * R);
  MDK_CK(cudaMemcpyAsync(red.data(), s.red, sizeof(double) * 9 * R, cudaMemcpyDeviceToHost,
                         c->stream));
  if (F && c->N > 0) {
    launch_store_forces(s, s.tmp, c->stream);
    MDK_CK(cudaMemcpyAsync(F, s.tmp, sizeof(double) * 3 * c->N, cudaMemcpyDeviceToHost, c->stream));
  }
  DevStatus st;
  r = read_status(c, &st);
  if (r) return r;
  for (int q = 0; q < R; ++q) {
    if (E) E[q] = red[(size_t)9 * q + 1];
    if (virial)
      for (int k = 0; k < 6; ++k) virial[6 * q + k] = red[(size_t)9 * q + 2 + k];
  }
  return status_from_bits(st.bits);
}

int mdk_eam_vjp(mdk_ctx *c, const double *gE, const double *gF, double *dtheta, int on_device) {
  Nvtx range("mdk_eam_vjp");
  if (check_ctx(c) || !dtheta) return MDK_ERR_BAD_ARG;
  if (c->pot != 2 || c->win_on) return MDK_ERR_ORDER;
  int r = ensure_ready(c);
  if (r) return r;
  use_list_kind(c, MDK_LIST_FULL);  // the adjoint passes read full lists
  if (!c->list_built) {
    r = build_now(c);
    if (r) return r;
  }
  Sys &s = c->sys;
  const EAMParams &e = c->eam;
  const size_t Nc = (size_t)std::max<int64_t>(c->N_cap, 1);
  const size_t n_out = (size_t)2 * e.nr + e.nrho;
  const cudaMemcpyKind in_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (gE)
    MDK_CK(cudaMemcpyAsync(c->adj_gE, gE, sizeof(double) * c->n_rep, in_kind, c->stream));
  else
    MDK_CK(cudaMemsetAsync(c->adj_gE, 0, sizeof(double) * c->n_rep, c->stream));
  // scratch: gF in internal order [0, 4 Nc), lambda [4 Nc, 5 Nc), staged gF [6 Nc, 9 Nc)
  const double *gF_dev = (c->N > 0) ? gF : nullptr;
  if (gF && !on_device && c->N > 0) {
    MDK_CK(cudaMemcpyAsync(s.tmp + 6 * Nc, gF, sizeof(double) * 3 * c->N, cudaMemcpyHostToDevice,
                           c->stream));
    gF_dev = s.tmp + 6 * Nc;
  }
  MDK_CK(cudaMemsetAsync(c->adj_acc, 0, sizeof(double2) * n_out, c->stream));
  MDK_CK(cudaMemsetAsync(c->adj_aux, 0, sizeof(long long) * 8, c->stream));
  AdjArgs a{};
  a.cur = c->cur;
  a.gE = c->adj_gE;
  a.gint = s.tmp;
  a.lam = s.tmp + 4 * Nc;
  a.acc_phi = reinterpret_cast<longlong2 *>(c->adj_acc);
  a.acc_rho = reinterpret_cast<longlong2 *>(c->adj_acc + e.nr);
  a.acc_F = c->adj_acc + 2 * e.nr;
  a.aux = c->adj_aux;
  a.out = on_device ? dtheta : c->adj_out;
  launch_eam_rho(s, e, c->precision, StepArgs{0.0, c->cur, 0, 0.0f}, c->cfg, c->stream);
  if (launch_eam_adjoint(s, e, c->precision, gF_dev, a, c->N, c->stream)) return MDK_ERR_CUDA;
  c->launches += 6;
  MDK_CK(cudaPeekAtLastError());
  if (on_device) return MDK_OK;
  MDK_CK(cudaMemcpyAsync(dtheta, c->adj_out, sizeof(double) * n_out, cudaMemcpyDeviceToHost,
                         c->stream));
  DevStatus st;
  r = read_status(c, &st);
  if (r) return r;
  return status_from_bits(st.bits);
}

int mdk_get_per_atom(mdk_ctx *c, double *Ui, double *Wi) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (!c->per_atom_valid) return MDK_ERR_ORDER;
  Sys &s = c->sys;
  if (c->win_on) {
    int64_t n = 0;
    int r = device_n(c, &n);
    if (!r && Ui) r = gather_by_id(c, n, s.ea, 1, Ui, 0);
    if (!r && Wi) r = gather_by_id(c, n, s.wa, 6, Wi, 0);
    return r;
  }
  if (c->N == 0) return MDK_OK;
  double *stage = s.tmp;
  launch_store_per_atom(s, Ui ? stage : nullptr, Wi ? stage + c->N : nullptr, c->stream);
  if (Ui) MDK_CK(cudaMemcpyAsync(Ui, stage, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
  if (Wi)
    MDK_CK(cudaMemcpyAsync(Wi, stage + c->N, sizeof(double) * 6 * c->N, cudaMemcpyDeviceToHost,
                           c->stream));
  MDK_CK(cudaStreamSynchronize(c->stream));
  return MDK_OK;
}

int mdk_step(mdk_ctx *c, double dt, int64_t nsteps) {
  Nvtx range("mdk_step");
  if (check_ctx(c) || nsteps < 0 || !(dt > 0.0)) return MDK_ERR_BAD_ARG;
  int r = ensure_ready(c);
  if (r) return r;
  if (nsteps == 0) return MDK_OK;
  if ((c->lang_n > 0 || c->lang_rep_on) && dt != c->lang_dt) {  // amplitudes depend on dt
    c->lang_dt = dt;
    fill_sys_params(c);
    r = upload_lang_rep(c);
    if (r) return r;
  }
  if (!c->list_built) {
    r = build_now(c);
    if (r) return r;
  }
  Sys &s = c->sys;
  if (c->pending) {
    // a restored mid-step state: its first half-kick, drift and list build
    // are done; the steps start with the pending force pass
    c->pending = false;
  } else {
    if (!c->forces_valid) {
      r = force_pass(c, kForceOnly, 0, dt);
      if (r) return r;
    }
    // the force passes of the mixed full-list LJ and EAM kernels end a step
    // with FP32 forces; half lists and BPNN with FP64 sums
    const int f32 = c->precision == MDK_MIXED && (c->pot == 1 || c->pot == 2) && c->cfg.half != 1;
    StepArgs a{dt, c->cur, 0, (float)(0.5 * dt), f32};
    r = timed(c, c->ev_kick, 1, [&] { launch_kick_drift(s, c->precision, a, c->stream); });
    if (r) return r;
    c->cur ^= 1;
    r = rebuild_chain(c, 1);
    if (r) return r;
  }
  const uint64_t key = c->graphs_on ? graph_key(c, dt) : 0;
  auto is_thermo = [&](int64_t q) {
    return c->thermo_every > 0 && ((c->steps_done + q) % c->thermo_every) == 0;
  };
  for (int64_t q = 1; q <= nsteps; ++q) {
    // two plain steps (neither the last nor a thermo step) run as one graph
    if (c->graphs_on && !c->prof && q + 1 < nsteps && !is_thermo(q) && !is_thermo(q + 1)) {
      const int par = c->cur;
      if (!c->gexec[par] || c->gkey[par] != key) {
        r = capture_two_steps(c, par, dt, key);
        if (r) return r;
      }
      MDK_CK(cudaGraphLaunch(c->gexec[par], c->stream));
      c->launches += c->graph_kernels;
      ++q;  // the graph ran steps q and q + 1; the parity is back to par
      continue;
    }
    const int64_t gstep = c->steps_done + q;
    const int thermo = is_thermo(q);
    const bool last = q == nsteps;
    r = force_pass(c, last ? kFinal : kStep, thermo, dt);
    if (r) return r;
    if (thermo) {
      c->launches += launch_reduce(s, 1, c->stream) + 1;
      const int slot = (int)(c->thermo_written % std::max(c->thermo_cap, 1));
      k_thermo_store<<<1, std::max(32, ((c->n_rep + 31) / 32) * 32), 0, c->stream>>>(
          s, c->thermo_ring, slot, (double)gstep);
      c->thermo_written++;
    }
    if (!last) {
      c->cur ^= 1;
      r = rebuild_chain(c, 1);
      if (r) return r;
    }
  }
  MDK_CK(cudaPeekAtLastError());
  c->steps_done += nsteps;
  c->forces_valid = true;
  c->per_atom_valid = false;
  return MDK_OK;
}

int mdk_set_thermo(mdk_ctx *c, int every, int capacity) {
  if (check_ctx(c) || every < 0 || capacity < 0) return MDK_ERR_BAD_ARG;
  if (capacity > c->thermo_cap) c->ws_ok = false;  // ring lives in the workspace
  c->thermo_every = every;
  c->thermo_cap = std::max(capacity, c->thermo_cap);
  c->thermo_written = c->thermo_read = 0;
  return c->ws_ok ? MDK_OK : MDK_ERR_WORKSPACE;
}

int mdk_set_outer_skin(mdk_ctx *c, double skin_outer) {
  if (check_ctx(c) || !(skin_outer >= 0.0) || !std::isfinite(skin_outer)) return MDK_ERR_BAD_ARG;
  if (!c->planned) return MDK_ERR_ORDER;
  if (skin_outer != 0.0 && !(skin_outer > c->skin)) return MDK_ERR_BAD_ARG;
  // the pre-filter band (1e-4 of r^2) holds FP32 offsets of cells up to
  // ~100 r_ns; refuse outer cells beyond a tenth of that
  if (skin_outer > 10.0 * (c->rc_list + c->skin)) return MDK_ERR_BAD_ARG;
  const int old_nmax = c->nmax, old_cells = c->n_cells, old_nmax1 = c->nmax1;
  const double keep = c->skin_outer;
  c->skin_outer = skin_outer;
  c->nmax1_grow = 0;
  const int r = plan(c, c->rc_list, c->skin, c->nmax_req, c->rebuild_every);
  if (r) {
    c->skin_outer = keep;
    plan(c, c->rc_list, c->skin, c->nmax_req, c->rebuild_every);
    return r;
  }
  if (c->nmax != old_nmax || c->n_cells != old_cells || c->nmax1 != old_nmax1) c->need_ws = true;
  c->list_built = false;
  return MDK_OK;
}

int mdk_get_build_counts(mdk_ctx *c, int64_t *n_builds, int64_t *n_full) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (!c->ws_ok) return MDK_ERR_WORKSPACE;
  DevStatus st;
  int r = read_status(c, &st);
  if (r) return r;
  if (n_builds) *n_builds = st.n_builds;
  if (n_full) *n_full = c->nmax1 > 0 ? st.n_full_builds : st.n_builds;
  return MDK_OK;
}

int mdk_get_thermo(mdk_ctx *c, double *out, int max_samples, int *n_out) {
  if (check_ctx(c) || !n_out) return MDK_ERR_BAD_ARG;
  *n_out = 0;
  if (!c->ws_ok) return MDK_ERR_WORKSPACE;
  const int cap = std::max(c->thermo_cap, 1);
  int64_t first = std::max(c->thermo_read, c->thermo_written - cap);
  const int per = c->n_rep * 10;
  std::vector<double> ring((size_t)cap * per);
  MDK_CK(cudaMemcpyAsync(ring.data(), c->thermo_ring, sizeof(double) * ring.size(),
                         cudaMemcpyDeviceToHost, c->stream));
  MDK_CK(cudaStreamSynchronize(c->stream));
  int n = 0;
  int64_t q = first;
  for (; q < c->thermo_written && n < max_samples; ++q) {
    const double *smp = ring.data() + (size_t)(q % cap) * per;
    if (std::isnan(smp[0])) continue;  // a step that stepping did not reach
    memcpy(out + (size_t)n * per, smp, sizeof(double) * per);
    ++n;
  }
  c->thermo_read = q;
  *n_out = n;
  return MDK_OK;
}

int mdk_get_counters(mdk_ctx *c, int64_t *n_builds, int64_t *n_steps) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (!c->ws_ok) return MDK_ERR_WORKSPACE;
  DevStatus st;
  int r = read_status(c, &st);
  if (r) return r;
  if (n_builds) *n_builds = st.n_builds;
  if (n_steps) *n_steps = c->steps_done;
  return MDK_OK;
}

int mdk_last_device_status(mdk_ctx *c, int *bits) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (!c->ws_ok) return MDK_ERR_WORKSPACE;
  DevStatus st;
  int r = read_status(c, &st);
  if (r) return r;
  if (bits) *bits = (int)st.bits;
  if (st.bits & kStOverflow) {
    note_overflow(c, st);
    c->need_ws = true;
    c->list_built = false;
  }
  k_clear_bits<<<1, 32, 0, c->stream>>>(c->sys);
  MDK_CK(cudaPeekAtLastError());
  return status_from_bits(st.bits);
}

int mdk_set_piston(mdk_ctx *c, double u_p, const uint8_t *is_piston) {
  if (check_ctx(c) || !isfinite(u_p)) return MDK_ERR_BAD_ARG;
  if (!c->ws_ok || !c->state_set) return MDK_ERR_ORDER;
  if (c->win_on) return MDK_ERR_ORDER;  // ids are no longer 0..N-1
  c->u_p = u_p;
  c->sys.u_p = u_p;
  // the host copy of the info words keeps the flags across a new workspace
  for (int64_t q = 0; q < c->N; ++q)
    c->info0[(size_t)q] = (c->info0[(size_t)q] & ~kInfoPiston) |
                          ((is_piston && is_piston[q]) ? kInfoPiston : 0u);
  const uint8_t *dflags = nullptr;
  if (is_piston && c->N > 0) {
    uint8_t *stage = reinterpret_cast<uint8_t *>(c->sys.tmp);
    MDK_CK(cudaMemcpyAsync(stage, is_piston, (size_t)c->N, cudaMemcpyHostToDevice, c->stream));
    dflags = stage;
  }
  launch_set_piston(c->sys, dflags, c->N, c->stream);
  MDK_CK(cudaPeekAtLastError());
  MDK_CK(cudaStreamSynchronize(c->stream));
  // the gather copies carry the info word: regenerate them with a rebuild
  if (c->list_built) return build_now(c);
  return MDK_OK;
}

int mdk_autotune(mdk_ctx *c, int reps, int *tpa_out, int *block_out, double *ms_out) {
  Nvtx range("mdk_autotune");
  if (check_ctx(c) || reps < 0) return MDK_ERR_BAD_ARG;
  int r = ensure_ready(c);
  if (r) return r;
  if (!c->list_built) {
    r = build_now(c);
    if (r) return r;
  }
  if (reps == 0) reps = 3;
  cudaEvent_t e0, e1;
  MDK_CK(cudaEventCreate(&e0));
  MDK_CK(cudaEventCreate(&e1));
  const LaunchCfg keep = c->cfg;
  const bool prof = c->prof;
  c->prof = false;
  LaunchCfg best = keep;
  float best_ms = -1.f;
  static const int kTpa[5] = {1, 2, 4, 8, 32};  // 32: a warp per atom
  static const int kBlock[3] = {128, 256, 512};
  // LJ and EAM: full lists in every shape, then half lists (one thread per
  // atom); LJ also the list-free cell kernel (one warp per cell)
  const int n_kinds = c->pot == 1 ? 3 : (c->pot == 2 ? 2 : 1);
  for (int kind = 0; kind < n_kinds && !r; ++kind)
  for (int a = 0; a < 5 && !r; ++a)
    for (int b = 0; b < 3; ++b) {
      if (c->pot == 1 && kBlock[b] > 256) continue;  // the LJ kernels take <= 256
      if (c->pot == 3 && (a > 0 || b > 0)) continue;  // BPNN: one warp per atom, one shape
      if (kind >= 1 && (kTpa[a] != 1 || kBlock[b] > 256)) continue;  // <= 256 threads
      if (c->cfg.half != kind || !c->list_built) {
        use_list_kind(c, kind);
        r = build_now(c);
        if (r) break;
      }
      c->cfg.tpa = kTpa[a];
      c->cfg.block = kBlock[b];
      r = force_pass(c, kForceOnly, 0, 0.0);  // warm-up (and grid set-up)
      if (r) break;
      MDK_CK(cudaEventRecord(e0, c->stream));
      for (int q = 0; q < reps && !r; ++q) r = force_pass(c, kForceOnly, 0, 0.0);
      MDK_CK(cudaEventRecord(e1, c->stream));
      MDK_CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      MDK_CK(cudaEventElapsedTime(&ms, e0, e1));
      ms /= (float)reps;
      if (best_ms < 0.f || ms < best_ms) {
        best_ms = ms;
        best = c->cfg;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->prof = prof;
  if (!r && best.half != c->cfg.half) {
    use_list_kind(c, best.half);
    r = build_now(c);
  }
  if (r) {
    use_list_kind(c, keep.half);
    c->cfg = keep;
    return r;
  }
  c->cfg = best;
  c->forces_valid = true;  // the passes left the forces of the current positions
  c->per_atom_valid = false;
  if (tpa_out) *tpa_out = best.tpa;
  if (block_out) *block_out = best.block;
  if (ms_out) *ms_out = best_ms;
  return MDK_OK;
}

int mdk_set_graphs(mdk_ctx *c, int enable) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  c->graphs_on = enable != 0;
  return MDK_OK;
}

int mdk_set_launch(mdk_ctx *c, int tpa, int block) {
  if (check_ctx(c) || (tpa != 1 && tpa != 2 && tpa != 4 && tpa != 8 && tpa != 32) ||
      (block != 128 && block != 256 && block != 512))
    return MDK_ERR_BAD_ARG;
  c->cfg.tpa = tpa;
  c->cfg.block = block;
  return MDK_OK;
}

int mdk_set_list_kind(mdk_ctx *c, int kind) {
  if (check_ctx(c) || (kind != MDK_LIST_FULL && kind != MDK_LIST_HALF && kind != MDK_LIST_CELLS))
    return MDK_ERR_BAD_ARG;
  if (kind == MDK_LIST_HALF && c->pot != 1 && c->pot != 2)
    return c->pot == 0 ? MDK_ERR_ORDER : MDK_ERR_BAD_ARG;
  if (kind == MDK_LIST_CELLS && c->pot != 1) return c->pot == 0 ? MDK_ERR_ORDER : MDK_ERR_BAD_ARG;
  use_list_kind(c, kind);
  return MDK_OK;
}

int mdk_get_list_kind(const mdk_ctx *c, int *kind) {
  if (check_ctx(c) || !kind) return MDK_ERR_BAD_ARG;
  *kind = c->cfg.half;
  return MDK_OK;
}

int mdk_profile(mdk_ctx *c, int enable) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (c->ws_ok) {
    DevStatus st;
    int r = read_status(c, &st);
    if (r) return r;
    c->graph_builds0 = st.n_graph_builds;
  }
  c->prof = enable != 0;
  c->ev_used = 0;
  c->ev_force.clear();
  c->ev_chain.clear();
  c->ev_kick.clear();
  c->launches = 0;
  return MDK_OK;
}

int mdk_get_profile(mdk_ctx *c, double *out) {
  if (check_ctx(c) || !out) return MDK_ERR_BAD_ARG;
  if (!c->ws_ok) return MDK_ERR_WORKSPACE;
  DevStatus st;
  int r = read_status(c, &st);
  if (r) return r;
  auto total = [&](const std::vector<std::pair<int, int>> &v) {
    double ms = 0.0;
    for (const auto &p : v) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, c->ev_pool[(size_t)p.first], c->ev_pool[(size_t)p.second]) ==
          cudaSuccess)
        ms += t;
    }
    return ms;
  };
  out[0] = total(c->ev_force);
  out[1] = (double)c->ev_force.size();
  out[2] = total(c->ev_chain);
  out[3] = (double)c->ev_chain.size();
  // kernels launched: those enqueued directly, those of every graph replay,
  // and the rebuild bodies that the graphs' conditional nodes ran
  out[4] = (double)c->launches + (double)c->body_kernels * (double)(st.n_graph_builds -
                                                                     c->graph_builds0);
  out[5] = (double)st.n_builds;
  out[6] = total(c->ev_kick);
  out[7] = (double)c->ev_kick.size();
  return MDK_OK;
}

int mdk_set_window(mdk_ctx *c, double L_behind, double L_ahead, const double *slab_x,
                   const double *slab_v, int64_t n_slab, double slab_lx, double slab_gap,
                   double slab_mass, double piston_depth, double front_bin,
                   double fixed_front) {
  if (check_ctx(c) || c->n_rep != 1 || !slab_x || !slab_v || n_slab < 1 ||
      n_slab >= ((int64_t)1 << 26) || !(slab_lx > 0.0) || !(L_behind >= 0.0) ||
      !(L_ahead >= 0.0) || !isfinite(slab_gap) || !(slab_mass > 0.0) || !(piston_depth >= 0.0) ||
      !(front_bin > 0.0) || c->per[0])
    return MDK_ERR_BAD_ARG;
  const double nb = ceil((c->hi[0] - c->lo[0]) / front_bin);
  if (!(nb <= (double)(1 << 24))) return MDK_ERR_BAD_ARG;
  int t = 0;
  while (t < c->n_types && c->type_mass[t] != slab_mass) ++t;
  if (t == c->n_types) {
    if (c->n_types == kMaxTypes) return MDK_ERR_BAD_ARG;
    c->type_mass[c->n_types++] = slab_mass;
  }
  c->win_on = true;
  c->win_L_behind = L_behind;
  c->win_L_ahead = L_ahead;
  c->win_slab_lx = slab_lx;
  c->win_gap = slab_gap;
  c->win_depth = piston_depth;
  c->win_info = (uint32_t)t;
  c->win_front_bin = front_bin;
  c->win_fixed_front = fixed_front;
  c->win_nbins = std::max(1, (int)nb);
  c->win_slab.assign((size_t)n_slab * 6, 0.0);
  for (int64_t q = 0; q < n_slab; ++q)
    for (int k = 0; k < 3; ++k) {
      c->win_slab[(size_t)q * 6 + k] = slab_x[3 * q + k];
      c->win_slab[(size_t)q * 6 + 3 + k] = slab_v[3 * q + k];
    }
  if (!c->ws_ok) return MDK_OK;
  if (n_slab > c->win_slab_cap || c->win_nbins > c->win_nbins_cap) {
    c->need_ws = true;  // the slab or bin area of the workspace is too small
    return MDK_ERR_WORKSPACE;
  }
  MDK_CK(cudaMemsetAsync(c->win_fbin, 0, sizeof(long long) * 2 * c->win_nbins, c->stream));
  MDK_CK(cudaMemcpyAsync(c->win_slab_dev, c->win_slab.data(), sizeof(double) * c->win_slab.size(),
                         cudaMemcpyHostToDevice, c->stream));
  fill_sys_params(c);
  MDK_CK(cudaStreamSynchronize(c->stream));
  return MDK_OK;
}

int mdk_set_langevin(mdk_ctx *c, int n_regions, const double *x_lo, const double *x_hi,
                     const double *T, const double *u, const double *beta, uint64_t seed) {
  if (check_ctx(c) || n_regions < 0 || n_regions > kMaxLang) return MDK_ERR_BAD_ARG;
  if (n_regions > 0 && (!x_lo || !x_hi || !T || !u || !beta)) return MDK_ERR_BAD_ARG;
  for (int q = 0; q < n_regions; ++q)
    if (!(x_lo[q] < x_hi[q]) || !(T[q] >= 0.0) || !(beta[q] >= 0.0) ||
        !(isfinite(u[3 * q]) && isfinite(u[3 * q + 1]) && isfinite(u[3 * q + 2])))
      return MDK_ERR_BAD_ARG;
  const double kB = 8.617333262e-5;  // eV/K
  c->lang_n = n_regions;
  for (int q = 0; q < kMaxLang; ++q) {
    const bool on = q < n_regions;
    c->lang_xlo[q] = on ? x_lo[q] : 0.0;
    c->lang_xhi[q] = on ? x_hi[q] : 0.0;
    c->lang_kT[q] = on ? kB * T[q] : 0.0;
    c->lang_beta[q] = on ? beta[q] : 0.0;
    for (int d = 0; d < 3; ++d) c->lang_u[q][d] = on ? u[3 * q + d] : 0.0;
  }
  c->lang_seed = seed;
  if (c->ws_ok) fill_sys_params(c);
  return MDK_OK;
}

int mdk_set_langevin_replicas(mdk_ctx *c, const double *T, const double *beta, uint64_t seed) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (!T) {  // off
    c->lang_rep_on = false;
    if (c->ws_ok) fill_sys_params(c);
    return MDK_OK;
  }
  if (!beta) return MDK_ERR_BAD_ARG;
  for (int r = 0; r < c->n_rep; ++r)
    if (!(T[r] >= 0.0) || !(beta[r] >= 0.0)) return MDK_ERR_BAD_ARG;
  c->lang_rep_T.assign(T, T + c->n_rep);
  c->lang_rep_beta.assign(beta, beta + c->n_rep);
  c->lang_rep_on = true;
  c->lang_seed = seed;
  if (c->ws_ok) {
    fill_sys_params(c);
    return upload_lang_rep(c);
  }
  return MDK_OK;
}

int mdk_get_ids(mdk_ctx *c, int64_t *ids) {
  if (check_ctx(c) || !ids) return MDK_ERR_BAD_ARG;
  if (!c->ws_ok || !c->state_set) return MDK_ERR_ORDER;
  int64_t n = 0;
  int r = device_n(c, &n);
  if (r) return r;
  std::vector<int32_t> ord, id;
  r = caller_order(c, n, ord, id);
  if (r) return r;
  for (int64_t q = 0; q < n; ++q) ids[q] = id[(size_t)ord[(size_t)q]];
  return MDK_OK;
}

int mdk_window_counts(mdk_ctx *c, int64_t *inserted, int64_t *deleted) {
  if (check_ctx(c)) return MDK_ERR_BAD_ARG;
  if (!c->ws_ok) return MDK_ERR_WORKSPACE;
  DevStatus st;
  int r = read_status(c, &st);
  if (r) return r;
  if (inserted) *inserted = st.n_inserted;
  if (deleted) *deleted = st.n_deleted;
  return MDK_OK;
}

int mdk_profiles(mdk_ctx *c, int axis, double origin, double bin_w, int nbins,
                 double cross_area, double *out, int on_device) {
  Nvtx range("mdk_profiles");
  if (check_ctx(c) || axis < 0 || axis > 2 || !(bin_w > 0.0) || nbins < 1 || !out ||
      !(cross_area > 0.0))
    return MDK_ERR_BAD_ARG;
  // accumulators live in the sort scratch (9 N_cap doubles)
  if ((size_t)nbins * (kProfWidth + kProfOut) > 9 * (size_t)std::max<int64_t>(c->N_cap, 1))
    return MDK_ERR_BAD_ARG;
  int r = ensure_ready(c);
  if (r) return r;
  if (!c->list_built) {
    r = build_now(c);
    if (r) return r;
  }
  // per-atom energies and virials at the current positions
  if (!c->per_atom_valid) {
    r = force_pass(c, kForceOnly, 1, 0.0);
    if (r) return r;
    c->forces_valid = true;
    c->per_atom_valid = true;
  }
  double *acc = c->sys.tmp;
  launch_profiles(c->sys, axis, origin, bin_w, nbins, cross_area, acc, c->stream);
  c->launches += 5;
  MDK_CK(cudaPeekAtLastError());
  acc += (size_t)nbins * kProfWidth;  // the outputs follow the accumulators
  const size_t bytes = sizeof(double) * kProfOut * nbins;
  if (on_device) {
    MDK_CK(cudaMemcpyAsync(out, acc, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return MDK_OK;
  }
  MDK_CK(cudaMemcpyAsync(out, acc, bytes, cudaMemcpyDeviceToHost, c->stream));
  MDK_CK(cudaStreamSynchronize(c->stream));
  return MDK_OK;
}

}  // extern "C"
