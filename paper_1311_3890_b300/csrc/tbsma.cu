// Host side of the TB-SMA wire MD library: the C ABI of include/tbsma.h.
//
// One context holds a ragged batch of wires packed atom-wise.  Every kernel
// runs over the flat atom array (pair, integrator) or over per-wire work
// lists (neighbour build, reductions), so a batch of thousands of wires of
// uneven size costs the same launches as a single wire.  The step loop is
// captured once per (dt, chunk) as a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/tbsma.h"
#include "device.cuh"
#include "md.cuh"
#include "nlist.cuh"
#include "pair.cuh"
#include "topo.cuh"
#include "persist.cuh"

using namespace tbsma;

namespace {

constexpr int kGraphChunk = 50;  // steps per captured graph
constexpr int64_t kGrowCheckSteps = 1000;  // steps between cell-grid checks inside one step call
static_assert(kGrowCheckSteps % kGraphChunk == 0, "grid checks fall on kick-sequence boundaries");

// An NVTX range over one library call, for timeline tools (nsys): the
// header-only NVTX3 API does nothing unless a tool is attached.  Inside the
// step graphs the kernels' own names mark the phases.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
constexpr int kMinCap = 64;   // neighbour-list row length, bounds (list_capacity)
constexpr int kMaxCap = 128;
constexpr int kMaxWindow = 4096; // largest shared-memory window of a pair-pass tile, atoms
constexpr int kMaxEamSamples = 1 << 22;  // samples per EAM table
// Largest disorder of a wire's atom order along the axis (max over atoms of
// the prefix max minus the suffix min of x, A) for which it takes the slab
// build: each A of disorder widens every slab by about a plane's worth of
// atoms at each end; beyond this the cell build is cheaper.
constexpr float kSlabDisorder = 4.0f;

struct Graph {
  cudaGraphExec_t exec = nullptr;
  int steps = 0;
};

}  // namespace

struct tbsma_ctx {
  tbsma_params P{};
  int prec = TBSMA_MIXED;
  int W = 0;
  int64_t N = 0;
  int64_t NS = 0;  // slots of the pair passes: every wire's atoms padded to whole tiles
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int sm_count = 148;
  int block = 256;   // atoms per tile of the pair passes
  int wcap = 1280;   // shared-memory window of a tile, atoms
  int cap = kMinCap;
  int64_t n_cells = 0;
  int64_t steps_done = 0;
  double dt_dyn = -1.0;  // dt the per-wire dynamic table was filled for
  std::string err;

  // caller-owned
  double* x = nullptr;
  double* v = nullptr;
  const uint8_t* kind = nullptr;

  // library-owned device memory
  std::vector<void*> allocs;
  WireDev* wd = nullptr;
  WireDyn* wdyn = nullptr;
  uint32_t* meta = nullptr;
  int4* xq = nullptr;
  int4* xq_b = nullptr;
  double4_32a* xd = nullptr;
  double4_32a* xd_b = nullptr;
  float* f32 = nullptr;
  double* f64 = nullptr;
  double* inv64 = nullptr;
  double* e_band = nullptr;
  double* e_atom = nullptr;
  double* w_atom = nullptr;
  double* s_atom = nullptr;
  int16_t* nbr = nullptr;
  int32_t* n_nbr = nullptr;
  int2* jrange = nullptr;
  int32_t* cell_count = nullptr;
  int32_t* cell_atoms = nullptr;
  int32_t* cell_of = nullptr;
  int32_t* perm = nullptr;     // slot -> atom of the pair passes (-1: a tile's padding slot)
  int32_t* slot_of = nullptr;  // atom -> slot
  int32_t* flag = nullptr;
  int32_t* wl_wire = nullptr;
  int64_t* wl_cell = nullptr;
  int64_t* wl_atom = nullptr;
  int64_t* wl_tile = nullptr;
  int32_t* cl_wire = nullptr;   // flagged wires that take the cell build (see NlWork)
  int64_t* cl_cell = nullptr;
  int64_t* cl_atom = nullptr;
  int32_t* n_cell = nullptr;
  uint32_t* merge_done = nullptr;
  int4* xq2 = nullptr;         // second position buffer of the persistent step kernel
  float2* xenv = nullptr;      // per atom: prefix max / suffix min of x (slab-build envelopes)
  float2* tenv = nullptr;      // per tile: max / min of x (slab-build envelopes)
  uint32_t* wdis = nullptr;    // per wire: disorder of the atom order along x (FP32 bits)
  float4* xf = nullptr;        // per group of four slots: FP32 x, y, z (slab-build candidates)
  int32_t* n_flagged = nullptr;
  int32_t* n_rebuilds = nullptr;
  int64_t* chains = nullptr;  // launches of the rebuild chain (launch accounting)
  int64_t* rebuilt = nullptr;  // [2] wires and atoms whose lists were built (accumulated)
  tbsma_wire* wires_d = nullptr;  // the wire table of tbsma_init (per-wire bounding boxes)
  double* bbox_d = nullptr;       // [W][7] bounding boxes and mobile counts (k_bbox)
  int64_t cells_alloc = 0;        // capacity of cell_count / cell_atoms, cells
  double cell_edge = 0.0;         // smallest cell edge of the grids (list radius + guard), A
  std::vector<cudaEvent_t> prof_ev;  // event pool of tbsma_step_profile
  int64_t* last_build = nullptr;  // per wire: step of its last list build
  uint8_t* banked = nullptr;      // per wire: rows in bank-group order at its last build
  uint32_t* wire_status = nullptr;
  NhState* nh = nullptr;            // per-wire Nosé–Hoover state
  BaroState* baro = nullptr;        // per-wire axial barostat state
  int* uf_parent = nullptr;         // union-find of the topology call (allocated on first use)
  uint32_t* uf_err = nullptr;
  tbsma_topology* topo_d = nullptr;
  int wait_limit = kUfSteps;        // bound of the topology's union-find walks and barrier waits
  int step_mode = TBSMA_STEPS_AUTO;  // graph replays or the persistent step kernel
  int lanes = 1;  // threads per atom in the MIXED pair passes: 1 or 4
  unsigned* bar = nullptr;           // [3] persistent kernel barrier: 64-bit arrival count, error word
  tbsma_protocol proto{};           // paper protocol mode (default: Langevin, continuous pull)
  double* d_grip = nullptr;
  int64_t* step_counter = nullptr;
  tbsma_obs* obs_d = nullptr;
  tbsma_fcheck* fcheck_d = nullptr;
  double* fc_part = nullptr;  // [NS / 256][5] per-tile partials of the force check

  std::vector<WireDev> wires_h;
  Graph graph;
  cudaGraphExec_t obs_graph = nullptr;  // a report's re-pack, rebuild and passes (launch_captured)
  // tbsma_step_observe's last kick sequence: the step graph with the
  // per-atom energy terms in its last step's passes
  cudaGraphExec_t seq_obs_graph = nullptr;
  int seq_obs_steps = 0;
  double seq_obs_dt = -1.0;
  cudaGraphExec_t fc_graph = nullptr;   // the force check's
  double graph_dt = -1.0;

  PairConsts pc{};
  bool eam_on = false;           // tabulated EAM instead of Eq. 1-3 (tbsma_set_eam)
  EamDev eam{};
  std::vector<void*> eam_allocs;  // the EAM tables (replaced by every tbsma_set_eam)
  float rlist2 = 0.f;   // list radius squared, A^2
  float rlist2u = 0.f;  // the same in fixed-point units squared (x 2^52, exact)
  float slab_range = 0.f;  // list radius plus the envelope guard, A (slab build)
  double half_skin2 = 0.0;
  double inv_m = 0.0;

  NlWork nw() const {
    NlWork w;
    w.flag = flag;
    w.wl_wire = wl_wire;
    w.wl_cell = wl_cell;
    w.wl_atom = wl_atom;
    w.wl_tile = wl_tile;
    w.xenv = xenv;
    w.tenv = tenv;
    w.wdis = wdis;
    w.xf = xf;
    w.N = N;
    w.slab_ok = prec == TBSMA_MIXED ? 1 : 0;
    w.max_disorder = kSlabDisorder;
    w.n_flagged = n_flagged;
    w.n_rebuilds = n_rebuilds;
    w.chains = chains;
    w.last_build = last_build;
    w.banked = banked;
    w.rebuilt = rebuilt;
    w.cl_wire = cl_wire;
    w.cl_cell = cl_cell;
    w.cl_atom = cl_atom;
    w.n_cell = n_cell;
    w.merge_done = merge_done;
    return w;
  }
};

namespace {

tbsma_status fail(tbsma_ctx* c, tbsma_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

tbsma_status cuda_fail(tbsma_ctx* c, cudaError_t e, const char* where) {
  if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? TBSMA_ENOMEM : TBSMA_ECUDA;
}

#define TB_CUDA(c, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
  } while (0)

template <typename T>
tbsma_status alloc(tbsma_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return TBSMA_OK;
}

#define TB_TRY(expr)                      \
  do {                                    \
    tbsma_status s_ = (expr);             \
    if (s_ != TBSMA_OK) return s_;        \
  } while (0)

inline unsigned grid_for(int64_t threads, int block) {
  return (unsigned)std::max<int64_t>(1, (threads + block - 1) / block);
}

// Cell grid of one wire around its bounding box lo[3], hi[3] (absolute A),
// the fixed-point origin d.origin already set: cell edge >= rl (the list
// radius with a guard), across the axis a margin of rl, along it half the
// wire's extent plus rl at each end (room to double its length before an
// atom leaves the grid).  False if an axis would need more than 1023 cells.
bool plan_grid(WireDev& d, const double* lo, const double* hi, double rl) {
  for (int k = 0; k < 3; ++k) {
    const double margin = (k == 0 ? 0.5 * (hi[k] - lo[k]) : 0.0) + rl;
    const double glo = lo[k] - d.origin[k] - margin, ghi = hi[k] - d.origin[k] + margin;
    const double cells = std::floor((ghi - glo) / rl);
    if (!(cells <= 1023.0)) return false;
    const int n = std::max(1, (int)cells);
    d.glo[k] = glo;
    d.einv[k] = n / (ghi - glo);
    d.nc[k] = n;
  }
  return true;
}

void fill_pair_consts(tbsma_ctx* c) {
  const tbsma_params& P = c->P;
  const double log2e = 1.4426950408889634073599246810019;
  PairConsts& k = c->pc;
  k.rc2f = (float)(P.r_cut * P.r_cut) * 4503599627370496.0f;  // x 2^52: fixed-point units^2
  const double unit = 1.0 / 67108864.0;  // 2^-26 A
  k.gA = (float)(-2.0 * P.q / P.r0 * log2e * unit);
  const double gB = -(double)k.gA * P.r0 / unit;
  k.gB = (float)gB;
  k.xi2g = (float)(P.xi * P.xi * std::exp2(gB - (double)k.gB));
  k.fgf = (float)(2.0 * P.q * P.xi * P.xi / P.r0);
  k.r0f = (float)P.r0;
  k.kgf = (float)(2.0 * P.q / P.r0 * log2e);
  k.khf = (float)((P.p - 2.0 * P.q) / P.r0 * log2e);
  k.fpf = (float)(2.0 * P.p * P.A / P.r0);
  k.Af = (float)P.A;
  k.rc2 = P.r_cut * P.r_cut;
  k.r0 = P.r0;
  k.A = P.A;
  k.xi2 = P.xi * P.xi;
  k.p = P.p;
  k.q = P.q;
  k.fp = 2.0 * P.p / P.r0;
  k.fg = 2.0 * P.q / P.r0;
  k.inv_r0 = 1.0 / P.r0;
  // list radius with a 1e-3 A guard so rounding in the build or in the
  // displacement check can never drop a pair that reaches r_cut
  const double rl = P.r_cut + P.r_skin + 1e-3;
  c->rlist2 = (float)(rl * rl);
  c->rlist2u = c->rlist2 * 4503599627370496.0f;  // x 2^52
  c->slab_range = (float)rl + kSlabGuard;
  c->half_skin2 = 0.25 * P.r_skin * P.r_skin;
  c->inv_m = 1.0 / (P.mass * kMvv2e);
  // List row length: the fcc sites (density sqrt(2)/r0^3 for nearest-neighbour
  // distance r0) in a sphere of the list radius, times 1.25 for thermal and
  // surface disorder, rounded up to 8 and kept within [kMinCap, kMaxCap].  A
  // bulk Au atom has 54 sites within 5.8 A and 24 more at 6.45 A, which
  // thermal motion brings inside a list radius of 6.2 A at 298 K.
  const double sites = std::sqrt(2.0) / (P.r0 * P.r0 * P.r0) * 4.0 / 3.0 *
                       3.141592653589793238462643383279 * rl * rl * rl;
  const int want = ((int)std::ceil(1.25 * sites) + 7) / 8 * 8;
  c->cap = std::min(kMaxCap, std::max(kMinCap, want));
}

// Cubic coefficients c0..c3 (in y per grid step, t = s/h - k) on every
// interval k of the Hermite interpolant of y[0..n) whose node slopes are the
// finite differences of the samples: central inside, one-sided second order
// at the two ends.  From the Hermite basis: c0 = y_k, c1 = m_k,
// c2 = 3 (y_{k+1} - y_k) - 2 m_k - m_{k+1}, c3 = 2 (y_k - y_{k+1}) + m_k + m_{k+1}.
std::vector<double> hermite_cubics(const double* y, int n) {
  auto m = [&](int k) {
    if (k == 0) return 0.5 * (-3.0 * y[0] + 4.0 * y[1] - y[2]);
    if (k == n - 1) return 0.5 * (3.0 * y[n - 1] - 4.0 * y[n - 2] + y[n - 3]);
    return 0.5 * (y[k + 1] - y[k - 1]);
  };
  std::vector<double> c(4 * (size_t)(n - 1));
  for (int k = 0; k + 1 < n; ++k) {
    const double a = y[k], b = y[k + 1], ma = m(k), mb = m(k + 1);
    c[4 * (size_t)k + 0] = a;
    c[4 * (size_t)k + 1] = ma;
    c[4 * (size_t)k + 2] = 3.0 * (b - a) - 2.0 * ma - mb;
    c[4 * (size_t)k + 3] = 2.0 * (a - b) + ma + mb;
  }
  return c;
}

// ------------------------------------------------------------- launchers
tbsma_status launch_pack(tbsma_ctx* c, cudaStream_t s, int check) {
  const unsigned g = grid_for(c->N, 256);
  if (c->prec == TBSMA_MIXED)
    k_pack<TBSMA_MIXED><<<g, 256, 0, s>>>(c->N, c->x, c->meta, c->wd, c->xq, c->xd, c->xq_b,
                                          c->xd_b, c->half_skin2, check, c->flag, c->wire_status);
  else
    k_pack<TBSMA_FP64><<<g, 256, 0, s>>>(c->N, c->x, c->meta, c->wd, c->xq, c->xd, c->xq_b,
                                         c->xd_b, c->half_skin2, check, c->flag, c->wire_status);
  TB_CUDA(c, cudaGetLastError());
  return TBSMA_OK;
}

// The list rebuild of the wires the plan selected (each kernel returns at
// once when none is selected): envelopes and the choice of build per wire,
// then the cell build (clear the cells, bin, sort each cell, build) of the
// wires that need it, then the slab build of the others (MIXED contexts).
tbsma_status launch_rebuild(tbsma_ctx* c, cudaStream_t s) {
  const bool mixed = c->prec == TBSMA_MIXED;
  if (mixed) {
    k_nl_env_tiles<<<(unsigned)(c->sm_count * 8), kSlotTile, 0, s>>>(c->nw(), c->wd, c->x);
    k_nl_env_merge<<<(unsigned)(c->sm_count * 8), kSlotTile, 0, s>>>(c->nw(), c->wd);
  }
  const unsigned gs = (unsigned)(c->sm_count * 4);
  k_nl_clear<<<gs, 256, 0, s>>>(c->nw(), c->wd, c->cell_count);
  k_nl_bin<<<gs, 256, 0, s>>>(c->nw(), c->wd, c->x, c->N, c->cell_count, c->cell_atoms,
                              c->cell_of, c->wire_status);
  k_nl_sort<<<gs * 2, 256, 0, s>>>(c->nw(), c->wd, c->cell_count, c->cell_atoms);
  const unsigned gb = (unsigned)(c->sm_count * 8);
  const size_t sbuf = (size_t)256 * c->cap * sizeof(int16_t);  // per-thread entry buffers
  if (mixed) {
    k_nl_build<int4><<<gb, 256, sbuf, s>>>(c->nw(), c->wd, c->cell_count, c->cell_atoms, c->cell_of,
                                           c->slot_of, c->rlist2u, c->nbr, c->n_nbr, c->cap, c->jrange,
                                           c->xq, c->xq_b, c->wire_status);
    const size_t sslab = (size_t)256 * ((c->cap + kSlabSlack) * sizeof(int16_t) + c->cap * sizeof(uint8_t));
    k_nl_build_slab<<<(unsigned)(c->sm_count * 3), 256, sslab, s>>>(
        c->nw(), c->wd, c->slot_of, c->rlist2, c->slab_range, c->nbr, c->n_nbr, c->cap,
        c->jrange, c->xq, c->xq_b, c->wire_status);
  } else {
    k_nl_build<double4_32a><<<gb, 256, sbuf, s>>>(c->nw(), c->wd, c->cell_count, c->cell_atoms,
                                                  c->cell_of, c->slot_of, c->rlist2, c->nbr, c->n_nbr,
                                                  c->cap, c->jrange, c->xd, c->xd_b, c->wire_status);
  }
  TB_CUDA(c, cudaGetLastError());
  return TBSMA_OK;
}

tbsma_status launch_nl(tbsma_ctx* c, cudaStream_t s, int force_all, int count_rebuild,
                       int64_t* step_counter) {
  k_nl_plan<<<1, 1024, 0, s>>>(c->W, c->nw(), c->wd, force_all, count_rebuild, step_counter,
                               c->step_counter);
  return launch_rebuild(c, s);
}

template <bool OBS, bool EAM, int LANES>
void pair_f32_pot(tbsma_ctx* c, cudaStream_t s, int which) {
  const unsigned g = grid_for(c->NS * LANES, c->block);
  const size_t smem = (size_t)c->wcap * sizeof(int4);
  if (which & 1)
    k_density_f32<OBS, EAM, LANES><<<g, c->block, smem, s>>>(c->NS, c->xq, c->nbr, c->n_nbr, c->perm,
                                                             c->jrange, c->cap, c->wcap, c->pc,
                                                             c->e_band, c->eam);
  if (which & 2)
    k_force_f32<OBS, EAM, LANES><<<g, c->block, smem, s>>>(c->NS, c->xq, c->nbr, c->n_nbr, c->perm,
                                                           c->jrange, c->cap, c->wcap, c->pc, c->f32,
                                                           c->f32 + c->N, c->f32 + 2 * c->N,
                                                           c->e_band, c->e_atom, c->w_atom, c->s_atom,
                                                           c->eam);
}

// Threads per atom of the MIXED pair passes.
int graph_lanes(const tbsma_ctx* c) { return c->lanes; }

template <bool OBS, bool EAM>
void pair_f32_lanes(tbsma_ctx* c, cudaStream_t s, int which) {
  switch (graph_lanes(c)) {
    case 4: pair_f32_pot<OBS, EAM, 4>(c, s, which); break;
    case 2: pair_f32_pot<OBS, EAM, 2>(c, s, which); break;
    default: pair_f32_pot<OBS, EAM, 1>(c, s, which);
  }
}

template <bool OBS>
void pair_f32(tbsma_ctx* c, cudaStream_t s, int which = 3) {
  if (c->eam_on) pair_f32_lanes<OBS, true>(c, s, which);
  else pair_f32_lanes<OBS, false>(c, s, which);
}

template <bool OBS, bool DECIDE32, bool EAM>
void pair_f64_pot(tbsma_ctx* c, cudaStream_t s, int which) {
  const unsigned g = grid_for(c->NS * kLanes64, kPair64Block);  // kLanes64 lanes per atom
  if (which & 1)
    k_density_f64<OBS, DECIDE32, EAM><<<g, kPair64Block, 0, s>>>(c->NS, c->xd, c->xq, c->nbr, c->n_nbr,
                                                              c->perm, c->cap, c->pc, c->inv64,
                                                              c->e_band, c->eam);
  if (which & 2)
    k_force_f64<OBS, DECIDE32, EAM><<<g, kPair64Block, 0, s>>>(c->N, c->NS, c->xd, c->xq, c->nbr, c->n_nbr,
                                                            c->perm, c->cap, c->pc, c->inv64, c->f64,
                                                            c->e_band, c->e_atom, c->w_atom, c->s_atom,
                                                            c->eam);
}

template <bool OBS, bool DECIDE32>
void pair_f64(tbsma_ctx* c, cudaStream_t s, int which = 3) {
  if (c->eam_on) pair_f64_pot<OBS, DECIDE32, true>(c, s, which);
  else pair_f64_pot<OBS, DECIDE32, false>(c, s, which);
}

// prec: arithmetic of the pass; decide32: FP64 pass taking the FP32 cutoff rule
template <bool OBS>
tbsma_status launch_pair(tbsma_ctx* c, cudaStream_t s, int prec, bool decide32 = false) {
  if (prec == TBSMA_MIXED) pair_f32<OBS>(c, s);
  else if (decide32) pair_f64<OBS, true>(c, s);
  else pair_f64<OBS, false>(c, s);
  TB_CUDA(c, cudaGetLastError());
  return TBSMA_OK;
}

// One pass alone (1 = density, 2 = force), context precision.
tbsma_status launch_one_pass(tbsma_ctx* c, cudaStream_t s, int pass) {
  if (c->prec == TBSMA_MIXED) pair_f32<false>(c, s, pass);
  else pair_f64<false, false>(c, s, pass);
  TB_CUDA(c, cudaGetLastError());
  return TBSMA_OK;
}

ProtoDev proto_dev(const tbsma_ctx* c) {
  ProtoDev p;
  p.thermo = c->proto.thermostat;
  p.pull = c->proto.pull;
  p.tau = c->proto.tau_fs;
  p.pull_step = c->proto.pull_step;
  p.interval = c->proto.pull_interval;
  p.t_start = c->proto.t_start;
  p.ramp = c->proto.ramp_steps;
  p.ramp_start = c->proto.ramp_start;
  p.baro = c->proto.baro_tau_fs > 0.0 ? 1 : 0;
  return p;
}

bool nose_hoover(const tbsma_ctx* c) { return c->proto.thermostat == TBSMA_THERMO_NOSE_HOOVER; }
bool barostat(const tbsma_ctx* c) { return c->proto.baro_tau_fs > 0.0; }

// A protocol other than the default (Langevin, continuous pull, no ramp, no barostat).
bool protocol_mode(const tbsma_ctx* c) {
  return c->proto.thermostat != TBSMA_THERMO_LANGEVIN || c->proto.pull != TBSMA_PULL_CONTINUOUS ||
         c->proto.ramp_steps > 0 || barostat(c);
}

template <int KICK, bool PROTO>
void integrate_as(tbsma_ctx* c, cudaStream_t s, double dt) {
  const unsigned g = grid_for(c->N, 256);
  // the mixed kernel takes the kick it applies at once: the merged full kick
  // of B A O A B, or the half kick that Nosé–Hoover applies on either side of
  // its scaling
  const double kick = 0.5 * (nose_hoover(c) ? 1 : KICK) * dt * c->inv_m;
  if (c->prec == TBSMA_MIXED)
    k_integrate_mixed<KICK, PROTO><<<g, 256, 0, s>>>(
        c->N, c->x, c->v, c->f32, c->meta, c->wd, c->wdyn, (float)kick, (float)(0.5 * dt),
        c->step_counter, c->xq, c->xq_b, (float)c->half_skin2, c->flag, c->wire_status,
        c->d_grip, proto_dev(c), c->nh, c->baro);
  else  // warp-sized blocks: FP64-bound, so a small context's atoms reach more SMs
    k_integrate<TBSMA_FP64, KICK, PROTO><<<grid_for(c->N, 32), 32, 0, s>>>(
        c->N, c->x, c->v, c->f32, c->f64, c->meta, c->wd, c->wdyn, dt, c->inv_m, c->step_counter,
        c->xq, c->xd, c->xq_b, c->xd_b, c->half_skin2, c->flag, c->wire_status, c->d_grip,
        proto_dev(c), c->nh, c->baro);
}

template <int KICK>
void integrate(tbsma_ctx* c, cudaStream_t s, double dt) {
  if (protocol_mode(c)) integrate_as<KICK, true>(c, s, dt);
  else integrate_as<KICK, false>(c, s, dt);
}

// Nosé–Hoover half steps at a step boundary (mode 1 end, 2 begin, 3 both);
// kick = the closing half kick still to be applied to v (0 if applied).
void nh_boundary(tbsma_ctx* c, cudaStream_t s, double dt, double kick, int mode) {
  k_nh<<<std::min(c->W, 65535), 256, 0, s>>>(c->W, c->wd, c->meta, c->N, c->v, c->f32, c->f64,
                                               c->prec, kick, mode, dt, proto_dev(c),
                                               c->P.mass * kMvv2e, c->step_counter, c->nh);
}

void half_kick(tbsma_ctx* c, cudaStream_t s, double hk) {
  const unsigned g = grid_for(c->N, 256);
  if (c->prec == TBSMA_MIXED)
    k_half_kick<TBSMA_MIXED><<<g, 256, 0, s>>>(c->N, c->v, c->f32, c->f64, c->meta, hk);
  else
    k_half_kick<TBSMA_FP64><<<g, 256, 0, s>>>(c->N, c->v, c->f32, c->f64, c->meta, hk);
}

// n steps under the axial Nosé–Hoover barostat, each step whole:
//   k_baro_begin (Z C), [NH begin], B S A S (integrator), [forces + virial],
//   B, [NH end], k_baro_end (C Z).
// The first pass recomputes the virial of the current positions (the forces
// it writes are those already held: same positions, same list).
tbsma_status enqueue_steps_baro(tbsma_ctx* c, cudaStream_t s, int n, double dt) {
  const double hk = 0.5 * dt * c->inv_m;
  const double rhs = 0.5 * c->P.r0;
  BaroArgs a;
  a.m_e = c->P.mass * kMvv2e;
  a.v_atom = 4.0 / 3.0 * 3.141592653589793238462643383279 * rhs * rhs * rhs;
  a.h = 0.5 * dt;
  a.p = c->proto.baro_pressure;
  a.inv_btau2 = 1.0 / (c->proto.baro_modulus * c->proto.baro_tau_fs * c->proto.baro_tau_fs);
  a.drag = std::exp(-c->proto.baro_drag / c->proto.baro_tau_fs * a.h);
  const unsigned gw = (unsigned)std::min(c->W, 65535);
  TB_TRY(launch_pair<true>(c, s, c->prec));
  for (int k = 0; k < n; ++k) {
    k_baro_begin<<<gw, 256, 0, s>>>(c->W, c->wd, c->meta, c->N, c->x, c->v, c->w_atom, a, c->baro);
    if (nose_hoover(c)) nh_boundary(c, s, dt, 0.0, 2);
    integrate<1>(c, s, dt);
    TB_TRY(launch_nl(c, s, 0, 1, c->step_counter));
    TB_TRY(launch_pair<true>(c, s, c->prec));
    half_kick(c, s, hk);
    if (nose_hoover(c)) {
      nh_boundary(c, s, dt, 0.0, 1);
      k_nh_scale<<<grid_for(c->N, 256), 256, 0, s>>>(c->N, c->v, c->meta, c->nh);
    }
    k_baro_end<<<gw, 256, 0, s>>>(c->W, c->wd, c->meta, c->N, c->v, c->w_atom, a, c->baro);
  }
  TB_CUDA(c, cudaGetLastError());
  return TBSMA_OK;
}

// Optional per-phase timing of directly enqueued steps (tbsma_step_profile):
// an event is recorded after each phase and tagged with the phase it closes.
struct PhaseMarks {
  tbsma_ctx* c;
  std::vector<int> tag;  // tag[k]: the phase that ended at event k (-1: the start)
  cudaError_t err = cudaSuccess;
  void mark(cudaStream_t s, int phase) {
    const size_t k = tag.size();
    if (k >= c->prof_ev.size()) {
      cudaEvent_t e = nullptr;
      const cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) {
        err = r;
        return;
      }
      c->prof_ev.push_back(e);
    }
    const cudaError_t r = cudaEventRecord(c->prof_ev[k], s);
    if (r != cudaSuccess) err = r;
    tag.push_back(phase);
  }
};

// n consecutive steps: first integrate with a half kick, the rest with a
// merged full kick, and a closing half kick after the last force pass.
// With `pm`, the list rebuild chain and the two pair passes are enqueued
// one by one with an event after each phase (same kernels, same order).
// obs_last: the last step's pair passes also form the per-atom energy and
// virial terms (the same forces), for a report at the sequence's end.
tbsma_status enqueue_steps(tbsma_ctx* c, cudaStream_t s, int n, double dt, PhaseMarks* pm = nullptr,
                           bool obs_last = false) {
  if (barostat(c)) return enqueue_steps_baro(c, s, n, dt);
  const double hk = 0.5 * dt * c->inv_m;
  for (int k = 0; k < n; ++k) {
    // Nosé–Hoover: the begin half step (first step of the sequence) or the
    // previous step's end half step followed by this step's begin half step
    if (nose_hoover(c)) nh_boundary(c, s, dt, k == 0 ? 0.0 : hk, k == 0 ? 2 : 3);
    if (k == 0) integrate<1>(c, s, dt);
    else integrate<2>(c, s, dt);
    if (!pm) {
      TB_TRY(launch_nl(c, s, 0, 1, c->step_counter));
      if (obs_last && k == n - 1) TB_TRY(launch_pair<true>(c, s, c->prec));
      else TB_TRY(launch_pair<false>(c, s, c->prec));
      continue;
    }
    pm->mark(s, TBSMA_PHASE_INTEGRATE);
    k_nl_plan<<<1, 1024, 0, s>>>(c->W, c->nw(), c->wd, 0, 1, c->step_counter, c->step_counter);
    pm->mark(s, TBSMA_PHASE_PLAN);
    TB_TRY(launch_rebuild(c, s));
    pm->mark(s, TBSMA_PHASE_REBUILD);
    TB_TRY(launch_one_pass(c, s, 1));
    pm->mark(s, TBSMA_PHASE_DENSITY);
    TB_TRY(launch_one_pass(c, s, 2));
    pm->mark(s, TBSMA_PHASE_FORCE);
  }
  half_kick(c, s, hk);
  if (nose_hoover(c)) {  // the last step's end half step
    nh_boundary(c, s, dt, 0.0, 1);
    k_nh_scale<<<grid_for(c->N, 256), 256, 0, s>>>(c->N, c->v, c->meta, c->nh);
  }
  if (pm) pm->mark(s, TBSMA_PHASE_KICK);
  TB_CUDA(c, cudaGetLastError());
  return TBSMA_OK;
}

void drop_graph(tbsma_ctx* c) {
  if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
  c->graph = Graph{};
  c->graph_dt = -1.0;
  for (cudaGraphExec_t* g : {&c->obs_graph, &c->fc_graph, &c->seq_obs_graph})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  c->seq_obs_steps = 0;
  c->seq_obs_dt = -1.0;
}

// Launch the kernels `enqueue` puts on a stream as one graph, captured on
// first use and kept until drop_graph (a report's dozen short launches cost
// more than their work on a small context).
template <class F>
tbsma_status launch_captured(tbsma_ctx* c, cudaGraphExec_t& exec, F enqueue) {
  if (!exec) {
    cudaGraph_t g = nullptr;
    TB_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    const tbsma_status st = enqueue(c->cap_stream);
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (st != TBSMA_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      exec = nullptr;
      return cuda_fail(c, ei, "cudaGraphInstantiate");
    }
  }
  TB_CUDA(c, cudaGraphLaunch(exec, c->stream));
  return TBSMA_OK;
}

tbsma_status set_dt(tbsma_ctx* c, double dt) {
  if (dt == c->dt_dyn) return TBSMA_OK;
  std::vector<WireDyn> dyn(c->W);
  for (int w = 0; w < c->W; ++w) {
    const WireDev& d = c->wires_h[w];
    const double c1 = std::exp(-d.gamma * dt);
    const double sig = std::sqrt(kBoltzmann * d.temperature * c->inv_m);
    dyn[w].c1 = c1;
    dyn[w].c2sig = std::sqrt(std::max(0.0, 1.0 - c1 * c1)) * sig;
    dyn[w].delta = d.strain_rate * 1.0e-15 * d.L0 * dt / 2.0;
    dyn[w].c1m1f = (float)std::expm1(-d.gamma * dt);
    dyn[w].c2sigf = (float)dyn[w].c2sig;
  }
  TB_CUDA(c, cudaMemcpyAsync(c->wdyn, dyn.data(), sizeof(WireDyn) * c->W, cudaMemcpyHostToDevice,
                             c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  c->dt_dyn = dt;
  drop_graph(c);
  return TBSMA_OK;
}

// Captures `steps` steps as one kick sequence (enqueue_steps) into *out.
tbsma_status capture_steps(tbsma_ctx* c, int steps, double dt, bool obs_last, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  TB_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  tbsma_status st = enqueue_steps(c, c->cap_stream, steps, dt, nullptr, obs_last);
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (st != TBSMA_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  return TBSMA_OK;
}

tbsma_status capture(tbsma_ctx* c, int steps, double dt) {
  NvtxRange range_("capture step graph");
  drop_graph(c);
  TB_TRY(capture_steps(c, steps, dt, false, &c->graph.exec));
  c->graph.steps = steps;
  c->graph_dt = dt;
  return TBSMA_OK;
}

// ------------------------------------------------ persistent step kernel
// Dynamic shared memory of the persistent step kernel: the largest of the
// pair passes' window with the tile cache and the two builds' buffers.
// Threads per block of the persistent step kernel: 256-atom tiles (MIXED),
// the FP64 passes' blocks (FP64).
int persist_block(const tbsma_ctx* c) { return c->prec == TBSMA_MIXED ? 256 : kPair64Block; }

size_t persist_smem(const tbsma_ctx* c) {
  if (c->prec != TBSMA_MIXED) return (size_t)kPair64Block * c->cap * sizeof(int16_t);  // the cell build's
  const int slots = 256 / c->lanes;
  const size_t window = (size_t)c->wcap * sizeof(int4) + tile_cache_bytes(c->cap, slots);
  const size_t cell = (size_t)256 * c->cap * sizeof(int16_t);
  const size_t slab = (size_t)256 * ((c->cap + kSlabSlack) * sizeof(int16_t) + c->cap);
  return std::max(window, std::max(cell, slab));
}

// Threads per atom of the persistent kernel's pair passes.
int persist_lanes(const tbsma_ctx* c) { return c->lanes; }

const void* persist_fn(const tbsma_ctx* c) {
  if (c->prec != TBSMA_MIXED)
    return c->eam_on ? (const void*)k_steps_persistent_fp64<true> : (const void*)k_steps_persistent_fp64<false>;
  switch (persist_lanes(c)) {
    case 4:
      return c->eam_on ? (const void*)k_steps_persistent<true, 4> : (const void*)k_steps_persistent<false, 4>;
    case 2:
      return c->eam_on ? (const void*)k_steps_persistent<true, 2> : (const void*)k_steps_persistent<false, 2>;
    default:
      return c->eam_on ? (const void*)k_steps_persistent<true, 1> : (const void*)k_steps_persistent<false, 1>;
  }
}

// Blocks of the persistent step kernel for this context, 0 if it cannot run
// it: the default protocol, 256-atom tiles, and (MIXED) every tile of the
// batch resident at once (one block per tile, at most the co-resident
// blocks of a cooperative launch).
int persist_blocks(tbsma_ctx* c) {
  if (protocol_mode(c) || c->block != 256) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_fn(c), persist_block(c),
                                                    persist_smem(c)) !=
      cudaSuccess)
    return 0;
  const int64_t tiles = c->NS / 256;
  const int64_t most = (int64_t)per_sm * c->sm_count;
  if (tiles < 1 || tiles > most) return 0;
  // FP64: kLanes64 lanes per slot over the grid, as many blocks as the
  // slots fill or as fit, beyond one per SM rounded down to whole rounds of
  // the SMs (a second block on only some SMs would double their FP64 work
  // and hold up every barrier)
  if (c->prec != TBSMA_MIXED) {
    int64_t b = std::min<int64_t>(c->NS * kLanes64 / kPair64Block, most);
    if (b > c->sm_count) b = b / c->sm_count * c->sm_count;
    return (int)b;
  }
  // one block per tile of the pair passes (256 / lanes atoms), as many as fit
  return (int)std::min<int64_t>(tiles * persist_lanes(c), most);
}

// n steps in one cooperative launch of the persistent step kernel (the
// caller has checked persist_blocks > 0 and set dt).  Same steps, kicks and
// step counts as enqueue_steps.
tbsma_status launch_persistent_fp64(tbsma_ctx* c, int blocks, int n, int seq, double dt) {
  PersistArgs64 a;
  a.N = c->N;
  a.NS = c->NS;
  a.W = c->W;
  a.x = c->x;
  a.v = c->v;
  a.f64 = c->f64;
  a.meta = c->meta;
  a.wd = c->wd;
  a.wdyn = c->wdyn;
  a.dt = dt;
  a.inv_m = c->inv_m;
  a.hk_close = 0.5 * dt * c->inv_m;
  a.xq = c->xq;
  a.xd = c->xd;
  a.xq_b = c->xq_b;
  a.xd_b = c->xd_b;
  a.half_skin2 = c->half_skin2;
  a.flag = c->flag;
  a.wire_status = c->wire_status;
  a.d_grip = c->d_grip;
  a.step_counter = c->step_counter;
  a.nw = c->nw();
  a.cell_count = c->cell_count;
  a.cell_atoms = c->cell_atoms;
  a.cell_of = c->cell_of;
  a.slot_of = c->slot_of;
  a.rlist2 = c->rlist2;
  a.nbr = c->nbr;
  a.n_nbr = c->n_nbr;
  a.cap = c->cap;
  a.jrange = c->jrange;
  a.perm = c->perm;
  a.pc = c->pc;
  a.inv64 = c->inv64;
  a.eam = c->eam;
  a.step0 = c->steps_done;
  a.n_steps = n;
  a.seq = seq;
  a.bar = GridBarrier{reinterpret_cast<unsigned long long*>(c->bar), c->bar + 2,
                      (unsigned)std::max(0, c->wait_limit - 1) * 4u};
  TB_CUDA(c, cudaMemsetAsync(c->bar, 0, 3 * sizeof(unsigned), c->stream));
  void* args[] = {&a};
  TB_CUDA(c, cudaLaunchCooperativeKernel(persist_fn(c), dim3((unsigned)blocks), dim3(kPair64Block), args,
                                         persist_smem(c), c->stream));
  return TBSMA_OK;
}

tbsma_status launch_persistent(tbsma_ctx* c, int blocks, int n, int seq, double dt) {
  if (c->prec != TBSMA_MIXED) return launch_persistent_fp64(c, blocks, n, seq, dt);
  if (!c->xq2) TB_TRY(alloc(c, &c->xq2, (size_t)c->N));  // the kernel's second position buffer
  PersistArgs a;
  a.N = c->N;
  a.NS = c->NS;
  a.W = c->W;
  a.x = c->x;
  a.v = c->v;
  a.f32 = c->f32;
  a.meta = c->meta;
  a.wd = c->wd;
  a.wdyn = c->wdyn;
  a.hk_open = (float)(0.5 * dt * c->inv_m);
  a.hk_full = (float)(dt * c->inv_m);
  a.hd = (float)(0.5 * dt);
  a.hk_close = 0.5 * dt * c->inv_m;
  a.xq = c->xq;
  a.xq2 = c->xq2;
  a.xq_b = c->xq_b;
  a.half_skin2 = (float)c->half_skin2;
  a.flag = c->flag;
  a.wire_status = c->wire_status;
  a.d_grip = c->d_grip;
  a.step_counter = c->step_counter;
  a.nw = c->nw();
  a.cell_count = c->cell_count;
  a.cell_atoms = c->cell_atoms;
  a.cell_of = c->cell_of;
  a.slot_of = c->slot_of;
  a.rlist2u = c->rlist2u;
  a.rlist2 = c->rlist2;
  a.slab_range = c->slab_range;
  a.nbr = c->nbr;
  a.n_nbr = c->n_nbr;
  a.cap = c->cap;
  a.jrange = c->jrange;
  a.perm = c->perm;
  a.wcap = c->wcap;
  a.pc = c->pc;
  a.eam = c->eam;
  a.step0 = c->steps_done;
  a.n_steps = n;
  a.seq = seq;
  a.bar = GridBarrier{reinterpret_cast<unsigned long long*>(c->bar), c->bar + 2,
                      (unsigned)std::max(0, c->wait_limit - 1) * 4u};
  TB_CUDA(c, cudaMemsetAsync(c->bar, 0, 3 * sizeof(unsigned), c->stream));
  void* args[] = {&a};
  TB_CUDA(c, cudaLaunchCooperativeKernel(persist_fn(c), dim3((unsigned)blocks), dim3(256), args,
                                         persist_smem(c), c->stream));
  return TBSMA_OK;
}

// The persistent kernel's barrier error word: ETIMEOUT if a wait gave up.
tbsma_status persist_verdict(tbsma_ctx* c) {
  unsigned err = 0;
  TB_CUDA(c, cudaMemcpyAsync(&err, c->bar + 2, sizeof err, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  if (err) return fail(c, TBSMA_ETIMEOUT, "a grid barrier of the persistent step kernel gave up");
  return TBSMA_OK;
}

tbsma_status read_status(tbsma_ctx* c, std::vector<uint32_t>& st) {
  st.resize(c->W);
  TB_CUDA(c, cudaMemcpyAsync(st.data(), c->wire_status, sizeof(uint32_t) * c->W,
                             cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  return TBSMA_OK;
}

// Replace the cell arrays by ones of `cells` cells (contents are not kept:
// cells carry nothing from one list build to the next).  Drops the captured
// graph, whose kernels hold the old pointers.
tbsma_status realloc_cells(tbsma_ctx* c, int64_t cells) {
  auto release = [&](void* p) {
    c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), p), c->allocs.end());
    cudaFree(p);
  };
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  drop_graph(c);
  release(c->cell_count);
  release(c->cell_atoms);
  c->cell_count = nullptr;
  c->cell_atoms = nullptr;
  c->cells_alloc = 0;
  TB_TRY(alloc(c, &c->cell_count, cells));
  TB_TRY(alloc(c, &c->cell_atoms, (size_t)cells * kCellCap));
  c->cells_alloc = cells;
  return TBSMA_OK;
}

// Grow the cell grids of the wires whose status (st, just read) carries
// kWireGridClamp or kWireCellOverflow: re-plan each around its current
// bounding box (plan_grid, the fixed-point origin unchanged), give every
// wire its new first cell, enlarge the cell arrays if needed (by at least
// a quarter), clear the two bits (in st and on the device) and rebuild
// those wires' lists.  Where a cell overflowed, the forces at the current
// positions are recomputed as well (the list they came from missed atoms).
// Poisoned (non-finite) wires keep their grid; their clamp bit is cleared.
tbsma_status grow_grids(tbsma_ctx* c, std::vector<uint32_t>& st) {
  const uint32_t grow_bits = kWireGridClamp | kWireCellOverflow;
  std::vector<int> g;
  bool overflowed = false;
  for (int w = 0; w < c->W; ++w) {
    if (!(st[w] & grow_bits)) continue;
    if (st[w] & kWireNonFinite) {
      st[w] &= ~kWireGridClamp;
      continue;
    }
    g.push_back(w);
    overflowed |= (st[w] & kWireCellOverflow) != 0;
  }
  if (!g.empty()) {
    k_bbox<<<std::min(c->W, 65535), 256, 0, c->stream>>>(c->W, c->wires_d, c->x, c->N, c->kind,
                                                         c->bbox_d);
    TB_CUDA(c, cudaGetLastError());
    std::vector<double> bbox((size_t)c->W * 7);
    TB_CUDA(c, cudaMemcpyAsync(bbox.data(), c->bbox_d, sizeof(double) * 7 * c->W,
                               cudaMemcpyDeviceToHost, c->stream));
    TB_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<WireDev> grids = c->wires_h;
    for (int w : g) {
      const double* lo = &bbox[(size_t)w * 7];
      if (!(std::isfinite(lo[0]) && std::isfinite(lo[1]) && std::isfinite(lo[2]) &&
            std::isfinite(lo[3]) && std::isfinite(lo[4]) && std::isfinite(lo[5])))
        continue;  // non-finite since the status was read: left to the verdict
      if (!plan_grid(grids[w], lo, lo + 3, c->cell_edge)) {
        char buf[128];
        snprintf(buf, sizeof buf, "wire %d: its cell grid would need more than 1023 cells per axis", w);
        return fail(c, TBSMA_EOVERFLOW, buf);
      }
    }
    int64_t cells = 0;
    for (int w = 0; w < c->W; ++w) {
      grids[w].cell_base = cells;
      cells += (int64_t)grids[w].nc[0] * grids[w].nc[1] * grids[w].nc[2];
    }
    if (cells > c->cells_alloc) TB_TRY(realloc_cells(c, std::max(cells, c->cells_alloc + c->cells_alloc / 4)));
    c->wires_h = grids;
    c->n_cells = cells;
    TB_CUDA(c, cudaMemcpyAsync(c->wd, c->wires_h.data(), sizeof(WireDev) * c->W,
                               cudaMemcpyHostToDevice, c->stream));
    std::vector<int32_t> flag(c->W);
    TB_CUDA(c, cudaMemcpyAsync(flag.data(), c->flag, sizeof(int32_t) * c->W, cudaMemcpyDeviceToHost,
                               c->stream));
    TB_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int w : g) {
      flag[w] = 1;
      st[w] &= ~grow_bits;
    }
    TB_CUDA(c, cudaMemcpyAsync(c->flag, flag.data(), sizeof(int32_t) * c->W, cudaMemcpyHostToDevice,
                               c->stream));
  }
  TB_CUDA(c, cudaMemcpyAsync(c->wire_status, st.data(), sizeof(uint32_t) * c->W,
                             cudaMemcpyHostToDevice, c->stream));
  if (!g.empty()) {
    TB_TRY(launch_nl(c, c->stream, 0, 0, nullptr));
    if (overflowed) TB_TRY(launch_pair<false>(c, c->stream, c->prec));
  }
  TB_CUDA(c, cudaStreamSynchronize(c->stream));  // st (host) was read by the copy above
  return TBSMA_OK;
}

// Read the wires' status words and grow the grids that need it.  Returns
// whether some wire's cell had overflowed (its grid is grown now, but the
// steps since its previous list build ran on a list that missed atoms).
tbsma_status check_grids(tbsma_ctx* c, std::vector<uint32_t>& st, int& overflowed_wire) {
  TB_TRY(read_status(c, st));
  overflowed_wire = -1;
  uint32_t grow = 0;
  for (int w = 0; w < c->W; ++w) {
    grow |= st[w] & (kWireGridClamp | kWireCellOverflow);
    if ((st[w] & kWireCellOverflow) && overflowed_wire < 0) overflowed_wire = w;
  }
  if (grow) TB_TRY(grow_grids(c, st));
  return TBSMA_OK;
}

tbsma_status status_verdict(tbsma_ctx* c) {
  std::vector<uint32_t> st;
  int ofw = -1;
  TB_TRY(check_grids(c, st, ofw));
  uint32_t any = 0;
  int first = -1;
  for (int w = 0; w < c->W; ++w) {
    any |= st[w];
    if (st[w] && first < 0) first = w;
  }
  char buf[224];
  if (!any) {
    if (ofw < 0) return TBSMA_OK;
    snprintf(buf, sizeof buf,
             "wire %d: a cell overflowed; its cell grid is grown and its list rebuilt, but the steps "
             "since its previous list build used a list that missed atoms (repeat them from saved state)",
             ofw);
    return fail(c, TBSMA_EOVERFLOW, buf);
  }
  snprintf(buf, sizeof buf, "wire %d status 0x%x (bits over all wires 0x%x)", first, st[first], any);
  if (ofw >= 0 || (any & (kWireNbrOverflow | kWireCellOverflow))) return fail(c, TBSMA_EOVERFLOW, buf);
  return fail(c, TBSMA_EWIRE, buf);
}

// Re-read positions, rebuild flagged (or all) wires, forces in `prec`.
tbsma_status refresh(tbsma_ctx* c, int force_all) {
  TB_TRY(launch_pack(c, c->stream, force_all ? 0 : 1));
  TB_TRY(launch_nl(c, c->stream, force_all, 0, nullptr));
  return TBSMA_OK;
}

// Upload validated EAM tables (tbsma_set_eam) and switch the context to them;
// on an error the context keeps eam_on = false.
tbsma_status upload_eam(tbsma_ctx* c, const tbsma_eam* t) {
  const std::vector<double> cf = hermite_cubics(t->f, t->n_r);
  const std::vector<double> cp = hermite_cubics(t->phi, t->n_r);
  const std::vector<double> cF = hermite_cubics(t->F, t->n_rho);
  const size_t nr = (size_t)t->n_r - 1, nF = (size_t)t->n_rho - 1;
  std::vector<float4> f32(nr), d32(2 * nr), p32(nr), F32(nF);
  const double idr = 1.0 / t->d_r;
  for (size_t k = 0; k < nr; ++k) {
    const double* a = &cf[4 * k];
    const double* b = &cp[4 * k];
    f32[k] = make_float4((float)a[0], (float)a[1], (float)a[2], (float)a[3]);
    p32[k] = make_float4((float)b[0], (float)b[1], (float)b[2], (float)b[3]);
    d32[2 * k] = make_float4((float)(a[1] * idr), (float)(2.0 * a[2] * idr), (float)(3.0 * a[3] * idr),
                             (float)(b[1] * idr));
    d32[2 * k + 1] = make_float4((float)(2.0 * b[2] * idr), (float)(3.0 * b[3] * idr), 0.f, 0.f);
  }
  for (size_t k = 0; k < nF; ++k)
    F32[k] = make_float4((float)cF[4 * k], (float)cF[4 * k + 1], (float)cF[4 * k + 2],
                         (float)cF[4 * k + 3]);
  // one allocation, every table 256-byte aligned
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t o_f32 = 0, o_d32 = o_f32 + up(nr * 16), o_p32 = o_d32 + up(2 * nr * 16);
  const size_t o_F32 = o_p32 + up(nr * 16), o_f64 = o_F32 + up(nF * 16);
  const size_t o_p64 = o_f64 + up(nr * 32), o_F64 = o_p64 + up(nr * 32);
  const size_t total = o_F64 + up(nF * 32);
  void* base = nullptr;
  cudaError_t e = cudaMalloc(&base, total);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc (EAM tables)");
  c->eam_allocs.push_back(base);
  char* b = static_cast<char*>(base);
  const struct {
    size_t off;
    const void* src;
    size_t bytes;
  } parts[] = {{o_f32, f32.data(), nr * 16},     {o_d32, d32.data(), 2 * nr * 16},
               {o_p32, p32.data(), nr * 16},     {o_F32, F32.data(), nF * 16},
               {o_f64, cf.data(), nr * 32},      {o_p64, cp.data(), nr * 32},
               {o_F64, cF.data(), nF * 32}};
  for (const auto& q : parts)
    TB_CUDA(c, cudaMemcpyAsync(b + q.off, q.src, q.bytes, cudaMemcpyHostToDevice, c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));  // the host staging vectors go out of scope
  EamDev& d = c->eam;
  d.f32 = reinterpret_cast<const float4*>(b + o_f32);
  d.d32 = reinterpret_cast<const float4*>(b + o_d32);
  d.p32 = reinterpret_cast<const float4*>(b + o_p32);
  d.F32 = reinterpret_cast<const float4*>(b + o_F32);
  d.f64 = reinterpret_cast<const double*>(b + o_f64);
  d.p64 = reinterpret_cast<const double*>(b + o_p64);
  d.F64 = reinterpret_cast<const double*>(b + o_F64);
  const double ifx = idr / kFixedScale;  // per fixed-point unit of r
  d.inv_dr_hi = (float)ifx;
  d.inv_dr_lo = (float)(ifx - (double)d.inv_dr_hi);
  const double irho = 1.0 / t->d_rho;
  d.inv_drho_hi = (float)irho;
  d.inv_drho_lo = (float)(irho - (double)d.inv_drho_hi);
  d.kmax_r = t->n_r - 2;
  d.kmax_rho = t->n_rho - 2;
  d.inv_dr = idr;
  d.inv_drho = irho;
  c->eam_on = true;
  return TBSMA_OK;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

tbsma_status tbsma_init(const tbsma_params* params, tbsma_precision precision, int32_t n_wires,
                        const tbsma_wire* wires, double* x, double* v, const uint8_t* kind,
                        void* cuda_stream, tbsma_ctx** out) {
  NvtxRange range_("tbsma_init");
  if (!out) return TBSMA_EINVAL;
  *out = nullptr;
  if (!params || !wires || !x || !v || !kind || n_wires < 1) return TBSMA_EINVAL;
  if (precision != TBSMA_FP64 && precision != TBSMA_MIXED) return TBSMA_EINVAL;
  const tbsma_params& P = *params;
  if (!(P.r0 > 0 && P.r_cut > 0 && P.r_skin >= 0 && P.mass > 0 && P.xi > 0 && P.A >= 0))
    return TBSMA_EINVAL;
  int64_t N = 0;
  for (int w = 0; w < n_wires; ++w) {
    if (wires[w].atom_offset != N || wires[w].n_atoms < 1 || wires[w].reserved != 0 ||
        !(wires[w].L0 > 0) || wires[w].gamma < 0 || wires[w].temperature < 0)
      return TBSMA_EINVAL;
    N += wires[w].n_atoms;
  }
  if (N >= (int64_t)1 << 31) return TBSMA_EINVAL;  // neighbour indices are int32

  tbsma_ctx* c = new tbsma_ctx();
  c->P = P;
  c->prec = precision;
  c->W = n_wires;
  c->N = N;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->x = x;
  c->v = v;
  c->kind = kind;
  fill_pair_consts(c);

  auto bail = [&](tbsma_status s) {
    tbsma_destroy(c);
    return s;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return bail(TBSMA_ECUDA);
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(TBSMA_ECUDA);
  const int smem_max = kMaxWindow * (int)sizeof(int4);
  const auto smem_attr = [&](const void* k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) == cudaSuccess;
  };
  if (!smem_attr((const void*)k_density_f32<false, false, 1>) ||
      !smem_attr((const void*)k_density_f32<true, false, 1>) ||
      !smem_attr((const void*)k_force_f32<false, false, 1>) ||
      !smem_attr((const void*)k_force_f32<true, false, 1>) ||
      !smem_attr((const void*)k_density_f32<false, true, 1>) ||
      !smem_attr((const void*)k_density_f32<true, true, 1>) ||
      !smem_attr((const void*)k_force_f32<false, true, 1>) ||
      !smem_attr((const void*)k_force_f32<true, true, 1>) ||
      !smem_attr((const void*)k_density_f32<false, false, 4>) ||
      !smem_attr((const void*)k_density_f32<true, false, 4>) ||
      !smem_attr((const void*)k_force_f32<false, false, 4>) ||
      !smem_attr((const void*)k_force_f32<true, false, 4>) ||
      !smem_attr((const void*)k_density_f32<false, true, 4>) ||
      !smem_attr((const void*)k_density_f32<true, true, 4>) ||
      !smem_attr((const void*)k_force_f32<false, true, 4>) ||
      !smem_attr((const void*)k_force_f32<true, true, 4>) ||
      !smem_attr((const void*)k_density_f32<false, false, 2>) ||
      !smem_attr((const void*)k_density_f32<true, false, 2>) ||
      !smem_attr((const void*)k_force_f32<false, false, 2>) ||
      !smem_attr((const void*)k_force_f32<true, false, 2>) ||
      !smem_attr((const void*)k_density_f32<false, true, 2>) ||
      !smem_attr((const void*)k_density_f32<true, true, 2>) ||
      !smem_attr((const void*)k_force_f32<false, true, 2>) ||
      !smem_attr((const void*)k_force_f32<true, true, 2>))
    return bail(TBSMA_ECUDA);
  const int sbuf_max = 256 * kMaxCap * (int)sizeof(int16_t);  // k_nl_build's entry buffers
  const int slab_max = 256 * ((kMaxCap + kSlabSlack) * (int)sizeof(int16_t) + kMaxCap);  // k_nl_build_slab's
  if (cudaFuncSetAttribute(k_nl_build<int4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sbuf_max) != cudaSuccess ||
      cudaFuncSetAttribute(k_nl_build<double4_32a>, cudaFuncAttributeMaxDynamicSharedMemorySize, sbuf_max) != cudaSuccess ||
      cudaFuncSetAttribute(k_nl_build_slab, cudaFuncAttributeMaxDynamicSharedMemorySize, slab_max) != cudaSuccess)
    return bail(TBSMA_ECUDA);
  // the persistent kernel: the largest window with its tile cache, or a
  // build's buffers, up to what a block may opt in to (a context whose
  // shape needs more runs graph replays: persist_blocks finds no room)
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return bail(TBSMA_ECUDA);
  const int persist_max = std::min(
      optin, std::max(std::max(smem_max + (int)tile_cache_bytes(kMaxCap, 256), sbuf_max), slab_max));
  if (cudaFuncSetAttribute(k_steps_persistent<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, persist_max) != cudaSuccess ||
      cudaFuncSetAttribute(k_steps_persistent<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, persist_max) != cudaSuccess ||
      cudaFuncSetAttribute(k_steps_persistent<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, persist_max) != cudaSuccess ||
      cudaFuncSetAttribute(k_steps_persistent<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, persist_max) != cudaSuccess ||
      cudaFuncSetAttribute(k_steps_persistent<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, persist_max) != cudaSuccess ||
      cudaFuncSetAttribute(k_steps_persistent<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, persist_max) != cudaSuccess ||
      cudaFuncSetAttribute(k_steps_persistent_fp64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sbuf_max) != cudaSuccess ||
      cudaFuncSetAttribute(k_steps_persistent_fp64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sbuf_max) != cudaSuccess)
    return bail(TBSMA_ECUDA);
  const int W = n_wires;
  tbsma_status s = TBSMA_OK;
#define ALLOC(ptr, n)                          \
  if ((s = alloc(c, &(ptr), (n))) != TBSMA_OK) \
    return bail(s);
  // per-wire bounding boxes on the device (init only)
  ALLOC(c->wires_d, W);
  ALLOC(c->bbox_d, (size_t)W * 7);
  if (cudaMemcpyAsync(c->wires_d, wires, sizeof(tbsma_wire) * W, cudaMemcpyHostToDevice, c->stream) !=
      cudaSuccess)
    return bail(TBSMA_ECUDA);
  k_bbox<<<std::min(W, 65535), 256, 0, c->stream>>>(W, c->wires_d, x, N, kind, c->bbox_d);
  std::vector<double> bbox((size_t)W * 7);
  if (cudaMemcpyAsync(bbox.data(), c->bbox_d, sizeof(double) * 7 * W, cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(TBSMA_ECUDA);

  // per-wire cell grids: edge >= list radius (with a 1e-4 relative guard so
  // rounding in the cell coordinate never separates two atoms by two cells)
  const double rl = std::sqrt((double)c->rlist2) * 1.0001;
  c->cell_edge = rl;
  c->wires_h.resize(W);
  int64_t cells = 0, slots = 0;
  for (int w = 0; w < W; ++w) {
    WireDev& d = c->wires_h[w];
    std::memset(&d, 0, sizeof d);
    d.offset = wires[w].atom_offset;
    d.n = wires[w].n_atoms;
    d.n_mobile = (int32_t)bbox[w * 7 + 6];
    d.seed = wires[w].seed;
    d.L0 = wires[w].L0;
    d.strain_rate = wires[w].strain_rate;
    d.temperature = wires[w].temperature;
    d.gamma = wires[w].gamma;
    for (int k = 0; k < 3; ++k) {
      const double lo = bbox[w * 7 + k], hi = bbox[w * 7 + 3 + k];
      if (!std::isfinite(lo) || !std::isfinite(hi)) return bail(fail(c, TBSMA_EINVAL, "non-finite positions"));
      if (!(std::fabs(0.5 * (lo + hi)) < kFixedRange))
        return bail(fail(c, TBSMA_EINVAL, "wire centre beyond 1e7 A of the coordinate origin"));
      // origin on the 2^-26 grid, so that fixed_coord's offset is an exact integer
      d.origin[k] = std::nearbyint(0.5 * (lo + hi) * kFixedScale) / kFixedScale;
      d.ofixm[k] = kFixedMagic - d.origin[k] * kFixedScale;
    }
    if (!plan_grid(d, &bbox[w * 7], &bbox[w * 7 + 3], rl))
      return bail(fail(c, TBSMA_EINVAL, "wire too large for the cell grid (1023 cells per axis)"));
    d.cell_base = cells;
    cells += (int64_t)d.nc[0] * d.nc[1] * d.nc[2];
    d.slot_base = slots;
    slots += (d.n + kSlotTile - 1) / kSlotTile * (int64_t)kSlotTile;
  }
  c->n_cells = cells;
  c->cells_alloc = cells;
  c->NS = slots;
  const int64_t NS = slots;

  ALLOC(c->wd, W);
  ALLOC(c->wdyn, W);
  ALLOC(c->meta, N);
  ALLOC(c->xq, N);
  ALLOC(c->xq_b, N);
  ALLOC(c->xd, N);
  ALLOC(c->xd_b, N);
  ALLOC(c->f32, 3 * N);
  ALLOC(c->f64, 3 * N);
  ALLOC(c->inv64, N);
  ALLOC(c->e_band, N);
  ALLOC(c->e_atom, N);
  ALLOC(c->w_atom, N);
  ALLOC(c->s_atom, N);
  // + one group row: the force pass prefetches the group after a row's last one
  ALLOC(c->nbr, (size_t)((NS + 31) / 32) * 32 * c->cap + 32 * 4);
  ALLOC(c->jrange, NS);
  ALLOC(c->cell_of, N);
  ALLOC(c->perm, NS);
  ALLOC(c->slot_of, N);
  ALLOC(c->n_nbr, NS);
  ALLOC(c->cell_count, cells);
  ALLOC(c->cell_atoms, (size_t)cells * kCellCap);
  ALLOC(c->flag, W);
  ALLOC(c->wl_wire, W);
  ALLOC(c->wl_cell, W + 1);
  ALLOC(c->wl_atom, W + 1);
  ALLOC(c->wl_tile, W + 1);
  ALLOC(c->cl_wire, W);
  ALLOC(c->cl_cell, W + 1);
  ALLOC(c->cl_atom, W + 1);
  ALLOC(c->n_cell, 1);
  ALLOC(c->merge_done, 1);
  ALLOC(c->xenv, N);
  ALLOC(c->tenv, (size_t)(NS / kSlotTile));
  ALLOC(c->wdis, W);
  if (c->prec == TBSMA_MIXED) ALLOC(c->xf, (size_t)(NS / 4) * 3);  // slab-build candidates
  ALLOC(c->n_flagged, 1);
  ALLOC(c->n_rebuilds, W);
  ALLOC(c->chains, 1);
  ALLOC(c->rebuilt, 2);
  ALLOC(c->bar, 3);
  ALLOC(c->last_build, W);
  ALLOC(c->banked, W);
  ALLOC(c->wire_status, W);
  ALLOC(c->nh, W);
  ALLOC(c->baro, W);
  ALLOC(c->d_grip, W);
  ALLOC(c->step_counter, 1);
  ALLOC(c->obs_d, W);
  ALLOC(c->fcheck_d, W);
  ALLOC(c->fc_part, (size_t)(NS / 256) * 5);
#undef ALLOC

  cudaStream_t st = c->stream;
  bool ok = cudaMemcpyAsync(c->wd, c->wires_h.data(), sizeof(WireDev) * W, cudaMemcpyHostToDevice,
                            st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->flag, 0, sizeof(int32_t) * W, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->n_rebuilds, 0, sizeof(int32_t) * W, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->chains, 0, sizeof(int64_t), st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->n_cell, 0, sizeof(int32_t), st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->merge_done, 0, sizeof(uint32_t), st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->rebuilt, 0, 2 * sizeof(int64_t), st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->bar, 0, 3 * sizeof(unsigned), st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->last_build, 0, sizeof(int64_t) * W, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->banked, 0, W, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->wdis, 0xff, sizeof(uint32_t) * W, st) == cudaSuccess;  // NaN: cells
  ok = ok && cudaMemsetAsync(c->wire_status, 0, sizeof(uint32_t) * W, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->nh, 0, sizeof(NhState) * W, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->baro, 0, sizeof(BaroState) * W, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->d_grip, 0, sizeof(double) * W, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->step_counter, 0, sizeof(int64_t), st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->n_nbr, 0, sizeof(int32_t) * NS, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->jrange, 0, sizeof(int2) * NS, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->f32, 0, sizeof(float) * 3 * N, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->f64, 0, sizeof(double) * 3 * N, st) == cudaSuccess;
  if (!ok) return bail(TBSMA_ECUDA);
  k_meta<<<std::min(W, 65535), 256, 0, st>>>(W, c->wd, kind, c->meta);
  // build once in atom order, rank each tile's atoms by list length, build again
  k_slot_init<<<std::min(W, 65535), 256, 0, st>>>(W, c->wd, NS, c->perm, c->slot_of);
  if ((s = refresh(c, 1)) != TBSMA_OK) return bail(s);
  k_slot_order<<<grid_for(NS, kSlotTile), kSlotTile, 0, st>>>(NS, c->n_nbr, c->perm, c->slot_of);
  if ((s = refresh(c, 1)) != TBSMA_OK) return bail(s);
  if ((s = launch_pair<false>(c, st, c->prec)) != TBSMA_OK) return bail(s);
  if (cudaStreamSynchronize(st) != cudaSuccess) return bail(TBSMA_ECUDA);
  if ((s = status_verdict(c)) != TBSMA_OK && s != TBSMA_EWIRE && s != TBSMA_EOVERFLOW)
    return bail(s);
  *out = c;
  return s;
}

tbsma_status tbsma_init_velocities(tbsma_ctx* c) {
  NvtxRange range_("tbsma_init_velocities");
  if (!c) return TBSMA_EINVAL;
  k_init_velocities<<<std::min(c->W, 65535), 256, 0, c->stream>>>(c->W, c->wd, c->meta, c->N, c->v,
                                                                  c->P.mass * kMvv2e);
  TB_CUDA(c, cudaGetLastError());
  return TBSMA_OK;
}

tbsma_status tbsma_build_neighbors(tbsma_ctx* c, int32_t force_all, int32_t* n_rebuilt) {
  NvtxRange range_("tbsma_build_neighbors");
  if (!c) return TBSMA_EINVAL;
  TB_TRY(refresh(c, force_all ? 1 : 0));
  if (n_rebuilt) {
    TB_CUDA(c, cudaMemcpyAsync(n_rebuilt, c->n_flagged, sizeof(int32_t), cudaMemcpyDeviceToHost,
                               c->stream));
    TB_CUDA(c, cudaStreamSynchronize(c->stream));
    return status_verdict(c);
  }
  return TBSMA_OK;
}

tbsma_status tbsma_compute_forces(tbsma_ctx* c, float* f32_out, double* f64_out) {
  NvtxRange range_("tbsma_compute_forces");
  if (!c) return TBSMA_EINVAL;
  TB_TRY(refresh(c, 0));
  const int other = c->prec == TBSMA_MIXED ? TBSMA_FP64 : TBSMA_MIXED;
  if ((other == TBSMA_MIXED && f32_out) || (other == TBSMA_FP64 && f64_out))
    TB_TRY(launch_pair<false>(c, c->stream, other));
  TB_TRY(launch_pair<false>(c, c->stream, c->prec));
  const size_t n3 = 3 * (size_t)c->N;
  if (f32_out)
    TB_CUDA(c, cudaMemcpyAsync(f32_out, c->f32, n3 * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  if (f64_out)
    TB_CUDA(c, cudaMemcpyAsync(f64_out, c->f64, n3 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return TBSMA_OK;
}

tbsma_status tbsma_atom_energies(tbsma_ctx* c, double* e_out, double* w_out) {
  NvtxRange range_("tbsma_atom_energies");
  if (!c) return TBSMA_EINVAL;
  TB_TRY(refresh(c, 0));
  TB_TRY(launch_pair<true>(c, c->stream, c->prec));
  if (e_out)
    TB_CUDA(c, cudaMemcpyAsync(e_out, c->e_atom, c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  if (w_out)
    TB_CUDA(c, cudaMemcpyAsync(w_out, c->w_atom, c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return TBSMA_OK;
}

tbsma_status tbsma_step_nvt_pull(tbsma_ctx* c, int64_t n_steps, double dt_fs) {
  NvtxRange range_("tbsma_step_nvt_pull");
  if (!c) return TBSMA_EINVAL;
  if (n_steps < 0 || !(dt_fs > 0.0)) return fail(c, TBSMA_EINVAL, "n_steps < 0 or dt <= 0");
  if (n_steps == 0) return TBSMA_OK;
  TB_TRY(set_dt(c, dt_fs));
  const int pblocks = c->step_mode == TBSMA_STEPS_GRAPH ? 0 : persist_blocks(c);
  if (c->step_mode == TBSMA_STEPS_PERSISTENT && pblocks == 0)
    return fail(c, TBSMA_EINVAL, "this context cannot run the persistent step kernel");
  if (pblocks > 0) {
    // kick sequences as the graph path runs them: min(n_steps, kGraphChunk)
    // steps each (kGrowCheckSteps is a multiple of kGraphChunk)
    const int seq = (int)std::min<int64_t>(n_steps, kGraphChunk);
    int64_t left = n_steps;
    while (left > 0) {
      const int n = (int)std::min<int64_t>(left, kGrowCheckSteps);
      TB_TRY(launch_persistent(c, pblocks, n, seq, dt_fs));
      left -= n;
      c->steps_done += n;
      TB_TRY(persist_verdict(c));
      if (left > 0) {
        std::vector<uint32_t> st;
        int ofw = -1;
        TB_TRY(check_grids(c, st, ofw));
        if (ofw >= 0) return status_verdict(c);
      }
    }
    return status_verdict(c);
  }
  const int chunk = (int)std::min<int64_t>(n_steps, kGraphChunk);
  if (!c->graph.exec || c->graph_dt != dt_fs || c->graph.steps != chunk) TB_TRY(capture(c, chunk, dt_fs));
  int64_t left = n_steps, since_check = 0;
  while (left > 0) {
    if (left >= chunk) {
      if (!c->graph.exec) TB_TRY(capture(c, chunk, dt_fs));  // dropped by a grid growth
      TB_CUDA(c, cudaGraphLaunch(c->graph.exec, c->stream));
      left -= chunk;
      c->steps_done += chunk;
      since_check += chunk;
    } else {
      TB_TRY(enqueue_steps(c, c->stream, (int)left, dt_fs));
      c->steps_done += left;
      left = 0;
    }
    // a long call looks at the status words every kGrowCheckSteps steps, so
    // that a wire whose atoms leave its cell grid gets a larger grid before
    // the clamped edge cells can overflow; a cell overflow ends the call
    if (left > 0 && since_check >= kGrowCheckSteps) {
      since_check = 0;
      std::vector<uint32_t> st;
      int ofw = -1;
      TB_TRY(check_grids(c, st, ofw));
      if (ofw >= 0) return status_verdict(c);
    }
  }
  return status_verdict(c);
}

namespace {

// The per-wire reduction of a report from the per-atom terms the last pair
// passes formed at the current positions, copied to the host.
tbsma_status observe_out(tbsma_ctx* c, tbsma_obs* out) {
  const double rhs = 0.5 * c->P.r0;
  const double v_atom = 4.0 / 3.0 * 3.141592653589793238462643383279 * rhs * rhs * rhs;
  k_observe<<<std::min(c->W, 65535), 256, 0, c->stream>>>(
      c->W, c->wd, c->meta, c->N, c->e_atom, c->w_atom, c->v, c->d_grip, c->n_rebuilds,
      c->wire_status, c->steps_done, c->P.mass * kMvv2e, v_atom, c->obs_d);
  TB_CUDA(c, cudaGetLastError());
  TB_CUDA(c, cudaMemcpyAsync(out, c->obs_d, sizeof(tbsma_obs) * c->W, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  // the grid-clamp mark is not a fault, and status_verdict grows the grid now
  for (int w = 0; w < c->W; ++w) out[w].status &= ~(int32_t)kWireGridClamp;
  return status_verdict(c);
}

}  // namespace

tbsma_status tbsma_reduce_observables(tbsma_ctx* c, tbsma_obs* out) {
  NvtxRange range_("tbsma_reduce_observables");
  if (!c || !out) return TBSMA_EINVAL;
  // re-pack, rebuild flagged wires, both passes with the per-atom terms
  TB_TRY(launch_captured(c, c->obs_graph, [c](cudaStream_t s) {
    TB_TRY(launch_pack(c, s, 1));
    TB_TRY(launch_nl(c, s, 0, 0, nullptr));
    return launch_pair<true>(c, s, c->prec);
  }));
  return observe_out(c, out);
}

tbsma_status tbsma_step_observe(tbsma_ctx* c, int64_t n_steps, double dt_fs, tbsma_obs* out) {
  NvtxRange range_("tbsma_step_observe");
  if (!c || !out) return TBSMA_EINVAL;
  if (n_steps < 0 || !(dt_fs > 0.0)) return fail(c, TBSMA_EINVAL, "n_steps < 0 or dt <= 0");
  // Graph replays under the default protocol fold the report into the
  // call's last step; the persistent step kernel, the protocol mode and an
  // empty call step, then report.
  const bool fold = n_steps > 0 && !protocol_mode(c) &&
                    (c->step_mode == TBSMA_STEPS_GRAPH ||
                     (c->step_mode == TBSMA_STEPS_AUTO && persist_blocks(c) == 0));
  if (!fold) {
    const tbsma_status st = tbsma_step_nvt_pull(c, n_steps, dt_fs);
    if (st != TBSMA_OK && st != TBSMA_EWIRE) return st;
    return tbsma_reduce_observables(c, out);
  }
  // the call's kick sequences as tbsma_step_nvt_pull splits them: whole
  // graph chunks, then the remainder (or the last whole chunk)
  const int64_t chunk = std::min<int64_t>(n_steps, kGraphChunk);
  const int64_t last = n_steps % chunk == 0 ? chunk : n_steps % chunk;
  if (n_steps > last) {
    const tbsma_status st = tbsma_step_nvt_pull(c, n_steps - last, dt_fs);
    if (st != TBSMA_OK && st != TBSMA_EWIRE) return st;  // a bad wire stops no other
  }
  TB_TRY(set_dt(c, dt_fs));
  if (last == chunk) {  // a whole chunk: its own graph, replayed
    if (!c->seq_obs_graph || c->seq_obs_steps != chunk || c->seq_obs_dt != dt_fs) {
      if (c->seq_obs_graph) cudaGraphExecDestroy(c->seq_obs_graph);
      c->seq_obs_graph = nullptr;
      TB_TRY(capture_steps(c, (int)chunk, dt_fs, true, &c->seq_obs_graph));
      c->seq_obs_steps = (int)chunk;
      c->seq_obs_dt = dt_fs;
    }
    TB_CUDA(c, cudaGraphLaunch(c->seq_obs_graph, c->stream));
  } else {
    TB_TRY(enqueue_steps(c, c->stream, (int)last, dt_fs, nullptr, true));
  }
  c->steps_done += last;
  return observe_out(c, out);
}

tbsma_status tbsma_force_check(tbsma_ctx* c, tbsma_fcheck* out) {
  NvtxRange range_("tbsma_force_check");
  if (!c || !out) return TBSMA_EINVAL;
  TB_TRY(launch_captured(c, c->fc_graph, [c](cudaStream_t s) {
    TB_TRY(launch_pack(c, s, 1));
    TB_TRY(launch_nl(c, s, 0, 0, nullptr));
    TB_TRY(launch_pair<false>(c, s, TBSMA_MIXED));
    TB_TRY(launch_pair<true>(c, s, TBSMA_FP64, true));
    k_force_check_tiles<<<(unsigned)(c->NS / 256), 256, 0, s>>>(c->NS, c->N, c->perm, c->f32,
                                                                c->f64, c->s_atom, c->fc_part);
    k_force_check<<<std::min(c->W, 65535), 256, 0, s>>>(c->W, c->wd, c->fc_part, c->fcheck_d);
    TB_CUDA(c, cudaGetLastError());
    return TBSMA_OK;
  }));
  TB_CUDA(c, cudaMemcpyAsync(out, c->fcheck_d, sizeof(tbsma_fcheck) * c->W, cudaMemcpyDeviceToHost,
                             c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  return status_verdict(c);
}

tbsma_status tbsma_upload_state(tbsma_ctx* c, const double* x_host, const double* v_host) {
  NvtxRange range_("tbsma_upload_state");
  if (!c) return TBSMA_EINVAL;
  const size_t bytes = 3 * (size_t)c->N * sizeof(double);
  if (x_host) TB_CUDA(c, cudaMemcpyAsync(c->x, x_host, bytes, cudaMemcpyHostToDevice, c->stream));
  if (v_host) TB_CUDA(c, cudaMemcpyAsync(c->v, v_host, bytes, cudaMemcpyHostToDevice, c->stream));
  if (x_host) {
    TB_TRY(refresh(c, 0));
    TB_TRY(launch_pair<false>(c, c->stream, c->prec));
  }
  return TBSMA_OK;
}

tbsma_status tbsma_download_state(tbsma_ctx* c, double* x_host, double* v_host) {
  NvtxRange range_("tbsma_download_state");
  if (!c) return TBSMA_EINVAL;
  const size_t bytes = 3 * (size_t)c->N * sizeof(double);
  if (x_host) TB_CUDA(c, cudaMemcpyAsync(x_host, c->x, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (v_host) TB_CUDA(c, cudaMemcpyAsync(v_host, c->v, bytes, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  return TBSMA_OK;
}

tbsma_status tbsma_get_wire_status(tbsma_ctx* c, int32_t* status_host) {
  if (!c || !status_host) return TBSMA_EINVAL;
  std::vector<uint32_t> st;
  TB_TRY(read_status(c, st));
  for (int w = 0; w < c->W; ++w) status_host[w] = (int32_t)st[w];
  return TBSMA_OK;
}

int32_t tbsma_nbr_capacity(const tbsma_ctx* c) { return c ? c->cap : 0; }

tbsma_status tbsma_get_rebuild_chains(tbsma_ctx* c, int64_t* n) {
  if (!c || !n) return TBSMA_EINVAL;
  TB_CUDA(c, cudaMemcpyAsync(n, c->chains, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  return TBSMA_OK;
}

tbsma_status tbsma_get_neighbors(tbsma_ctx* c, int32_t* n_nbr, int32_t* nbr, int32_t cap) {
  if (!c || cap != c->cap) return TBSMA_EINVAL;
  if (!n_nbr && !nbr) return TBSMA_OK;
  k_list_rows<<<grid_for(c->N * c->cap, 256), 256, 0, c->stream>>>(c->N, c->cap, c->nbr, c->n_nbr,
                                                                   c->slot_of, n_nbr, nbr);
  TB_CUDA(c, cudaGetLastError());
  return TBSMA_OK;
}

tbsma_status tbsma_set_launch(tbsma_ctx* c, int32_t block_threads, int32_t window_atoms) {
  if (!c) return TBSMA_EINVAL;
  if (block_threads != 64 && block_threads != 128 && block_threads != 256)
    return fail(c, TBSMA_EINVAL, "block_threads must be 64, 128 or 256");
  if (window_atoms < 0 || window_atoms > kMaxWindow)
    return fail(c, TBSMA_EINVAL, "window_atoms must be in [0, 4096]");
  c->block = block_threads;
  c->wcap = window_atoms;
  drop_graph(c);
  return TBSMA_OK;
}

tbsma_status tbsma_set_protocol(tbsma_ctx* c, const tbsma_protocol* p) {
  if (!c || !p) return TBSMA_EINVAL;
  if (p->thermostat != TBSMA_THERMO_LANGEVIN && p->thermostat != TBSMA_THERMO_NOSE_HOOVER)
    return fail(c, TBSMA_EINVAL, "unknown thermostat");
  if (p->pull != TBSMA_PULL_CONTINUOUS && p->pull != TBSMA_PULL_STEPWISE)
    return fail(c, TBSMA_EINVAL, "unknown pull mode");
  if (p->thermostat == TBSMA_THERMO_NOSE_HOOVER && !(p->tau_fs > 0.0 && std::isfinite(p->tau_fs)))
    return fail(c, TBSMA_EINVAL, "tau_fs must be positive");
  if (p->pull == TBSMA_PULL_STEPWISE && (p->pull_interval < 1 || !std::isfinite(p->pull_step)))
    return fail(c, TBSMA_EINVAL, "stepwise pull needs pull_interval >= 1 and a finite pull_step");
  if (!(p->t_start >= 0.0 && std::isfinite(p->t_start)) || p->ramp_steps < 0 || p->ramp_start < 0)
    return fail(c, TBSMA_EINVAL, "ramp needs t_start >= 0, ramp_steps >= 0 and ramp_start >= 0");
  if (!(p->baro_tau_fs >= 0.0 && std::isfinite(p->baro_tau_fs)))
    return fail(c, TBSMA_EINVAL, "baro_tau_fs must be >= 0 (0 = no barostat)");
  if (p->baro_tau_fs > 0.0 &&
      !(p->baro_modulus > 0.0 && std::isfinite(p->baro_modulus) && std::isfinite(p->baro_pressure) &&
        p->baro_drag >= 0.0 && std::isfinite(p->baro_drag)))
    return fail(c, TBSMA_EINVAL,
                "the barostat needs baro_modulus > 0, baro_drag >= 0 and a finite baro_pressure");
  c->proto = *p;
  drop_graph(c);
  TB_CUDA(c, cudaMemsetAsync(c->nh, 0, sizeof(NhState) * c->W, c->stream));
  return TBSMA_OK;
}

tbsma_status tbsma_eam_cubics(const double* y, int32_t n, double* coeffs) {
  if (!y || !coeffs || n < 3 || n > kMaxEamSamples) return TBSMA_EINVAL;
  const std::vector<double> c = hermite_cubics(y, n);
  std::copy(c.begin(), c.end(), coeffs);
  return TBSMA_OK;
}

tbsma_status tbsma_set_eam(tbsma_ctx* c, const tbsma_eam* t) {
  NvtxRange range_("tbsma_set_eam");
  if (!c) return TBSMA_EINVAL;
  constexpr int kMaxSamples = kMaxEamSamples;
  if (t) {
    if (!t->F || !t->f || !t->phi) return fail(c, TBSMA_EINVAL, "null EAM table");
    if (t->n_rho < 3 || t->n_r < 3 || t->n_rho > kMaxSamples || t->n_r > kMaxSamples)
      return fail(c, TBSMA_EINVAL, "EAM tables need 3 to 2^22 samples");
    if (!(t->d_rho > 0.0 && std::isfinite(t->d_rho) && t->d_r > 0.0 && std::isfinite(t->d_r)))
      return fail(c, TBSMA_EINVAL, "EAM grid spacings must be positive and finite");
    if ((t->n_r - 1) * t->d_r < c->P.r_cut)
      return fail(c, TBSMA_EINVAL, "the EAM r grid ends before r_cut");
    for (int k = 0; k < t->n_rho; ++k)
      if (!std::isfinite(t->F[k])) return fail(c, TBSMA_EINVAL, "non-finite EAM sample");
    for (int k = 0; k < t->n_r; ++k)
      if (!std::isfinite(t->f[k]) || !std::isfinite(t->phi[k]))
        return fail(c, TBSMA_EINVAL, "non-finite EAM sample");
  }
  // kernels in flight (or a captured graph) may hold the old tables
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  drop_graph(c);
  for (void* p : c->eam_allocs) cudaFree(p);
  c->eam_allocs.clear();
  c->eam = EamDev{};
  c->eam_on = false;
  if (t) {
    const tbsma_status st = upload_eam(c, t);
    if (st != TBSMA_OK) {
      // the earlier tables are gone: leave the context on TB-SMA with its forces
      const std::string msg = c->err;
      if (refresh(c, 0) == TBSMA_OK) launch_pair<false>(c, c->stream, c->prec);
      c->err = msg;
      return st;
    }
  }
  TB_TRY(refresh(c, 0));
  TB_TRY(launch_pair<false>(c, c->stream, c->prec));
  return TBSMA_OK;
}

tbsma_status tbsma_get_barostat(tbsma_ctx* c, double* lambda, double* zeta) {
  if (!c) return TBSMA_EINVAL;
  std::vector<BaroState> b(c->W);
  TB_CUDA(c, cudaMemcpyAsync(b.data(), c->baro, sizeof(BaroState) * c->W, cudaMemcpyDeviceToHost,
                             c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int w = 0; w < c->W; ++w) {
    if (lambda) lambda[w] = b[w].lam;
    if (zeta) zeta[w] = b[w].zeta;
  }
  return TBSMA_OK;
}

tbsma_status tbsma_get_thermostat(tbsma_ctx* c, double* xi, double* eta) {
  if (!c) return TBSMA_EINVAL;
  std::vector<NhState> st(c->W);
  TB_CUDA(c, cudaMemcpyAsync(st.data(), c->nh, sizeof(NhState) * c->W, cudaMemcpyDeviceToHost,
                             c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  const bool on = nose_hoover(c);
  for (int w = 0; w < c->W; ++w) {
    if (xi) xi[w] = on ? st[w].xi : 0.0;
    if (eta) eta[w] = on ? st[w].eta : 0.0;
  }
  return TBSMA_OK;
}

tbsma_status tbsma_wire_topology(tbsma_ctx* c, tbsma_topology* out, int32_t* labels) {
  NvtxRange range_("tbsma_wire_topology");
  if (!c || !out) return TBSMA_EINVAL;
  if (!c->uf_parent) {
    if (alloc(c, &c->uf_parent, c->N) != TBSMA_OK || alloc(c, &c->uf_err, 1) != TBSMA_OK ||
        alloc(c, &c->topo_d, c->W) != TBSMA_OK)
      return fail(c, TBSMA_ENOMEM, "topology buffers");
  }
  TB_TRY(refresh(c, 0));
  const unsigned g = grid_for(c->N, 256);
  TB_CUDA(c, cudaMemsetAsync(c->uf_err, 0, sizeof(uint32_t), c->stream));
  k_uf_init<<<g, 256, 0, c->stream>>>(c->N, c->uf_parent);
  if (c->prec == TBSMA_MIXED)
    k_uf_link<TBSMA_MIXED><<<grid_for(c->NS, 256), 256, 0, c->stream>>>(c->NS, c->xq, c->xd, c->nbr, c->n_nbr, c->perm,
                                                      c->cap, c->pc, c->uf_parent, c->wait_limit,
                                                      c->uf_err);
  else
    k_uf_link<TBSMA_FP64><<<grid_for(c->NS, 256), 256, 0, c->stream>>>(c->NS, c->xq, c->xd, c->nbr, c->n_nbr, c->perm,
                                                     c->cap, c->pc, c->uf_parent, c->wait_limit,
                                                     c->uf_err);
  k_uf_compress<<<g, 256, 0, c->stream>>>(c->N, c->uf_parent, c->wait_limit, c->uf_err);
  k_topology<<<std::min(c->W, 65535), 256, 0, c->stream>>>(c->W, c->wd, c->meta, c->N, c->x,
                                                           c->uf_parent, c->topo_d);
  TB_CUDA(c, cudaGetLastError());
  if (labels)
    TB_CUDA(c, cudaMemcpyAsync(labels, c->uf_parent, sizeof(int32_t) * c->N,
                               cudaMemcpyDeviceToDevice, c->stream));
  uint32_t err = 0;
  TB_CUDA(c, cudaMemcpyAsync(out, c->topo_d, sizeof(tbsma_topology) * c->W, cudaMemcpyDeviceToHost,
                             c->stream));
  TB_CUDA(c, cudaMemcpyAsync(&err, c->uf_err, sizeof err, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  if (err) {
    for (int w = 0; w < c->W; ++w) out[w].status = 2;
    return fail(c, TBSMA_ETIMEOUT, "a bounded union-find loop gave up");
  }
  return TBSMA_OK;
}

tbsma_status tbsma_set_wait_limit(tbsma_ctx* c, int32_t steps) {
  if (!c) return TBSMA_EINVAL;
  if (steps < 1) return fail(c, TBSMA_EINVAL, "the wait limit must be >= 1");
  c->wait_limit = steps;
  return TBSMA_OK;
}

tbsma_status tbsma_set_pair_lanes(tbsma_ctx* c, int32_t lanes) {
  if (!c) return TBSMA_EINVAL;
  if (lanes != 1 && lanes != 2 && lanes != 4) return fail(c, TBSMA_EINVAL, "lanes must be 1, 2 or 4");
  c->lanes = lanes;
  drop_graph(c);
  return TBSMA_OK;
}

tbsma_status tbsma_set_step_mode(tbsma_ctx* c, int32_t mode, int32_t* blocks) {
  if (!c) return TBSMA_EINVAL;
  if (mode != TBSMA_STEPS_AUTO && mode != TBSMA_STEPS_GRAPH && mode != TBSMA_STEPS_PERSISTENT)
    return fail(c, TBSMA_EINVAL, "unknown step mode");
  c->step_mode = mode;
  if (blocks) *blocks = mode == TBSMA_STEPS_GRAPH ? 0 : persist_blocks(c);
  return TBSMA_OK;
}

// Rebuild every wire's list from the current positions and recompute the
// forces: the state after this is a function of (x, v, counters) alone.
tbsma_status rebuild_all(tbsma_ctx* c) {
  TB_TRY(refresh(c, 1));
  TB_TRY(launch_pair<false>(c, c->stream, c->prec));
  return TBSMA_OK;
}

tbsma_status tbsma_save_state(tbsma_ctx* c, double* x_host, double* v_host,
                              tbsma_wire_state* wires, int64_t* step) {
  NvtxRange range_("tbsma_save_state");
  if (!c || !x_host || !v_host || !wires || !step) return TBSMA_EINVAL;
  TB_TRY(rebuild_all(c));
  const size_t bytes = 3 * (size_t)c->N * sizeof(double);
  std::vector<double> dg(c->W);
  std::vector<int32_t> nr(c->W);
  std::vector<uint32_t> ws(c->W);
  std::vector<NhState> nh(c->W);
  std::vector<BaroState> bs(c->W);
  int64_t sc = 0;
  TB_CUDA(c, cudaMemcpyAsync(x_host, c->x, bytes, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(v_host, c->v, bytes, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(dg.data(), c->d_grip, sizeof(double) * c->W, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(nr.data(), c->n_rebuilds, sizeof(int32_t) * c->W, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(ws.data(), c->wire_status, sizeof(uint32_t) * c->W, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(nh.data(), c->nh, sizeof(NhState) * c->W, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(bs.data(), c->baro, sizeof(BaroState) * c->W, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(&sc, c->step_counter, sizeof sc, cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int w = 0; w < c->W; ++w) {
    wires[w].d_grip = dg[w];
    wires[w].xi = nh[w].xi;
    wires[w].eta = nh[w].eta;
    wires[w].log_stretch = bs[w].lam;
    wires[w].stretch_rate = bs[w].zeta;
    wires[w].n_rebuilds = nr[w];
    wires[w].status = ws[w];
  }
  *step = sc;
  if (sc != c->steps_done) return fail(c, TBSMA_ESTATE, "device and host step counts disagree");
  return TBSMA_OK;
}

tbsma_status tbsma_restore_state(tbsma_ctx* c, const double* x_host, const double* v_host,
                                 const tbsma_wire_state* wires, int64_t step) {
  NvtxRange range_("tbsma_restore_state");
  if (!c || !x_host || !v_host || !wires || step < 0) return TBSMA_EINVAL;
  const size_t bytes = 3 * (size_t)c->N * sizeof(double);
  std::vector<double> dg(c->W);
  std::vector<int32_t> nr(c->W);
  std::vector<uint32_t> ws(c->W);
  std::vector<NhState> nh(c->W);
  std::vector<BaroState> bs(c->W);
  for (int w = 0; w < c->W; ++w) {
    dg[w] = wires[w].d_grip;
    nr[w] = wires[w].n_rebuilds;
    ws[w] = wires[w].status;
    nh[w] = NhState{wires[w].xi, wires[w].eta, 1.0, 0.f};
    bs[w] = BaroState{wires[w].stretch_rate, wires[w].log_stretch, 0.0, 1.0};
  }
  TB_CUDA(c, cudaMemcpyAsync(c->x, x_host, bytes, cudaMemcpyHostToDevice, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(c->v, v_host, bytes, cudaMemcpyHostToDevice, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(c->d_grip, dg.data(), sizeof(double) * c->W, cudaMemcpyHostToDevice, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(c->n_rebuilds, nr.data(), sizeof(int32_t) * c->W, cudaMemcpyHostToDevice, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(c->wire_status, ws.data(), sizeof(uint32_t) * c->W, cudaMemcpyHostToDevice, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(c->nh, nh.data(), sizeof(NhState) * c->W, cudaMemcpyHostToDevice, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(c->baro, bs.data(), sizeof(BaroState) * c->W, cudaMemcpyHostToDevice, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(c->step_counter, &step, sizeof step, cudaMemcpyHostToDevice, c->stream));
  c->steps_done = step;
  TB_TRY(rebuild_all(c));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));  // the host buffers may be released on return
  return TBSMA_OK;
}

tbsma_status tbsma_run_pass(tbsma_ctx* c, int32_t pass, int32_t reps) {
  NvtxRange range_("tbsma_run_pass");
  if (!c || (pass != 1 && pass != 2) || reps < 1) return TBSMA_EINVAL;
  for (int r = 0; r < reps; ++r) TB_TRY(launch_one_pass(c, c->stream, pass));
  return TBSMA_OK;
}

tbsma_status tbsma_step_profile(tbsma_ctx* c, int64_t n_steps, double dt_fs, double* phase_ms) {
  NvtxRange range_("tbsma_step_profile");
  if (!c || !phase_ms) return TBSMA_EINVAL;
  if (n_steps < 1 || n_steps > (1 << 20) || !(dt_fs > 0.0))
    return fail(c, TBSMA_EINVAL, "n_steps must be in [1, 2^20] and dt > 0");
  if (barostat(c)) return fail(c, TBSMA_EINVAL, "tbsma_step_profile does not cover the barostat's steps");
  TB_TRY(set_dt(c, dt_fs));
  for (int p = 0; p < TBSMA_N_PHASES; ++p) phase_ms[p] = 0.0;
  PhaseMarks pm{c, {}, cudaSuccess};
  pm.mark(c->stream, -1);
  int64_t left = n_steps;
  while (left > 0) {  // sequences of at most one graph chunk, as the graph replays run them
    const int n = (int)std::min<int64_t>(left, kGraphChunk);
    TB_TRY(enqueue_steps(c, c->stream, n, dt_fs, &pm));
    left -= n;
  }
  if (pm.err != cudaSuccess) return cuda_fail(c, pm.err, "cudaEventRecord");
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  for (size_t k = 1; k < pm.tag.size(); ++k) {
    float ms = 0.f;
    TB_CUDA(c, cudaEventElapsedTime(&ms, c->prof_ev[k - 1], c->prof_ev[k]));
    phase_ms[pm.tag[k]] += ms;
  }
  c->steps_done += n_steps;
  return status_verdict(c);
}

tbsma_status tbsma_get_rebuild_stats(tbsma_ctx* c, int64_t* out) {
  if (!c || !out) return TBSMA_EINVAL;
  int64_t h[3] = {0, 0, 0};
  TB_CUDA(c, cudaMemcpyAsync(h, c->chains, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaMemcpyAsync(h + 1, c->rebuilt, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  TB_CUDA(c, cudaStreamSynchronize(c->stream));
  out[0] = h[0];
  out[1] = h[1];
  out[2] = h[2];
  return TBSMA_OK;
}

tbsma_status tbsma_philox4x32_10(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out,
                                 void* cuda_stream) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return TBSMA_EINVAL;
  if (n == 0) return TBSMA_OK;
  k_philox<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(ctr, key, n, out);
  return cudaGetLastError() == cudaSuccess ? TBSMA_OK : TBSMA_ECUDA;
}

tbsma_status tbsma_normals(uint64_t seed, const uint32_t* atoms, int64_t n, int64_t step, uint32_t tag,
                           tbsma_precision precision, double* out, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!atoms || !out)) || step < 0) return TBSMA_EINVAL;
  if (n == 0) return TBSMA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (precision == TBSMA_MIXED)
    k_normals<TBSMA_MIXED><<<grid_for(n, 256), 256, 0, s>>>(seed, atoms, n, (uint64_t)step, tag, out);
  else if (precision == TBSMA_FP64)
    k_normals<TBSMA_FP64><<<grid_for(n, 256), 256, 0, s>>>(seed, atoms, n, (uint64_t)step, tag, out);
  else
    return TBSMA_EINVAL;
  return cudaGetLastError() == cudaSuccess ? TBSMA_OK : TBSMA_ECUDA;
}

const char* tbsma_last_error(const tbsma_ctx* c) { return c ? c->err.c_str() : "null context"; }

void tbsma_destroy(tbsma_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  for (void* p : c->eam_allocs) cudaFree(p);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

}  // extern "C"

// ======================================================= allocation-free forces
// Some callers cannot allocate device memory at the point where they need
// forces: a host application that hands the GPU a fixed, pre-reserved memory
// budget to plug-ins, or a caller in the middle of a latency-critical loop where
// cudaMalloc would synchronise the device.  tbsma_forces_noalloc serves them:
// the FP64 two-pass force of one cluster, pairs found by brute force, with the
// only scratch (1/(2 sqrt(rho_i)) per atom) in the file-scope array below.
// Every GPU that loads this library keeps that array until the process exits.
namespace {

constexpr int kNoAllocMaxAtoms = TBSMA_NOALLOC_MAX_ATOMS;
static __device__ __align__(256) double g_noalloc_inv[kNoAllocMaxAtoms];

__global__ void k_noalloc_density(int n, const double* __restrict__ x, PairConsts pc,
                                  double* __restrict__ inv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xi = x[i], yi = x[n + i], zi = x[2 * n + i];
  double rho = 0.0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    const double dx = x[j] - xi, dy = x[n + j] - yi, dz = x[2 * n + j] - zi;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 <= pc.rc2) {
      const double s = sqrt(r2) / pc.r0 - 1.0;
      rho += pc.xi2 * exp(-2.0 * pc.q * s);
    }
  }
  inv[i] = rho > 0.0 ? 1.0 / (2.0 * sqrt(rho)) : 0.0;
}

__global__ void k_noalloc_force(int n, const double* __restrict__ x, PairConsts pc,
                                const double* __restrict__ inv, double* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xi = x[i], yi = x[n + i], zi = x[2 * n + i], inv_i = inv[i];
  double fx = 0.0, fy = 0.0, fz = 0.0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    const double dx = xi - x[j], dy = yi - x[n + j], dz = zi - x[2 * n + j];
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 <= pc.rc2) {
      const double r = sqrt(r2);
      const double s = r / pc.r0 - 1.0;
      const double phi = pc.A * exp(-pc.p * s);
      const double g = pc.xi2 * exp(-2.0 * pc.q * s);
      const double f = pc.fp * phi - pc.fg * g * (inv_i + inv[j]);
      fx += f * dx / r;
      fy += f * dy / r;
      fz += f * dz / r;
    }
  }
  F[i] = fx;
  F[n + i] = fy;
  F[2 * n + i] = fz;
}

}  // namespace

extern "C" tbsma_status tbsma_forces_noalloc(const tbsma_params* params, int32_t n_atoms,
                                             const double* x, double* f_out, void* cuda_stream) {
  if (!params || n_atoms < 0) return TBSMA_EINVAL;
  if (n_atoms > kNoAllocMaxAtoms) return TBSMA_EOVERFLOW;
  if (n_atoms == 0) return TBSMA_OK;
  if (!x || !f_out) return TBSMA_EINVAL;
  const tbsma_params& P = *params;
  if (!(P.r0 > 0 && P.r_cut > 0 && P.xi > 0 && P.A >= 0)) return TBSMA_EINVAL;
  // A launch error that an earlier, unrelated call left pending is not ours
  // to report or to clear: give up before launching anything.
  if (cudaPeekAtLastError() != cudaSuccess) return TBSMA_ECUDA;
  // The scratch array's device address, looked up on every call with the
  // caller's device (and context) current: in host code the array's name is
  // only a host-side stand-in, and the address differs per device and per
  // context (after cudaDeviceReset the module is loaded again elsewhere).
  // The lookup is a runtime query, cheap next to the n^2 kernels, and keeps
  // no host-side state, so concurrent first calls from several host
  // threads are safe.
  double* inv = nullptr;
  {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_inv) != cudaSuccess || !p) return TBSMA_ECUDA;
    inv = static_cast<double*>(p);
  }
  PairConsts pc{};
  pc.rc2 = P.r_cut * P.r_cut;
  pc.r0 = P.r0;
  pc.A = P.A;
  pc.xi2 = P.xi * P.xi;
  pc.p = P.p;
  pc.q = P.q;
  pc.fp = 2.0 * P.p / P.r0;
  pc.fg = 2.0 * P.q / P.r0;
  pc.inv_r0 = 1.0 / P.r0;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int block = 128;
  const unsigned grid = (unsigned)((n_atoms + block - 1) / block);
  // every inv slot the force pass reads is written by the density pass first
  k_noalloc_density<<<grid, block, 0, s>>>(n_atoms, x, pc, inv);
  if (cudaGetLastError() != cudaSuccess) return TBSMA_ECUDA;
  k_noalloc_force<<<grid, block, 0, s>>>(n_atoms, x, pc, inv, f_out);
  return cudaGetLastError() == cudaSuccess ? TBSMA_OK : TBSMA_ECUDA;
}
