// The persistent step kernel for small contexts.
//
// A step of the graph path is about ten kernels; for one wire of a few
// thousand to a hundred thousand atoms each of them is a short launch, and
// the launches, not the work, set the time per step.  This kernel runs up
// to a thousand steps (the same B A O A, plan, list rebuild, density, force
// phases, with the same per-atom and per-tile code, and the kicks split
// into the same sequences as the graph replays, hence bitwise the same
// trajectory) in one cooperative launch whose blocks meet at grid-wide
// barriers between the phases.  It covers MIXED contexts under the default
// protocol (Langevin, continuous pull), TB-SMA or tabulated EAM (FP64
// contexts have their own, k_steps_persistent_fp64, at the end).  Two
// barriers per step without a rebuild: after the density pass, and after
// the force pass, in which each atom's thread, its force at hand, also
// integrates the atom's next step (into the other of two position buffers,
// since other blocks may still read this step's).  Each block owning one
// tile keeps the tile's lists, atoms and window in shared memory between
// rebuilds.
//
// Every barrier wait is bounded: a block that has polled `limit` times
// without seeing the others sets the error word and leaves; every block
// polls the word while it waits and leaves too, so a lost block never
// hangs the GPU and the host reports TBSMA_ETIMEOUT.
#pragma once

#include "device.cuh"
#include "md.cuh"
#include "nlist.cuh"
#include "pair.cuh"

namespace tbsma {

// State of the grid barrier (device memory, zeroed before each launch):
// the arrival count and the error word.  The count only grows within a
// launch: the k-th barrier is passed once its low word reaches
// k * gridDim.x, so an arrival is one atomic add and a wait is a poll of one
// word (no reset by the last block, no second word to flip).  Its high word
// counts the arrivals of blocks that flagged a list rebuild, so the barrier
// after an integrate also tells every block whether any atom crossed half
// the skin (no separate flag word to read after it).
struct GridBarrier {
  unsigned long long* count;
  unsigned* err;
  unsigned limit;  // polls before giving up
};

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}
__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// Polls a wait spins before it starts to sleep between polls.
constexpr unsigned kSpinPolls = 256;

// All blocks of the grid meet here; `target` is the block's running count of
// arrivals expected so far (advanced by gridDim.x per barrier, starting at
// 0).  `flag` (shared memory, or null): set by any thread of the block that
// flagged a rebuild since the last barrier; it is read and cleared here, and
// `flagged` receives the launch's running count of flagging arrivals.
// Returns false when the barrier gave up (this block's wait ran out, or
// another block's did and set the error word): the caller leaves.
__device__ __forceinline__ bool grid_sync(const GridBarrier& b, unsigned& target,
                                          int32_t* flag = nullptr, unsigned* flagged = nullptr) {
  __shared__ unsigned s_ok, s_flagged;
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    unsigned ok = 1;
    unsigned long long add = 1;
    if (flag && *flag) {
      add += 1ull << 32;
      *flag = 0;
    }
    __threadfence();  // the block's writes (ordered by the block barrier) before the arrival
    atomicAdd(b.count, add);
    unsigned polls = 0;
    unsigned long long c;
    while ((int)((unsigned)(c = ld_volatile(b.count)) - target) < 0) {
      if (polls++ >= b.limit || ld_volatile(b.err)) {
        atomicOr(b.err, 1u);
        ok = 0;
        break;
      }
      if (polls > kSpinPolls) __nanosleep(64);
    }
    __threadfence();  // the other blocks' writes before this block's next reads
    s_ok = ok;
    s_flagged = (unsigned)(c >> 32);
  }
  __syncthreads();
  if (flagged) *flagged = s_flagged;
  return s_ok != 0;
}

// Everything one launch needs (pointers into the context's memory).
struct PersistArgs {
  int64_t N, NS;
  int W;
  double* x;
  double* v;
  float* f32;
  const uint32_t* meta;
  const WireDev* wd;
  const WireDyn* wdyn;
  float hk_open, hk_full, hd;  // kicks of the first step (dt/2) and of later steps (dt), dt/2
  double hk_close;             // the closing half kick
  int4* xq;
  int4* xq2;  // the second position buffer (see k_steps_persistent)
  int4* xq_b;
  float half_skin2;
  int32_t* flag;
  uint32_t* wire_status;
  double* d_grip;
  int64_t* step_counter;
  NlWork nw;
  int32_t* cell_count;
  int32_t* cell_atoms;
  int32_t* cell_of;
  const int32_t* slot_of;
  float rlist2u, rlist2, slab_range;  // list radius^2 in fixed-point units^2 and in A^2
  int16_t* nbr;
  int32_t* n_nbr;
  int cap;
  int2* jrange;
  const int32_t* perm;
  int wcap;
  PairConsts pc;
  EamDev eam;
  int64_t step0;
  int n_steps;
  int seq;  // steps per kick sequence: the graph path's chunk (a call's steps split the same way)
  GridBarrier bar;
};

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// The force pass's epilogue in the persistent kernel: the closing half kick
// if a kick sequence ends at this step, then, unless it is the launch's
// last, the atom's next step (B A O A with the opening half kick after a
// closed sequence, else with the merged closing and opening kicks).  pre()
// brings the atom's state into L1 while the tile computes its force.
struct StepEpilogue {
  int64_t N;
  double* x;
  double* v;
  const uint32_t* meta;
  const WireDev* wd;
  const WireDyn* wdyn;
  float hk_open, hk_full, hd;
  double hk_close;
  const int4* xq_b;
  float half_skin2;
  int32_t* flag;
  uint32_t* wire_status;
  double* d_grip;
  long long step;  // the next step
  bool close, more;
  int4* xq_next;
  int32_t* any_next;
  __device__ void pre(int64_t i) const {
    if (!more) return;
    prefetch_l1(meta + i);
    for (int d = 0; d < 3; ++d) {
      prefetch_l1(x + d * N + i);
      prefetch_l1(v + d * N + i);
    }
  }
  __device__ void operator()(int64_t i, float3 F) const {
    const ProtoDev proto{};
    if (close) half_kick_atom_f(i, N, v, F, meta, hk_close);
    if (!more) return;
    if (close)
      integrate_mixed_atom<1, false>(i, step, N, x, v, F, meta, wd, wdyn, hk_open, hd, xq_next, xq_b,
                                     half_skin2, flag, any_next, wire_status, d_grip, proto, nullptr,
                                     nullptr);
    else
      integrate_mixed_atom<2, false>(i, step, N, x, v, F, meta, wd, wdyn, hk_full, hd, xq_next, xq_b,
                                     half_skin2, flag, any_next, wire_status, d_grip, proto, nullptr,
                                     nullptr);
  }
};

template <bool EAM, int LANES>
__global__ void __launch_bounds__(256) k_steps_persistent(PersistArgs a) {
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ntiles = a.NS * LANES / blockDim.x;  // pair-pass tiles of blockDim / LANES atoms
  // every block owns one tile (or none): its lists, atoms and window stay in
  // shared memory between rebuilds (a block owning several reads them from
  // global memory each pass)
  const bool own = ntiles <= gridDim.x, mine = blockIdx.x < ntiles;
  if (own && mine)
    tile_cache_fill<LANES>(blockIdx.x, a.nbr, a.n_nbr, a.perm, a.jrange, a.cap, a.wcap);
  const ProtoDev proto{};
  unsigned bt = 0;  // barrier target
  __shared__ int32_t s_any;  // some atom of this block flagged a rebuild since the last barrier
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  unsigned flagged = 0, flagged_before = 0;  // flagging arrivals so far, and at the last step
  // The positions of step k go to one of two buffers, the last step's to
  // a.xq (the context's) and earlier ones alternately to a.xq2 and a.xq: an
  // atom's next step is integrated while other blocks may still read this
  // step's positions.
  auto xq_of = [&](int k) { return ((a.n_steps - 1 - k) & 1) ? a.xq2 : a.xq; };
  // B A O A, pack, displacement check of the launch's first step (the first
  // of a sequence: it opens with a half kick)
  for (int64_t i = gtid; i < a.N; i += nthreads)
    integrate_mixed_atom<1, false>(
        i, a.step0, a.N, a.x, a.v, make_float3(a.f32[i], a.f32[a.N + i], a.f32[2 * a.N + i]),
        a.meta, a.wd, a.wdyn, a.hk_open, a.hd, xq_of(0), a.xq_b, a.half_skin2, a.flag, &s_any,
        a.wire_status, a.d_grip, proto, nullptr, nullptr);
  if (!grid_sync(a.bar, bt, &s_any, &flagged)) return;
  for (int k = 0; k < a.n_steps; ++k) {
    const long long step = a.step0 + k;
    int4* xq = xq_of(k);
    // list rebuild of the flagged wires (every block read the same count of
    // flagging arrivals at the barrier after this step's integrate)
    const bool rebuild = flagged != flagged_before;
    flagged_before = flagged;
    if (rebuild) {
      if (blockIdx.x == 0) nl_plan_body(a.W, a.nw, a.wd, 0, 1, nullptr, step);
      if (!grid_sync(a.bar, bt)) return;
      nl_env_tiles_body(a.nw, a.wd, a.x);
      if (!grid_sync(a.bar, bt)) return;
      nl_env_merge_body(a.nw, a.wd);
      if (!grid_sync(a.bar, bt)) return;
      // the cell build's phases only when a wire takes it (the count read from
      // L2, so that every block takes the same branch and meets the same
      // barriers)
      if (__ldcg(a.nw.n_cell) > 0) {
        nl_clear_body(a.nw, a.wd, a.cell_count);
        if (!grid_sync(a.bar, bt)) return;
        nl_bin_body(a.nw, a.wd, a.x, a.N, a.cell_count, a.cell_atoms, a.cell_of, a.wire_status);
        if (!grid_sync(a.bar, bt)) return;
        nl_sort_body(a.nw, a.wd, a.cell_count, a.cell_atoms);
        if (!grid_sync(a.bar, bt)) return;
      }
      nl_build_body<int4>(a.nw, a.wd, a.cell_count, a.cell_atoms, a.cell_of, a.slot_of, a.rlist2u,
                          a.nbr, a.n_nbr, a.cap, a.jrange, xq, a.xq_b, a.wire_status);
      nl_build_slab_body(a.nw, a.wd, a.slot_of, a.rlist2, a.slab_range, a.nbr, a.n_nbr, a.cap,
                         a.jrange, xq, a.xq_b, a.wire_status);
      if (!grid_sync(a.bar, bt)) return;
      // the builds used the shared memory: refill the tile's cache
      if (own && mine)
        tile_cache_fill<LANES>(blockIdx.x, a.nbr, a.n_nbr, a.perm, a.jrange, a.cap, a.wcap);
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.nw.chains[0] += 1;  // the plan of a step without a rebuild, as in the graph path
    }
    // density pass
    if (own) {
      if (mine)
        density_f32_tile<false, EAM, LANES, true>(blockIdx.x, a.NS, xq, a.nbr, a.n_nbr, a.perm,
                                                  a.jrange, a.cap, a.wcap, a.pc, nullptr, a.eam);
    } else {
      for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        density_f32_tile<false, EAM, LANES>(tile, a.NS, xq, a.nbr, a.n_nbr, a.perm, a.jrange, a.cap,
                                            a.wcap, a.pc, nullptr, a.eam);
    }
    if (!grid_sync(a.bar, bt)) return;
    // force pass; with its force at hand, each atom's thread closes the kick
    // sequence if it ends here (half kick) and integrates the atom's next
    // step: B A O A with the opening half kick after a closed sequence, else
    // with the merged closing and opening kicks
    const bool close = (k + 1) % a.seq == 0 || k + 1 == a.n_steps;
    const bool more = k + 1 < a.n_steps;
    int4* xq_next = xq_of(k + 1);
    int32_t* any_next = &s_any;
    const StepEpilogue epi{a.N,     a.x,          a.v,         a.meta,  a.wd,     a.wdyn,
                           a.hk_open, a.hk_full,  a.hd,        a.hk_close, a.xq_b, a.half_skin2,
                           a.flag,  a.wire_status, a.d_grip,   step + 1, close,    more,
                           xq_next, any_next};
    if (own) {
      if (mine)
        force_f32_tile<false, EAM, LANES, true>(blockIdx.x, a.NS, xq, a.nbr, a.n_nbr, a.perm,
                                                a.jrange, a.cap, a.wcap, a.pc, a.f32, a.f32 + a.N,
                                                a.f32 + 2 * a.N, nullptr, nullptr, nullptr, nullptr,
                                                a.eam, epi);
    } else {
      for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        force_f32_tile<false, EAM, LANES>(tile, a.NS, xq, a.nbr, a.n_nbr, a.perm, a.jrange, a.cap,
                                          a.wcap, a.pc, a.f32, a.f32 + a.N, a.f32 + 2 * a.N, nullptr,
                                          nullptr, nullptr, nullptr, a.eam, epi);
    }
    if (!grid_sync(a.bar, bt, &s_any, &flagged)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.step_counter[0] = a.step0 + a.n_steps;
}

}  // namespace tbsma

namespace tbsma {

// The persistent step kernel of FP64 contexts: the same step as the graph
// path's (integrate, plan and cell-grid rebuild of the flagged wires,
// density pass, force pass, the closing half kick at a sequence's end) with
// the same per-atom and per-slot code, in one cooperative launch per call
// of up to a thousand steps, in blocks of kPair64Block threads.  The FP64
// passes run kLanes64 lanes per slot, strided over the grid's lane groups;
// three barriers per step without a rebuild.
struct PersistArgs64 {
  int64_t N, NS;
  int W;
  double* x;
  double* v;
  double* f64;
  const uint32_t* meta;
  const WireDev* wd;
  const WireDyn* wdyn;
  double dt, inv_m, hk_close;
  int4* xq;
  double4_32a* xd;
  const int4* xq_b;
  double4_32a* xd_b;
  double half_skin2;
  int32_t* flag;
  uint32_t* wire_status;
  double* d_grip;
  int64_t* step_counter;
  NlWork nw;
  int32_t* cell_count;
  int32_t* cell_atoms;
  int32_t* cell_of;
  const int32_t* slot_of;
  float rlist2;
  int16_t* nbr;
  int32_t* n_nbr;
  int cap;
  int2* jrange;
  const int32_t* perm;
  PairConsts pc;
  double* inv64;
  EamDev eam;
  int64_t step0;
  int n_steps;
  int seq;
  GridBarrier bar;
};

template <bool EAM>
__global__ void __launch_bounds__(kPair64Block) k_steps_persistent_fp64(PersistArgs64 a) {
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ngroups = nthreads / kLanes64, ggroup = gtid / kLanes64;
  const int q = threadIdx.x % kLanes64;
  // the integrate loops deal chunks of 8 consecutive atoms round-robin over
  // the blocks: an atom's step with its FP64 normals costs some 250 FP64
  // operations, which atom-by-thread order would leave to the first few
  // blocks of a small context (1035 atoms: 9 of 148)
  const int64_t i0 = ((int64_t)(threadIdx.x >> 3) * gridDim.x + blockIdx.x) * 8 + (threadIdx.x & 7);
  const ProtoDev proto{};
  unsigned bt = 0;  // barrier target
  __shared__ int32_t s_any;  // some atom of this block flagged a rebuild since the last barrier
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  unsigned flagged = 0, flagged_before = 0;
  for (int k = 0; k < a.n_steps; ++k) {
    const long long step = a.step0 + k;
    // B A O A, pack, displacement check; a sequence's first step opens with a
    // half kick, later ones merge the previous closing and this opening kick
    for (int64_t i = i0; i < a.N; i += nthreads) {
      if (k % a.seq == 0)
        integrate_atom<TBSMA_FP64, 1, false>(i, step, a.N, a.x, a.v, nullptr, a.f64, a.meta, a.wd,
                                             a.wdyn, a.dt, a.inv_m, a.xq, a.xd, a.xq_b, a.xd_b,
                                             a.half_skin2, a.flag, a.wire_status, a.d_grip, proto,
                                             nullptr, nullptr, &s_any);
      else
        integrate_atom<TBSMA_FP64, 2, false>(i, step, a.N, a.x, a.v, nullptr, a.f64, a.meta, a.wd,
                                             a.wdyn, a.dt, a.inv_m, a.xq, a.xd, a.xq_b, a.xd_b,
                                             a.half_skin2, a.flag, a.wire_status, a.d_grip, proto,
                                             nullptr, nullptr, &s_any);
    }
    if (!grid_sync(a.bar, bt, &s_any, &flagged)) return;
    const bool rebuild = flagged != flagged_before;
    flagged_before = flagged;
    if (rebuild) {
      if (blockIdx.x == 0) nl_plan_body(a.W, a.nw, a.wd, 0, 1, nullptr, step);
      if (!grid_sync(a.bar, bt)) return;
      nl_clear_body(a.nw, a.wd, a.cell_count);
      if (!grid_sync(a.bar, bt)) return;
      nl_bin_body(a.nw, a.wd, a.x, a.N, a.cell_count, a.cell_atoms, a.cell_of, a.wire_status);
      if (!grid_sync(a.bar, bt)) return;
      nl_sort_body(a.nw, a.wd, a.cell_count, a.cell_atoms);
      if (!grid_sync(a.bar, bt)) return;
      nl_build_body<double4_32a>(a.nw, a.wd, a.cell_count, a.cell_atoms, a.cell_of, a.slot_of,
                                 a.rlist2, a.nbr, a.n_nbr, a.cap, a.jrange, a.xd, a.xd_b,
                                 a.wire_status);
      if (!grid_sync(a.bar, bt)) return;
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.nw.chains[0] += 1;  // the plan of a step without a rebuild, as in the graph path
    }
    for (int64_t t = ggroup; t < a.NS; t += ngroups)
      density_f64_slot<false, false, EAM>(t, q, a.xd, a.xq, a.nbr, a.n_nbr, a.perm, a.cap, a.pc,
                                          a.inv64, nullptr, a.eam);
    if (!grid_sync(a.bar, bt)) return;
    for (int64_t t = ggroup; t < a.NS; t += ngroups)
      force_f64_slot<false, false, EAM>(t, q, a.N, a.xd, a.xq, a.nbr, a.n_nbr, a.perm, a.cap, a.pc,
                                        a.inv64, a.f64, nullptr, nullptr, nullptr, nullptr, a.eam);
    if (!grid_sync(a.bar, bt)) return;
    // a sequence's last step closes with a half kick (each thread kicks the
    // atoms it integrates next, so no barrier is needed before that)
    if ((k + 1) % a.seq == 0 || k + 1 == a.n_steps)
      for (int64_t i = i0; i < a.N; i += nthreads)
        half_kick_atom<TBSMA_FP64>(i, a.N, a.v, nullptr, a.f64, a.meta, a.hk_close);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.step_counter[0] = a.step0 + a.n_steps;
}

}  // namespace tbsma
