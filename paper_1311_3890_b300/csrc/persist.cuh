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
// protocol (Langevin, continuous pull), TB-SMA or tabulated EAM.
//
// Every barrier wait is bounded: a block that has polled `limit` times
// without seeing the others sets the error word and leaves; every block
// checks the word after each barrier and leaves too, so a lost block never
// hangs the GPU and the host reports TBSMA_ETIMEOUT.
#pragma once

#include "device.cuh"
#include "md.cuh"
#include "nlist.cuh"
#include "pair.cuh"

namespace tbsma {

// State of the grid barrier (device memory, zeroed at init): the arrival
// count, the generation, and the error word.
struct GridBarrier {
  unsigned* count;
  unsigned* gen;
  unsigned* err;
  unsigned limit;  // polls of the generation before giving up
};

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}

// All blocks of the grid meet here.  Returns false when the barrier gave up
// (this block's wait ran out, or another block's did): the caller leaves.
__device__ __forceinline__ bool grid_sync(const GridBarrier& b) {
  __shared__ unsigned s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned ok = 1;
    const unsigned g = ld_volatile(b.gen);
    __threadfence();
    if (atomicAdd(b.count, 1u) == gridDim.x - 1) {
      atomicExch(b.count, 0u);
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      unsigned polls = 0;
      while (ld_volatile(b.gen) == g) {
        if (polls++ >= b.limit || ld_volatile(b.err)) {
          atomicOr(b.err, 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (ld_volatile(b.err)) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
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
  int4* xq_b;
  float half_skin2;
  int32_t* flag;
  int32_t* any_flag;  // [2]: some wire flagged in a step of this parity
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

template <bool EAM, int LANES>
__global__ void __launch_bounds__(256) k_steps_persistent(PersistArgs a) {
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ntiles = a.NS * LANES / blockDim.x;  // pair-pass tiles of blockDim / LANES atoms
  const ProtoDev proto{};
  for (int k = 0; k < a.n_steps; ++k) {
    const long long step = a.step0 + k;
    int32_t* any = a.any_flag + (step & 1);
    // B A O A, pack, displacement check; a sequence's first step opens with a
    // half kick, later ones merge the previous closing and this opening kick
    for (int64_t i = gtid; i < a.N; i += nthreads) {
      if (k % a.seq == 0)
        integrate_mixed_atom<1, false>(i, step, a.N, a.x, a.v, a.f32, a.meta, a.wd, a.wdyn,
                                       a.hk_open, a.hd, a.xq, a.xq_b, a.half_skin2, a.flag, any,
                                       a.wire_status, a.d_grip, proto, nullptr, nullptr);
      else
        integrate_mixed_atom<2, false>(i, step, a.N, a.x, a.v, a.f32, a.meta, a.wd, a.wdyn,
                                       a.hk_full, a.hd, a.xq, a.xq_b, a.half_skin2, a.flag, any,
                                       a.wire_status, a.d_grip, proto, nullptr, nullptr);
    }
    if (!grid_sync(a.bar)) return;
    // list rebuild of the flagged wires (every block sees the same flag word:
    // it was written before the barrier and is cleared only a step later)
    const bool rebuild = ld_volatile(reinterpret_cast<const unsigned*>(any)) != 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.any_flag[(step + 1) & 1] = 0;
    if (rebuild) {
      if (blockIdx.x == 0) nl_plan_body(a.W, a.nw, a.wd, 0, 1, nullptr, step);
      if (!grid_sync(a.bar)) return;
      nl_env_tiles_body(a.nw, a.wd, a.x);
      if (!grid_sync(a.bar)) return;
      nl_env_merge_body(a.nw, a.wd);
      if (!grid_sync(a.bar)) return;
      nl_clear_body(a.nw, a.wd, a.cell_count);
      if (!grid_sync(a.bar)) return;
      nl_bin_body(a.nw, a.wd, a.x, a.N, a.cell_count, a.cell_atoms, a.cell_of, a.wire_status);
      if (!grid_sync(a.bar)) return;
      nl_sort_body(a.nw, a.wd, a.cell_count, a.cell_atoms);
      if (!grid_sync(a.bar)) return;
      nl_build_body<int4>(a.nw, a.wd, a.cell_count, a.cell_atoms, a.cell_of, a.slot_of, a.rlist2u,
                          a.nbr, a.n_nbr, a.cap, a.jrange, a.xq, a.xq_b, a.wire_status);
      nl_build_slab_body(a.nw, a.wd, a.slot_of, a.rlist2, a.slab_range, a.nbr, a.n_nbr, a.cap,
                         a.jrange, a.xq, a.xq_b, a.wire_status);
      if (!grid_sync(a.bar)) return;
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.nw.chains[0] += 1;  // the plan of a step without a rebuild, as in the graph path
    }
    // density pass, force pass
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
      density_f32_tile<false, EAM, LANES>(tile, a.NS, a.xq, a.nbr, a.n_nbr, a.perm, a.jrange, a.cap,
                                   a.wcap, a.pc, nullptr, a.eam);
    if (!grid_sync(a.bar)) return;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
      force_f32_tile<false, EAM, LANES>(tile, a.NS, a.xq, a.nbr, a.n_nbr, a.perm, a.jrange, a.cap, a.wcap,
                                 a.pc, a.f32, a.f32 + a.N, a.f32 + 2 * a.N, nullptr, nullptr,
                                 nullptr, nullptr, a.eam);
    if (!grid_sync(a.bar)) return;
    // a sequence's last step closes with a half kick (each thread kicks the
    // atoms it integrates next, so no barrier is needed before that)
    if ((k + 1) % a.seq == 0 || k + 1 == a.n_steps)
      for (int64_t i = gtid; i < a.N; i += nthreads)
        half_kick_atom<TBSMA_MIXED>(i, a.N, a.v, a.f32, nullptr, a.meta, a.hk_close);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.step_counter[0] = a.step0 + a.n_steps;
    a.any_flag[0] = 0;
    a.any_flag[1] = 0;
  }
}

}  // namespace tbsma
