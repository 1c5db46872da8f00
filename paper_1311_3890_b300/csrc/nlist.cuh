// Per-wire cell lists and Verlet neighbour lists (Results, "TB-SMA
// benchmarks": a neighbour list with buffer radius r_buff; atoms kept in
// their [100] order, no re-sorting).
//
// Only wires whose rebuild flag is set are processed.  k_nl_plan turns the
// flags into a compact work list (flagged wires with prefix sums of their
// cells and atoms); the other kernels stride over that list, so a step in
// which no wire moved far enough costs four near-empty launches.
//
// Cells: a grid per wire (edge >= list radius), atoms outside the grid
// clamped into edge cells (clamping is monotone, so two atoms within one
// edge of each other still land in adjacent cells) and the wire marked
// (kWireGridClamp) so that the host grows its grid.  Each cell holds up to
// kCellCap atom indices, sorted ascending so that the list order, and hence
// every force sum, is deterministic.
#pragma once

#include <climits>

#include "device.cuh"

namespace tbsma {

struct NlWork {
  int32_t* flag;        // [W] rebuild requested
  int32_t* wl_wire;     // [W] flagged wires
  int64_t* wl_cell;     // [W+1] prefix of their cell counts
  int64_t* wl_atom;     // [W+1] prefix of their atom counts
  int64_t* wl_tile;     // [W+1] prefix of their tiles (kSlotTile consecutive atoms each)
  float2* xenv;         // [N] along the atom order: prefix max and suffix min of x (envelopes)
  float2* tenv;         // [NS / kSlotTile] per tile: max and min of x (envelopes)
  uint32_t* wdis;       // [W] disorder of the atom order along x, A (FP32 bits; envelopes)
  float4* xf;           // [3 NS / 4] slab-build candidates: per group of four slots, x, y, z
                        // (four FP32 coordinates relative to the wire's origin each)
  int64_t N;            // atoms (the stride of the position planes)
  int slab_ok;          // the context may use the slab build (MIXED)
  float max_disorder;   // largest disorder for which a wire takes the slab build, A
  int32_t* n_flagged;   // [1]
  int32_t* n_rebuilds;  // [W]
  int64_t* chains;      // [1] launches of the rebuild chain (clear, bin, sort, build)
  int64_t* last_build;  // [W] step of the wire's last list build
  uint8_t* banked;      // [W] the wire's rows in bank-group order (k_nl_build) at this build
  int64_t* rebuilt;     // [2] wires and atoms whose lists were built, accumulated
  // the flagged wires that take the cell build (MIXED: those the envelopes
  // do not give to the slab build; written by the last block of the envelope
  // merge), with the prefixes of their cells and atoms
  int32_t* cl_wire;        // [W]
  int64_t* cl_cell;        // [W+1]
  int64_t* cl_atom;        // [W+1]
  int32_t* n_cell;         // [1]
  uint32_t* merge_done;    // [1] envelope-merge blocks done (zeroed by the plan)
};

// Shortest life (steps) of a wire's previous list for which the cell build
// puts its rebuilt rows in bank-group order (see k_nl_build; the slab build
// always does).
constexpr int64_t kBankedInterval = 128;

// Atoms per tile of the pair passes (see k_slot_order); the slab build
// works on the same tiles.
constexpr int kSlotTile = 256;

// Whether wire w takes the slab build at this rebuild (its disorder, from
// k_nl_env_merge, small enough; NaN positions give a NaN disorder: cells).
__device__ __forceinline__ bool use_slab(const NlWork& nw, int w) {
  return nw.slab_ok && __uint_as_float(nw.wdis[w]) <= nw.max_disorder;
}

// The flagged wires the cell build (clear, bin, sort, build) works on: all
// of them in a context without the slab build, else the list the envelope
// merge compacted (so the cell build's kernels walk no slab wire's cells or
// atoms; most steps they have none to walk).
struct CellList {
  int n;
  const int32_t* wire;
  const int64_t* cell;
  const int64_t* atom;
};
__device__ __forceinline__ CellList cell_list(const NlWork& nw) {
  if (!nw.slab_ok) return CellList{nw.n_flagged[0], nw.wl_wire, nw.wl_cell, nw.wl_atom};
  return CellList{nw.n_cell[0], nw.cl_wire, nw.cl_cell, nw.cl_atom};
}

// Binary search: largest k < nf with pre[k] <= idx.
__device__ __forceinline__ int wl_find(const int64_t* pre, int nf, int64_t idx) {
  int lo = 0, hi = nf - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= idx) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Inclusive warp scan.
template <typename T>
__device__ __forceinline__ T warp_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive block scan of four counters (blockDim.x a multiple of 32, at
// most 1024); returns the block totals in tot[4].
__device__ __forceinline__ void block_scan4(int64_t (&v)[4], int64_t* tot) {
  __shared__ int64_t s[4][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    inc[q] = warp_scan(v[q]);
    if (lane == 31) s[q][warp] = inc[q];
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t x = lane < nw ? s[q][lane] : 0;
      const int64_t sx = warp_scan(x);
      s[q][lane] = sx - x;  // exclusive prefix of the warp totals
      if (lane == 31) tot[q] = sx;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = s[q][warp] + inc[q] - v[q];
}

// One block: compact flagged wires, clear their flags, count the rebuild,
// and (in the step loop) advance the step counter; `steps` is the step
// count at this plan.  (Skipping the rest of the chain through a
// conditional graph node when no wire is flagged measured 5 us per step
// slower than launching its kernels, which return at once.)
__device__ __forceinline__ void nl_plan_body(int W, NlWork nw, const WireDev* __restrict__ wd,
                                             int force_all, int count_rebuild,
                                             int64_t* step_counter, int64_t steps) {
  __shared__ int64_t tot[4];
  const int t = threadIdx.x;
  const int chunk = (W + (int)blockDim.x - 1) / (int)blockDim.x;
  const int w0 = min(W, t * chunk), w1 = min(W, w0 + chunk);
  auto tiles_of = [](int n) { return (int64_t)((n + kSlotTile - 1) / kSlotTile); };
  int64_t v[4] = {0, 0, 0, 0};  // cells, atoms, tiles, wires
  for (int w = w0; w < w1; ++w) {
    if (force_all || nw.flag[w]) {
      v[0] += (int64_t)wd[w].nc[0] * wd[w].nc[1] * wd[w].nc[2];
      v[1] += wd[w].n;
      v[2] += tiles_of(wd[w].n);
      v[3] += 1;
    }
  }
  block_scan4(v, tot);
  int64_t c_pre = v[0], a_pre = v[1], t_pre = v[2], k = v[3];
  for (int w = w0; w < w1; ++w) {
    if (force_all || nw.flag[w]) {
      nw.wl_wire[k] = w;
      nw.wl_cell[k] = c_pre;
      nw.wl_atom[k] = a_pre;
      nw.wl_tile[k] = t_pre;
      c_pre += (int64_t)wd[w].nc[0] * wd[w].nc[1] * wd[w].nc[2];
      a_pre += wd[w].n;
      t_pre += tiles_of(wd[w].n);
      ++k;
      nw.flag[w] = 0;
      if (count_rebuild) nw.n_rebuilds[w] += 1;
      // bank-group row order when the previous list lived long enough to
      // repay it (always on a full rebuild: init, checkpoint save / restore)
      nw.banked[w] = force_all || steps - nw.last_build[w] >= kBankedInterval;
      nw.last_build[w] = steps;
    }
  }
  if (t == 0) {
    const int nf = (int)tot[3];
    nw.n_flagged[0] = nf;
    nw.n_cell[0] = 0;      // the envelope merge lists the cell-build wires, if any
    nw.merge_done[0] = 0;
    nw.wl_cell[nf] = tot[0];
    nw.wl_atom[nf] = tot[1];
    nw.wl_tile[nf] = tot[2];
    if (step_counter) step_counter[0] += 1;
    nw.chains[0] += 1;
    nw.rebuilt[0] += nf;
    nw.rebuilt[1] += tot[1];
  }
}

__global__ void __launch_bounds__(1024)
    k_nl_plan(int W, NlWork nw, const WireDev* __restrict__ wd, int force_all, int count_rebuild,
              int64_t* step_counter, const int64_t* __restrict__ steps_now) {
  nl_plan_body(W, nw, wd, force_all, count_rebuild, step_counter, steps_now[0]);
}

__device__ __forceinline__ void nl_clear_body(NlWork nw, const WireDev* __restrict__ wd,
                                              int32_t* cell_count) {
  const CellList cl = cell_list(nw);
  if (cl.n == 0) return;
  const int64_t total = cl.cell[cl.n];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = wl_find(cl.cell, cl.n, idx);
    const WireDev& w = wd[cl.wire[k]];
    cell_count[w.cell_base + (idx - cl.cell[k])] = 0;
  }
}
__global__ void k_nl_clear(NlWork nw, const WireDev* __restrict__ wd, int32_t* cell_count) {
  nl_clear_body(nw, wd, cell_count);
}

// Cell coordinate along one axis, clamped into the grid; `out` is set when
// the atom lies outside it.
__device__ __forceinline__ int cell_coord(double rel, double lo, double einv, int n, bool& out) {
  const double u = floor((rel - lo) * einv);
  out |= !(u >= 0.0 && u < (double)n);
  return u >= 0.0 ? (u < (double)n ? (int)u : n - 1) : 0;  // NaN: cell 0 (flagged non-finite elsewhere)
}

// Bin the atoms of flagged wires (positions from the caller's FP64 array).
// The atom's cell coordinates are kept (packed cx << 20 | cy << 10 | cz) for the build.
__device__ __forceinline__ void nl_bin_body(NlWork nw, const WireDev* __restrict__ wd,
                                            const double* __restrict__ x, int64_t N,
                                            int32_t* cell_count, int32_t* cell_atoms,
                                            int32_t* cell_of, uint32_t* wire_status) {
  const CellList cl = cell_list(nw);
  if (cl.n == 0) return;
  const int64_t total = cl.atom[cl.n];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = wl_find(cl.atom, cl.n, idx);
    const int wi = cl.wire[k];
    const WireDev& w = wd[wi];
    const int64_t i = w.offset + (idx - cl.atom[k]);
    bool out = false;
    const int cx = cell_coord(x[i] - w.origin[0], w.glo[0], w.einv[0], w.nc[0], out);
    const int cy = cell_coord(x[N + i] - w.origin[1], w.glo[1], w.einv[1], w.nc[1], out);
    const int cz = cell_coord(x[2 * N + i] - w.origin[2], w.glo[2], w.einv[2], w.nc[2], out);
    if (out) atomicOr(&wire_status[wi], kWireGridClamp);
    const int64_t c = w.cell_base + ((int64_t)cx * w.nc[1] + cy) * w.nc[2] + cz;
    cell_of[i] = (cx << 20) | (cy << 10) | cz;
    const int slot = atomicAdd(&cell_count[c], 1);
    if (slot < kCellCap) cell_atoms[c * kCellCap + slot] = (int32_t)i;
    else atomicOr(&wire_status[wi], kWireCellOverflow);
  }
}
__global__ void k_nl_bin(NlWork nw, const WireDev* __restrict__ wd, const double* __restrict__ x,
                         int64_t N, int32_t* cell_count, int32_t* cell_atoms, int32_t* cell_of,
                         uint32_t* wire_status) {
  nl_bin_body(nw, wd, x, N, cell_count, cell_atoms, cell_of, wire_status);
}

// Warp per flagged cell: sort its members ascending (rank by counting).
__device__ __forceinline__ void nl_sort_body(NlWork nw, const WireDev* __restrict__ wd,
                                             const int32_t* cell_count, int32_t* cell_atoms) {
  const CellList cl = cell_list(nw);
  if (cl.n == 0) return;
  const int64_t total = cl.cell[cl.n];
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t idx = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; idx < total;
       idx += warps) {
    const int k = wl_find(cl.cell, cl.n, idx);
    const int64_t c = wd[cl.wire[k]].cell_base + (idx - cl.cell[k]);
    const int cnt = min(cell_count[c], kCellCap);
    const int32_t m = lane < cnt ? cell_atoms[c * kCellCap + lane] : INT32_MAX;
    int rank = 0;
    for (int l = 0; l < cnt; ++l) rank += (__shfl_sync(0xffffffffu, m, l) < m) ? 1 : 0;
    __syncwarp();
    if (lane < cnt) cell_atoms[c * kCellCap + rank] = m;
  }
}
__global__ void k_nl_sort(NlWork nw, const WireDev* __restrict__ wd, const int32_t* cell_count,
                          int32_t* cell_atoms) {
  nl_sort_body(nw, wd, cell_count, cell_atoms);
}

// Distance test of the list builds on the packed positions: modular fixed
// point in fixed-point units squared (2^-52 A^2; the differences are exact
// and rounded once to FP32, and the power-of-two scale commutes with every
// rounding, so comparing against r_list^2 * 2^52 decides exactly as the
// same test in A^2 would); FP64 copies in an FP64 context, in A^2.
__device__ __forceinline__ float build_d2(int4 a, int4 b) {
  const float dx = (float)(int)((unsigned)b.x - (unsigned)a.x);
  const float dy = (float)(int)((unsigned)b.y - (unsigned)a.y);
  const float dz = (float)(int)((unsigned)b.z - (unsigned)a.z);
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}
__device__ __forceinline__ float build_d2(double4_32a a, double4_32a b) {
  const double dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
  return (float)(dx * dx + dy * dy + dz * dz);
}

// Byte g of a packed vector of eight 8-bit counters.
__device__ __forceinline__ int byte_of(uint64_t v, int g) { return (int)((v >> (8 * g)) & 0xffu); }

// Four threads per atom of a flagged wire (a quad of consecutive lanes);
// thread q of the quad visits the cells c = 0..26 with c % 4 == q, c the
// linear index of the offset (ox, oy, oz) in {-1, 0, 1}^3, each cell's
// (sorted) members in order, four at a time (one 16-byte read of member
// indices, then four independent position reads).  Accepted pairs go to
// the thread's shared-memory buffer; the quad then exchanges its counts and
// writes the row as the concatenation of the four buffers (q = 0 first), so
// the list order is a fixed function of the cell contents.  Splitting the
// 27 cells four ways shortens each thread's chain of dependent reads and
// puts four times as many threads in flight; a rebuild touches only a few
// wires, so the build is bound by that latency.  The list is stored at the
// atom's slot (see k_slot_order).  Also records the range [jmin, jmax] of
// the atom's neighbour indices (the pair passes stage the union of a tile's
// ranges in shared memory) and copies the atom's packed position to the
// build snapshot used by the displacement check.
//
// Row order: the pair passes gather neighbour positions from a shared-memory
// window whose base is a multiple of 8 rows, so row j lies in bank group
// j mod 8 of the 128-bit gathers, and the 8 lanes of a quarter-warp that
// load at the same list position conflict when their rows share a group.
// Each row is therefore emitted so that at position k the atom in lane l
// (its slot mod 8) takes an entry of group (k + l) mod 8 when it has one
// left, else one of the group with the most entries left (nearest to the
// preferred one on ties).  Groups are counted from the wire's first atom
// ((j - offset) mod 8) and a wire's slots start on a tile boundary, so the
// order is a function of the wire alone; within a tile the groups differ
// from the bank groups by one rotation, which keeps the lanes apart.  In a
// CPU replay of thermalised D3-wire lists this brings 8 random rows per
// quarter-warp load (2.6 deep in one bank group) down to ~1.6.  All four
// threads of the quad run the same schedule on packed per-group counters;
// each writes the positions that fall on its own entries.  The schedule
// costs ~1.3 ns per rebuilt atom and the ordered rows save ~10 ps per atom
// and step in the passes, so a wire takes it only when its previous list
// lived at least kBankedInterval steps (k_nl_plan decides from the wire's
// own counters, so the order stays a function of its trajectory); a wire
// that rebuilds more often (298 K) keeps the rows in quad order.
constexpr int kBuildQuad = 4;
template <typename PosT>
__device__ __forceinline__ void nl_build_body(
    NlWork nw, const WireDev* __restrict__ wd, const int32_t* __restrict__ cell_count,
    const int32_t* __restrict__ cell_atoms, const int32_t* __restrict__ cell_of,
    const int32_t* __restrict__ slot_of, float rlist2 /* in build_d2's units */,
    int16_t* __restrict__ nbr, int32_t* __restrict__ n_nbr, int cap, int2* __restrict__ jrange,
    const PosT* __restrict__ pos, PosT* __restrict__ pos_build, uint32_t* wire_status) {
  extern __shared__ int16_t sbuf[];  // [cap][blockDim.x]: entry e of thread x at e * blockDim.x + x
  const CellList cl = cell_list(nw);
  if (cl.n == 0) return;
  const int64_t total = cl.atom[cl.n] * kBuildQuad;
  const int q = threadIdx.x & (kBuildQuad - 1);
  const unsigned quad_mask = 0xfu << (threadIdx.x & 31 & ~(kBuildQuad - 1));
  // the stride is a multiple of 4, so a quad is always entirely in or out
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = idx / kBuildQuad;
    const int k = wl_find(cl.atom, cl.n, a);
    const int wi = cl.wire[k];
    const WireDev& w = wd[wi];
    const int64_t i = w.offset + (a - cl.atom[k]);
    const int32_t ii = (int32_t)i;
    const int co = cell_of[i];
    const int cx = co >> 20, cy = (co >> 10) & 1023, cz = co & 1023;
    const PosT pi = pos[i];
    int cnt_mine = 0, jmin = INT_MAX, jmax = INT_MIN;
    bool far = false;
    auto visit = [&](int32_t j, const PosT& pj) {
      const float d2 = build_d2(pi, pj);
      if (j == ii || d2 > rlist2) return;
      if (j - ii > kMaxOffset || ii - j > kMaxOffset) {
        far = true;  // not representable as an int16 offset: dropped, wire flagged
        return;
      }
      if (cnt_mine < cap) sbuf[cnt_mine * blockDim.x + threadIdx.x] = (int16_t)(j - ii);
      ++cnt_mine;
      jmin = min(jmin, j);
      jmax = max(jmax, j);
    };
    for (int c = q; c < 27; c += kBuildQuad) {
      const int nx = cx + c / 9 - 1, ny = cy + (c / 3) % 3 - 1, nz = cz + c % 3 - 1;
      if (nx < 0 || nx >= w.nc[0] || ny < 0 || ny >= w.nc[1] || nz < 0 || nz >= w.nc[2]) continue;
      const int64_t cn = w.cell_base + ((int64_t)nx * w.nc[1] + ny) * w.nc[2] + nz;
      const int cnt = min(cell_count[cn], kCellCap);
      const int4* members = reinterpret_cast<const int4*>(cell_atoms + cn * kCellCap);
      // slots past the count are stale and stand in as atom i itself, which visit skips
      for (int m = 0; m < cnt; m += 4) {
        const int4 mj = members[m >> 2];
        const int32_t j1 = m + 1 < cnt ? mj.y : ii, j2 = m + 2 < cnt ? mj.z : ii,
                      j3 = m + 3 < cnt ? mj.w : ii;
        const PosT q0 = pos[mj.x], q1 = pos[j1], q2 = pos[j2], q3 = pos[j3];
        visit(mj.x, q0);
        visit(j1, q1);
        visit(j2, q2);
        visit(j3, q3);
      }
    }
    // quad: the four counts, total, index range
    int c4[kBuildQuad], count = 0;
#pragma unroll
    for (int r = 0; r < kBuildQuad; ++r) {
      c4[r] = __shfl_sync(quad_mask, cnt_mine, r, kBuildQuad);
      count += c4[r];
    }
#pragma unroll
    for (int o = 1; o < kBuildQuad; o <<= 1) {
      jmin = min(jmin, __shfl_xor_sync(quad_mask, jmin, o, kBuildQuad));
      jmax = max(jmax, __shfl_xor_sync(quad_mask, jmax, o, kBuildQuad));
    }
    const int64_t t = slot_of[i];
    {
      // the row keeps its first n entries in quad order; this thread holds
      // entries [pre, pre + mine) of them, in its own buffer
      const int n = min(count, cap);
      int pre = 0;
#pragma unroll
      for (int r = 0; r < kBuildQuad; ++r) pre += r < q ? c4[r] : 0;
      const int mine = max(0, min(min(cnt_mine, cap), n - pre));
      const bool banked = nw.banked[wi] != 0;
      if (!banked)
        for (int e = 0; e < mine; ++e) nbr[nbr_slot(t, pre + e, cap)] = sbuf[e * blockDim.x + threadIdx.x];
      const int il = (int)(i - w.offset);
      auto group = [&](int e) { return (il + sbuf[e * blockDim.x + threadIdx.x]) & 7; };
      uint64_t L = 0, P = 0, T = 0, R = 0, C = 0;
      for (int e = 0; banked && e < mine; ++e) L += 1ull << (8 * group(e));
#pragma unroll
      for (int r = 0; r < kBuildQuad; ++r) {
        const uint64_t Lr = __shfl_sync(quad_mask, L, r, kBuildQuad);
        P += r < q ? Lr : 0ull;
        T += Lr;
      }
      const int lane = (int)(t & 7);
      for (int k = 0; banked && k < n; ++k) {
        const int want = (k + lane) & 7;
        int g = want;
        if (byte_of(T, g) == 0) {
          int best = -1;
#pragma unroll
          for (int d = 0; d < 8; ++d) {
            const int h = (want + d) & 7;
            if (byte_of(T, h) > best) {
              best = byte_of(T, h);
              g = h;
            }
          }
        }
        const int r = byte_of(R, g), p = byte_of(P, g);
        R += 1ull << (8 * g);
        T -= 1ull << (8 * g);
        if (r >= p && r < p + byte_of(L, g)) {  // the position falls on one of my entries
          int cur = min(byte_of(C, g), mine - 1);  // mine >= 1 here; stays inside the buffer
          while (cur + 1 < mine && group(cur) != g) ++cur;
          nbr[nbr_slot(t, k, cap)] = sbuf[cur * blockDim.x + threadIdx.x];
          C = (C & ~(0xffull << (8 * g))) | ((uint64_t)(cur + 1) << (8 * g));
        }
      }
    }
    if (far || (q == 0 && count > cap)) atomicOr(&wire_status[wi], kWireNbrOverflow);
    if (q == 0) {
      n_nbr[t] = min(count, cap);
      jrange[t] = make_int2(jmin, jmax);
      pos_build[i] = pi;
    }
  }
}
template <typename PosT>
__global__ void __launch_bounds__(256)
    k_nl_build(NlWork nw, const WireDev* __restrict__ wd, const int32_t* __restrict__ cell_count,
               const int32_t* __restrict__ cell_atoms, const int32_t* __restrict__ cell_of,
               const int32_t* __restrict__ slot_of, float rlist2, int16_t* __restrict__ nbr,
               int32_t* __restrict__ n_nbr, int cap, int2* __restrict__ jrange,
               const PosT* __restrict__ pos, PosT* __restrict__ pos_build,
               uint32_t* wire_status) {
  nl_build_body<PosT>(nw, wd, cell_count, cell_atoms, cell_of, slot_of, rlist2, nbr, n_nbr, cap,
                      jrange, pos, pos_build, wire_status);
}

// ---------------------------------------------------------------- slab build
// Atoms keep their [100] order, so the neighbours of 32 consecutive atoms of
// a wire lie in one contiguous index range.  The envelopes bound that range
// for any positions: along the atom order, xenv[i] = (prefix max, suffix
// min) of x relative to the wire's origin (FP32).  For a group of atoms whose
// x lie in [xmin, xmax], every neighbour j satisfies xmin - R <= x_j <= xmax
// + R (R = list radius + guard), so j >= lo, the first index whose prefix max
// reaches xmin - R, and j <= hi, the last index whose suffix min is below
// xmax + R (both envelopes are monotone).  The range is tight when the order
// is nearly sorted; its excess grows with the wire's disorder D = max_i
// (prefix max - suffix min), so a wire with D above max_disorder (or any
// wire of an FP64 context) takes the cell build instead.  Two passes over
// the flagged wires' tiles, each fully parallel: k_nl_env_tiles scans each
// tile alone, k_nl_env_merge folds in the extrema of the wire's other tiles.
constexpr float kSlabGuard = 0.01f;  // A added to the list radius for the FP32 envelope
// The slab build tests candidates on FP32 coordinates relative to the
// wire's origin.  Within kSlabMaxCoord of it a coordinate is off by at most
// half an ulp of 2048 A (1.2e-4 A), a coordinate difference by 2.4e-4 A and
// a distance by 4.3e-4 A: inside the 1e-3 A guard the list radius carries,
// so no pair that can reach r_cut before the next rebuild is dropped.  Wires
// reaching farther (410 nm) take the cell build (exact fixed-point
// differences).
constexpr float kSlabMaxCoord = 2048.f;
constexpr float kSlabFar = 1e30f;  // padding slots' x: d^2 overflows to +inf, never accepted

// Block-wide inclusive max-scan from the left and min-scan from the right of
// (mx, mn) over the kSlotTile threads, and the block's max and min.
__device__ __forceinline__ void tile_scans(float& mx, float& mn, float& bmx, float& bmn) {
  __shared__ float s_mx[kSlotTile / 32], s_mn[kSlotTile / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float u = __shfl_up_sync(0xffffffffu, mx, o);
    const float d = __shfl_down_sync(0xffffffffu, mn, o);
    if (lane >= o) mx = fmaxf(mx, u);
    if (lane + o < 32) mn = fminf(mn, d);
  }
  if (lane == 31) s_mx[warp] = mx;  // the warp's max
  if (lane == 0) s_mn[warp] = mn;   // the warp's min
  __syncthreads();
  float before = -INFINITY, after = INFINITY;
  bmx = -INFINITY;
  bmn = INFINITY;
#pragma unroll
  for (int q = 0; q < kSlotTile / 32; ++q) {
    if (q < warp) before = fmaxf(before, s_mx[q]);
    if (q > warp) after = fminf(after, s_mn[q]);
    bmx = fmaxf(bmx, s_mx[q]);
    bmn = fminf(bmn, s_mn[q]);
  }
  mx = fmaxf(mx, before);
  mn = fminf(mn, after);
  __syncthreads();
}

__device__ __forceinline__ void nl_env_tiles_body(NlWork nw, const WireDev* __restrict__ wd,
                                                  const double* __restrict__ x) {
  const int nf = nw.n_flagged[0];
  if (nf == 0 || !nw.slab_ok) return;
  const int64_t tiles = nw.wl_tile[nf];
  for (int64_t tl = blockIdx.x; tl < tiles; tl += gridDim.x) {
    const int k = wl_find(nw.wl_tile, nf, tl);
    const int wi = nw.wl_wire[k];
    const WireDev& w = wd[wi];
    const int kt = (int)(tl - nw.wl_tile[k]);  // tile of the wire
    const int a = kt * kSlotTile + threadIdx.x;
    const bool valid = a < w.n;
    const int64_t i = w.offset + a;
    const float v = valid ? (float)(x[i] - w.origin[0]) : 0.f;
    const float vy = valid ? (float)(x[nw.N + i] - w.origin[1]) : 0.f;
    const float vz = valid ? (float)(x[2 * nw.N + i] - w.origin[2]) : 0.f;
    // the slab build's candidate coordinates (padding slots: far away, never
    // accepted); an atom beyond kSlabMaxCoord of the origin (or not finite)
    // gives its wire an infinite disorder, hence the cell build
    float* xf = reinterpret_cast<float*>(nw.xf + 3 * ((w.slot_base + a) >> 2)) + (a & 3);
    xf[0] = valid ? v : kSlabFar;
    xf[4] = vy;
    xf[8] = vz;
    const bool far =
        valid && !(fabsf(v) <= kSlabMaxCoord && fabsf(vy) <= kSlabMaxCoord && fabsf(vz) <= kSlabMaxCoord);
    float mx = valid ? (far ? INFINITY : v) : -INFINITY, mn = valid ? (far ? -INFINITY : v) : INFINITY;
    float bmx, bmn;
    tile_scans(mx, mn, bmx, bmn);
    if (valid) nw.xenv[w.offset + a] = make_float2(mx, mn);
    if (threadIdx.x == 0) {
      nw.tenv[w.slot_base / kSlotTile + kt] = make_float2(bmx, bmn);
      if (kt == 0) nw.wdis[wi] = 0u;
    }
  }
}
__global__ void __launch_bounds__(kSlotTile)
    k_nl_env_tiles(NlWork nw, const WireDev* __restrict__ wd, const double* __restrict__ x) {
  nl_env_tiles_body(nw, wd, x);
}

// One block: the flagged wires that take the cell build (disorder above the
// slab build's limit, read past L1: the other blocks' atomicMax results),
// compacted in flagged order with the prefixes of their cells and atoms.
__device__ __forceinline__ void nl_cell_list_block(NlWork nw, const WireDev* __restrict__ wd) {
  __shared__ int64_t tot[4];
  const int nf = nw.n_flagged[0];
  const int t = threadIdx.x;
  const int chunk = (nf + (int)blockDim.x - 1) / (int)blockDim.x;
  const int k0 = min(nf, t * chunk), k1 = min(nf, k0 + chunk);
  auto cells = [&](int wi) { return (int64_t)wd[wi].nc[0] * wd[wi].nc[1] * wd[wi].nc[2]; };
  auto cell_wire = [&](int wi) { return !(__uint_as_float(__ldcg(nw.wdis + wi)) <= nw.max_disorder); };
  int64_t v[4] = {0, 0, 0, 0};  // cells, atoms, -, wires
  for (int k = k0; k < k1; ++k) {
    const int wi = nw.wl_wire[k];
    if (cell_wire(wi)) {
      v[0] += cells(wi);
      v[1] += wd[wi].n;
      v[3] += 1;
    }
  }
  block_scan4(v, tot);
  int64_t c_pre = v[0], a_pre = v[1], kk = v[3];
  for (int k = k0; k < k1; ++k) {
    const int wi = nw.wl_wire[k];
    if (cell_wire(wi)) {
      nw.cl_wire[kk] = wi;
      nw.cl_cell[kk] = c_pre;
      nw.cl_atom[kk] = a_pre;
      c_pre += cells(wi);
      a_pre += wd[wi].n;
      ++kk;
    }
  }
  if (t == 0) {
    const int n = (int)tot[3];
    nw.cl_cell[n] = tot[0];
    nw.cl_atom[n] = tot[1];
    nw.n_cell[0] = n;
  }
}

__device__ __forceinline__ void nl_env_merge_body(NlWork nw, const WireDev* __restrict__ wd) {
  __shared__ float s_red[2][kSlotTile / 32];
  __shared__ int s_last;
  const int nf = nw.n_flagged[0];
  if (nf == 0 || !nw.slab_ok) return;
  const int64_t tiles = nw.wl_tile[nf];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t tl = blockIdx.x; tl < tiles; tl += gridDim.x) {
    const int k = wl_find(nw.wl_tile, nf, tl);
    const int wi = nw.wl_wire[k];
    const WireDev& w = wd[wi];
    const int kt = (int)(tl - nw.wl_tile[k]);
    const int nt = (w.n + kSlotTile - 1) / kSlotTile;
    const float2* te = nw.tenv + w.slot_base / kSlotTile;
    // max over the wire's earlier tiles, min over its later tiles
    float before = -INFINITY, after = INFINITY;
    for (int q = threadIdx.x; q < nt; q += blockDim.x) {
      const float2 e = te[q];
      if (q < kt) before = fmaxf(before, e.x);
      if (q > kt) after = fminf(after, e.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      before = fmaxf(before, __shfl_xor_sync(0xffffffffu, before, o));
      after = fminf(after, __shfl_xor_sync(0xffffffffu, after, o));
    }
    if (lane == 0) {
      s_red[0][warp] = before;
      s_red[1][warp] = after;
    }
    __syncthreads();
    before = -INFINITY;
    after = INFINITY;
#pragma unroll
    for (int q = 0; q < kSlotTile / 32; ++q) {
      before = fmaxf(before, s_red[0][q]);
      after = fminf(after, s_red[1][q]);
    }
    __syncthreads();
    const int a = kt * kSlotTile + threadIdx.x;
    float dis = 0.f;
    if (a < w.n) {
      float2 e = nw.xenv[w.offset + a];
      e.x = fmaxf(e.x, before);
      e.y = fminf(e.y, after);
      nw.xenv[w.offset + a] = e;
      dis = e.x - e.y;  // NaN positions: NaN, which fmaxf below does not drop into 0
      if (!(dis == dis)) dis = INFINITY;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dis = fmaxf(dis, __shfl_xor_sync(0xffffffffu, dis, o));
    if (lane == 0 && dis > 0.f) atomicMax(nw.wdis + wi, __float_as_uint(dis));
  }
  // the last block to finish lists the wires that take the cell build (every
  // block's disorder maxima fenced before its arrival is counted)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(nw.merge_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last) {
    __threadfence();
    nl_cell_list_block(nw, wd);
  }
}
__global__ void __launch_bounds__(kSlotTile) k_nl_env_merge(NlWork nw, const WireDev* __restrict__ wd) {
  nl_env_merge_body(nw, wd);
}

// First wire-relative index q <= top with env[q].x >= v (env[top].x >= v
// holds), found by the warp in rounds of 32 probes (stride 16, then 1).
__device__ __forceinline__ int slab_lo(const float2* env, int top, float v) {
  const int lane = threadIdx.x & 31;
  int step = 16;
  for (;;) {
    const int p = top - (lane + 1) * step;
    const bool below = p < 0 || env[p].x < v;
    const unsigned m = __ballot_sync(0xffffffffu, below);
    if (m == 0) {
      top -= 32 * step;  // every probe still reaches v
      continue;
    }
    const int l = __ffs(m) - 1;
    const int ok = top - l * step;  // the first index reaching v is in (ok - step, ok]
    if (step == 1) return ok;
    top = ok;
    step = 1;
  }
}

// Last wire-relative index q >= bot, q < n, with env[q].y <= v (env[bot].y
// <= v holds), by the same search forward.
__device__ __forceinline__ int slab_hi(const float2* env, int bot, int n, float v) {
  const int lane = threadIdx.x & 31;
  int step = 16;
  for (;;) {
    const int p = bot + (lane + 1) * step;
    const bool above = p >= n || env[p].y > v;
    const unsigned m = __ballot_sync(0xffffffffu, above);
    if (m == 0) {
      bot += 32 * step;
      continue;
    }
    const int l = __ffs(m) - 1;
    const int ok = bot + l * step;
    if (step == 1) return ok;
    bot = ok;
    step = 1;
  }
}

// The slab build (MIXED contexts, wires whose disorder allows it): one block
// per tile of kSlotTile consecutive atoms of a flagged wire, one warp per 32
// atoms, one atom per lane.  The warp bounds its candidates by the envelopes
// (slab_lo, slab_hi) and walks them in index order with broadcast loads
// (every lane reads the same candidate), each lane testing it against its
// own atom: d^2 <= r_list^2 on the FP32 coordinates k_nl_env_tiles stored
// (relative to the wire's origin; the cell build takes exact fixed-point
// differences instead, and the two can disagree only on pairs within
// 4.3e-4 A of r_list, inside its 1e-3 A guard).  The test is
// branch-free: each lane collects the outcomes of 32 consecutive candidates
// as the bits of a mask, then appends the set bits to its column of a
// shared-memory buffer as offsets j - i; the atom itself (offset 0, d2 = 0)
// is accepted too and dropped afterwards, so the loop needs no j != i test.
// The row is then written in
// bank-group order (see k_nl_build): the lane's entries are bucketed by
// group (j - wire offset) mod 8, ascending within a group, and at list
// position k the atom in pair-pass lane l = slot mod 8 takes the next entry
// of group (k + l) mod 8 while it has one, else of the group with the most
// entries left (the first such in the rotation from the preferred one); the
// order is a function of the wire alone.  Rows are written as 8-byte groups
// of four entries.  Also the index range [jmin, jmax] and the snapshot of
// the packed position, as the cell build.  The entry buffer has room for
// cap + kSlabSlack entries per lane (cap neighbours and the atom itself).
constexpr int kSlabSlack = 1;
__device__ __forceinline__ void nl_build_slab_body(
    NlWork nw, const WireDev* __restrict__ wd, const int32_t* __restrict__ slot_of, float rlist2,
    float xrange, int16_t* __restrict__ nbr,
    int32_t* __restrict__ n_nbr, int cap, int2* __restrict__ jrange, const int4* __restrict__ xq,
    int4* __restrict__ xq_b, uint32_t* wire_status) {
  extern __shared__ int16_t sA[];  // [cap + kSlabSlack][blockDim.x]: offsets, ascending, by column
  const int B = blockDim.x;
  uint8_t* sB = reinterpret_cast<uint8_t*>(sA + (size_t)(cap + kSlabSlack) * B);  // [cap][B]
  const int nf = nw.n_flagged[0];
  if (nf == 0 || !nw.slab_ok) return;
  const int64_t tiles = nw.wl_tile[nf];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int64_t tl = blockIdx.x; tl < tiles; tl += gridDim.x) {
    const int k = wl_find(nw.wl_tile, nf, tl);
    const int wi = nw.wl_wire[k];
    if (!use_slab(nw, wi)) continue;  // block-uniform
    const WireDev& w = wd[wi];
    const int n = w.n;
    const int a = (int)(tl - nw.wl_tile[k]) * kSlotTile + tid;  // wire-relative atom
    const int g0 = a - lane;                                    // the warp's first atom
    if (g0 >= n) continue;                                      // warp-uniform
    const bool valid = a < n;
    const int64_t i = w.offset + (valid ? a : g0);
    const int ii = (int)i;
    const float2* env = nw.xenv + w.offset;
    // the atom's FP32 coordinates, as its candidates carry them
    const float4* G = nw.xf + 3 * (w.slot_base >> 2);  // the wire's groups of four slots
    const int ai = valid ? a : g0;
    const float* own = reinterpret_cast<const float*>(G + 3 * (ai >> 2)) + (ai & 3);
    const float px = own[0], py = own[4], pz = own[8];
    // the group's extent along the axis, then its candidate range
    float xmin = valid ? px : INFINITY, xmax = valid ? px : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      xmin = fminf(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
      xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    const int glast = min(g0 + 31, n - 1);
    const int lo = slab_lo(env, g0, xmin - xrange);
    int hi = slab_hi(env, glast, n, xmax + xrange);
    if (hi - lo > kMaxOffset - 3) {  // offsets would not fit the int16 entries
      if (lane == 0) atomicOr(&wire_status[wi], kWireNbrOverflow);
      hi = lo + kMaxOffset - 3;
    }
    const int4 pi = xq[i];
    // every lane tests every candidate j in [lo, hi] (widened to whole groups
    // of four: the extra ones lie beyond the slab and fail the test), 32 at a
    // time into an acceptance mask (bit u: candidate j0 + u), whose set bits
    // are then appended to the lane's column as offsets j - i: rows 0..cap
    // hold the first cap + 1 accepted entries (cap neighbours and the atom
    // itself).  A group is three broadcast 16-byte loads (x, y, z of four
    // candidates), its differences and squared distances two FP32 pairs per
    // instruction.
    // Also counted on the way: the accepted entries before the atom's own
    // (negative offsets: the own entry's index), and the stored entries per
    // bank group (eight byte counters; the own entry excluded).
    const int il = (int)(i - w.offset);
    int n_all = 0, n_neg = 0;
    uint64_t T = 0;
    auto flush = [&](uint32_t m, int off0) {
      n_neg += __popc(off0 >= 0 ? 0u : off0 <= -32 ? m : m & ((1u << -off0) - 1u));
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int off = off0 + b;
        if (n_all <= cap) {
          sA[n_all * B + tid] = (int16_t)off;
          if (off != 0) T += 1ull << (8 * ((il + off) & 7));
        }
        ++n_all;
      }
    };
    const float2 nx = make_float2(-px, -px), ny = make_float2(-py, -py), nz = make_float2(-pz, -pz);
    auto test4 = [&](const float4* q, uint32_t bit, uint32_t& m) {
      const float4 X = __ldg(q), Y = __ldg(q + 1), Z = __ldg(q + 2);
      const float2 dx0 = __fadd2_rn(make_float2(X.x, X.y), nx), dx1 = __fadd2_rn(make_float2(X.z, X.w), nx);
      const float2 dy0 = __fadd2_rn(make_float2(Y.x, Y.y), ny), dy1 = __fadd2_rn(make_float2(Y.z, Y.w), ny);
      const float2 dz0 = __fadd2_rn(make_float2(Z.x, Z.y), nz), dz1 = __fadd2_rn(make_float2(Z.z, Z.w), nz);
      const float2 d0 = __ffma2_rn(dz0, dz0, __ffma2_rn(dy0, dy0, __fmul2_rn(dx0, dx0)));
      const float2 d1 = __ffma2_rn(dz1, dz1, __ffma2_rn(dy1, dy1, __fmul2_rn(dx1, dx1)));
      if (d0.x <= rlist2) m |= bit;
      if (d0.y <= rlist2) m |= bit << 1;
      if (d1.x <= rlist2) m |= bit << 2;
      if (d1.y <= rlist2) m |= bit << 3;
    };
    const int alo = lo & ~3, ahi = hi | 3;
    for (int j0 = alo; j0 <= ahi; j0 += 32) {
      uint32_t m = 0;
      const float4* q = G + 3 * (j0 >> 2);
      const int ng = min(8, (ahi - j0 + 1) >> 2);  // groups in this batch of 32
      if (ng == 8) {
#pragma unroll
        for (int g = 0; g < 8; ++g) test4(q + 3 * g, 1u << (4 * g), m);
      } else {
        for (int g = 0; g < ng; ++g) test4(q + 3 * g, 1u << (4 * g), m);
      }
      flush(m, (int)w.offset + j0 - ii);
    }
    if (!valid) continue;
    const bool ovf = n_all > cap + 1;
    n_all = min(n_all, cap + 1);  // accepted and stored, the atom itself included (if it fit)
    // drop the atom itself: offsets ascend, so it follows the negative ones
    // (its index is n_neg; n_all when it was not stored)
    const int self = min(n_neg, n_all);
    const int cnt = n_all - (self < n_all ? 1 : 0);
    if (ovf || cnt > cap) atomicOr(&wire_status[wi], kWireNbrOverflow);
    const int nr = min(cnt, cap);
    auto entry = [&](int e) { return sA[(e < self ? e : e + 1) * B + tid]; };  // e-th without self
    auto group = [&](int e) { return (il + entry(e)) & 7; };
    // bucket the entries by group (ascending within a group); the counts
    // came with the scan unless the row overflowed (then only nr of them)
    if (cnt > nr) {
      T = 0;
      for (int e = 0; e < nr; ++e) T += 1ull << (8 * group(e));
    }
    const uint64_t S = T * 0x0101010101010101ull - T;  // exclusive prefix of the 8 counts
    uint64_t P = S;
    for (int e = 0; e < nr; ++e) {
      const int g = group(e);
      sB[byte_of(P, g) * B + tid] = (uint8_t)e;
      P += 1ull << (8 * g);
    }
    // emit in bank-group order, four entries per 8-byte store
    const int64_t t = slot_of[i];
    const int pl = (int)(t & 7);
    uint64_t R = 0, rem = T;
    uint32_t w0 = 0, w1 = 0;
    uint2* rowg = reinterpret_cast<uint2*>(nbr);
    for (int q = 0; q < nr; ++q) {
      const int want = (q + pl) & 7;
      int g = want;
      if (byte_of(rem, g) == 0) {
        int best = -1;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
          const int h = (want + d) & 7;
          if (byte_of(rem, h) > best) {
            best = byte_of(rem, h);
            g = h;
          }
        }
      }
      const int e = sB[(byte_of(S, g) + byte_of(R, g)) * B + tid];
      R += 1ull << (8 * g);
      rem -= 1ull << (8 * g);
      const uint32_t v = (uint16_t)entry(e);
      const int s4 = q & 3;
      if (s4 == 0) w0 = v;
      else if (s4 == 1) w0 |= v << 16;
      else if (s4 == 2) w1 = v;
      else w1 |= v << 16;
      if (s4 == 3 || q == nr - 1) {
        if (s4 < 2) w1 = 0;
        rowg[nbr_group(t, q >> 2, cap)] = make_uint2(w0, w1);
      }
    }
    n_nbr[t] = nr;
    jrange[t] = nr > 0 ? make_int2(ii + entry(0), ii + entry(nr - 1)) : make_int2(INT_MAX, INT_MIN);
    xq_b[i] = pi;
  }
}
__global__ void __launch_bounds__(256)
    k_nl_build_slab(NlWork nw, const WireDev* __restrict__ wd, const int32_t* __restrict__ slot_of,
                    float rlist2, float xrange, int16_t* __restrict__ nbr,
                    int32_t* __restrict__ n_nbr, int cap, int2* __restrict__ jrange,
                    const int4* __restrict__ xq, int4* __restrict__ xq_b, uint32_t* wire_status) {
  nl_build_slab_body(nw, wd, slot_of, rlist2, xrange, nbr, n_nbr, cap, jrange, xq, xq_b,
                     wire_status);
}

// Row-major copy of the tiled lists (for the list accessor).
// Either output may be null: counts[N] per atom, rows[N * cap] row-major.
__global__ void k_list_rows(int64_t N, int cap, const int16_t* __restrict__ nbr,
                            const int32_t* __restrict__ n_nbr, const int32_t* __restrict__ slot_of,
                            int32_t* __restrict__ counts, int32_t* __restrict__ rows) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= N * cap) return;
  const int64_t i = u / cap;
  const int k = (int)(u - i * cap);
  const int64_t t = slot_of[i];
  if (counts && k == 0) counts[i] = n_nbr[t];
  if (rows) rows[u] = k < n_nbr[t] ? (int32_t)(i + nbr[nbr_slot(t, k, cap)]) : -1;
}

// Block per wire: the wire's atoms in its own slot range in atom order,
// the padding slots that complete its last tile empty (perm = -1).
__global__ void k_slot_init(int W, const WireDev* __restrict__ wd, int64_t NS,
                            int32_t* __restrict__ perm, int32_t* __restrict__ slot_of) {
  for (int w = blockIdx.x; w < W; w += gridDim.x) {
    const WireDev& wr = wd[w];
    const int64_t end = w + 1 < W ? wd[w + 1].slot_base : NS;
    for (int64_t s = wr.slot_base + threadIdx.x; s < end; s += blockDim.x) {
      const int64_t a = s - wr.slot_base;
      perm[s] = a < wr.n ? (int32_t)(wr.offset + a) : -1;
      if (a < wr.n) slot_of[wr.offset + a] = (int32_t)s;
    }
  }
}

// Slot order of the pair passes.  Every wire's slots form whole tiles of
// kSlotTile slots (its count rounded up; the padding slots hold no atom),
// so a tile never mixes wires and an atom's slot does not depend on the rest
// of the batch.  Within each tile the atoms are ranked by list length
// (longest first, ties by slot), so that the 32 threads of a warp walk lists
// of similar length (the core and surface atoms of a wire alternate along its
// [100] order); the padding slots stay last.  A tile keeps its set of atoms,
// so its neighbour-index window is unchanged.  The speed depends on this
// order, and the list rows are ordered for the lane (slot mod 8) an atom gets
// (k_nl_build); the lists are rebuilt after this kernel.
__global__ void __launch_bounds__(kSlotTile)
    k_slot_order(int64_t NS, const int32_t* __restrict__ n_nbr, int32_t* __restrict__ perm,
                 int32_t* __restrict__ slot_of) {
  __shared__ int sn[kSlotTile];
  const int64_t base = (int64_t)blockIdx.x * kSlotTile;
  const int a = threadIdx.x;
  const int64_t s = base + a;
  const int32_t i = s < NS ? perm[s] : -1;
  sn[a] = i >= 0 ? n_nbr[s] : -1;
  __syncthreads();
  if (s < NS) {
    const int na = sn[a];
    int rank = 0;
    for (int b = 0; b < kSlotTile; ++b) rank += (sn[b] > na) || (sn[b] == na && b < a);
    perm[base + rank] = i;
    if (i >= 0) slot_of[i] = (int32_t)(base + rank);
  }
}

}  // namespace tbsma
