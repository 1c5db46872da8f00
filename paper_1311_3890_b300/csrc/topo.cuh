// Wire topology: rupture and neck (Results, "Nanowire elongation": a wire
// fails when it comes apart, and the neck is its thinnest section before
// that; the paper gives no formal definition, see tbsma_wire_topology).
//
// Clusters are the connected components of the graph of interacting pairs,
// found with a lock-free union-find: every in-cutoff pair (i, j), j > i, of
// the neighbour lists links the larger of the two roots under the smaller
// with a compare-and-swap, so parent[x] <= x always holds and each
// component's root is its smallest atom index, whatever order the links
// land in (the labels are unique, not merely valid).  Reads of parent[] go
// through L2 (ld.global.cg) so that links made by other SMs are seen; every
// walk and retry loop is bounded and reports through an error word.
#pragma once

#include "md.cuh"
#include "pair.cuh"

namespace tbsma {

constexpr int kUfSteps = 1 << 20;    // default bound of one root walk (tbsma_set_wait_limit)
constexpr int kUfRetries = 1 << 16;  // bound of one link's retries
constexpr int kMaxSlabs = 4096;      // slabs per wire in the neck histogram
constexpr double kSlabWidth = 0.5 * 4.079;  // a/2, the (100) plane spacing of the wires, A
constexpr uint32_t kUfGaveUp = 2u;

__device__ __forceinline__ int uf_find(int* parent, int a, int limit, uint32_t* err) {
  for (int s = 0; s < limit; ++s) {
    const int p = __ldcg(parent + a);
    if (p == a) return a;
    const int gp = __ldcg(parent + p);
    if (gp != p) __stcg(parent + a, gp);  // path halving: gp is an ancestor, gp < a
    a = gp;
  }
  atomicOr(err, kUfGaveUp);
  return a;
}

__device__ __forceinline__ void uf_union(int* parent, int a, int b, int limit, uint32_t* err) {
  for (int r = 0; r < kUfRetries; ++r) {
    int ra = uf_find(parent, a, limit, err), rb = uf_find(parent, b, limit, err);
    if (ra == rb) return;
    if (ra > rb) {
      const int tmp = ra;
      ra = rb;
      rb = tmp;
    }
    if (atomicCAS(parent + rb, rb, ra) == rb) return;  // rb was still a root: linked
  }
  atomicOr(err, kUfGaveUp);
}

__global__ void k_uf_init(int64_t N, int* parent) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) parent[i] = (int)i;
}

// One thread per slot (NS slots): link the atom with every list neighbour j > i that
// interacts under the context's rule (the pair passes' cutoff decision).
template <int PREC>
__global__ void k_uf_link(int64_t NS, const int4* __restrict__ xq, const double4_32a* __restrict__ xd,
                          const int16_t* __restrict__ nbr, const int32_t* __restrict__ n_nbr,
                          const int32_t* __restrict__ perm, int cap, PairConsts pc, int* parent,
                          int limit, uint32_t* err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= NS) return;
  const int i = perm[t];
  if (i < 0) return;  // a tile's padding slot
  const int n = n_nbr[t];
  for (int k = 0; k < n; ++k) {
    const int j = i + nbr[nbr_slot(t, k, cap)];
    if (j <= i) continue;
    bool in;
    if (PREC == TBSMA_MIXED) {
      in = geom32(xq[i], xq[j]).r2 <= pc.rc2f;
    } else {
      const double4_32a pi = xd[i], pj = xd[j];
      const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
      in = dx * dx + dy * dy + dz * dz <= pc.rc2;
    }
    if (in) uf_union(parent, i, j, limit, err);
  }
}

__global__ void k_uf_compress(int64_t N, int* parent, int limit, uint32_t* err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) parent[i] = uf_find(parent, (int)i, limit, err);
}

// Block per wire: grip connectivity, cluster count and the neck histogram
// (slab arithmetic in FP64 on the caller's positions, as the oracle's).
__global__ void __launch_bounds__(256)
    k_topology(int W, const WireDev* __restrict__ wd, const uint32_t* __restrict__ meta, int64_t N,
               const double* __restrict__ x, const int* __restrict__ parent,
               tbsma_topology* __restrict__ out) {
  __shared__ double shd[256];
  __shared__ long long shl[256];
  __shared__ int cnt[kMaxSlabs];
  for (int w = blockIdx.x; w < W; w += gridDim.x) {
    const WireDev& wr = wd[w];
    long long left = LLONG_MAX, right = LLONG_MAX, roots = 0;
    double x_lo = -1e300, x_hi = 1e300;
    for (int a = threadIdx.x; a < wr.n; a += blockDim.x) {
      const int64_t i = wr.offset + a;
      const uint32_t kd = meta_kind(meta[i]);
      if (parent[i] == (int)i) ++roots;
      if (kd == 1) {
        left = min(left, (long long)i);
        x_lo = fmax(x_lo, x[i]);
      } else if (kd == 2) {
        right = min(right, (long long)i);
        x_hi = fmin(x_hi, x[i]);
      }
    }
    left = -block_max(-left, shl);
    right = -block_max(-right, shl);
    roots = block_sum(roots, shl);
    x_lo = block_max(x_lo, shd);
    x_hi = -block_max(-x_hi, shd);
    tbsma_topology o;
    o.n_clusters = (int32_t)roots;
    o.status = 0;
    o.neck = -1;
    o.neck_slab = -1;
    o.n_slabs = 0;
    const bool grips = left != LLONG_MAX && right != LLONG_MAX;
    o.connected = grips && parent[left] == parent[right];
    long long ns = grips && x_hi > x_lo ? (long long)floor((x_hi - x_lo) / kSlabWidth - 0.5) : 0;
    if (ns < 0) ns = 0;
    if (!grips) o.status = 3;
    else if (ns > kMaxSlabs) o.status = 1;
    if (grips && ns <= kMaxSlabs) {
      for (int k = threadIdx.x; k < ns; k += blockDim.x) cnt[k] = 0;
      __syncthreads();
      for (int a = threadIdx.x; a < wr.n; a += blockDim.x) {
        const double u = (x[wr.offset + a] - x_lo) / kSlabWidth - 0.5;
        if (u >= 0.0 && u < (double)ns) atomicAdd(&cnt[(int)floor(u)], 1);
      }
      __syncthreads();
      // smallest count, first slab on ties: minimise count * 2^32 + slab
      long long best = LLONG_MAX;
      for (int k = threadIdx.x; k < ns; k += blockDim.x)
        best = min(best, ((long long)cnt[k] << 32) | k);
      best = -block_max(-best, shl);
      o.n_slabs = (int32_t)ns;
      o.neck = 0;  // no slab between the grips: no section to count
      if (ns > 0) {
        o.neck = (int32_t)(best >> 32);
        o.neck_slab = (int32_t)(best & 0xffffffffLL);
      }
    }
    if (threadIdx.x == 0) out[w] = o;
    __syncthreads();
  }
}

}  // namespace tbsma
