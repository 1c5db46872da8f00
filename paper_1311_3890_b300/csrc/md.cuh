// Integrator, thermostat, grips, packing and per-wire reductions.
//
// Methods, "Simulation details": velocity Verlet with dt = 2 fs; two rigid
// gripping layers at each end displaced in opposite directions along [100];
// random Gaussian initial velocities.  The thermostat is Langevin, applied
// as the O step of a B A O A B splitting (gamma = 0 is plain velocity
// Verlet), with Gaussian noise from a counter-based Philox4x32-10 stream
// keyed by the wire's seed and counted by (atom index in wire, step, tag).
//
// Positions and velocities are FP64 throughout; the pair kernels read a
// packed copy written here (int4 modular fixed point for MIXED, 32-byte aligned
// double4 for FP64).
#pragma once

#include "device.cuh"
#include "../../include/tbsma.h"

namespace tbsma {

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  // fixed-order tree over the block (blockDim.x a power of two <= 1024)
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  const T r = sh[0];
  __syncthreads();
  return r;
}

template <typename T>
__device__ __forceinline__ T block_max(T v, T* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (t < s) sh[t] = sh[t + s] > sh[t] ? sh[t + s] : sh[t];
    __syncthreads();
  }
  const T r = sh[0];
  __syncthreads();
  return r;
}

// Block per wire: meta[i] = wire << 2 | kind[i].
__global__ void k_meta(int W, const WireDev* __restrict__ wd, const uint8_t* __restrict__ kind,
                       uint32_t* __restrict__ meta) {
  for (int w = blockIdx.x; w < W; w += gridDim.x) {
    const int64_t o = wd[w].offset;
    for (int a = threadIdx.x; a < wd[w].n; a += blockDim.x)
      meta[o + a] = ((uint32_t)w << 2) | (uint32_t)(kind[o + a] & 3u);
  }
}

// Block per wire: bounding box and mobile count, out[w*7 ..] = lo xyz, hi xyz, n_mobile.
__global__ void __launch_bounds__(256)
    k_bbox(int W, const tbsma_wire* __restrict__ wires, const double* __restrict__ x, int64_t N,
           const uint8_t* __restrict__ kind, double* __restrict__ out) {
  __shared__ double sh[256];
  for (int w = blockIdx.x; w < W; w += gridDim.x) {
    const int64_t o = wires[w].atom_offset;
    const int n = wires[w].n_atoms;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    double nm = 0.0;
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
      for (int d = 0; d < 3; ++d) {
        const double v = x[d * N + o + a];
        lo[d] = fmin(lo[d], v);
        hi[d] = fmax(hi[d], v);
      }
      nm += kind[o + a] == 0 ? 1.0 : 0.0;
    }
    for (int d = 0; d < 3; ++d) {
      const double l = -block_max(-lo[d], sh);
      const double h = block_max(hi[d], sh);
      if (threadIdx.x == 0) {
        out[w * 7 + d] = l;
        out[w * 7 + 3 + d] = h;
      }
    }
    const double m = block_sum(nm, sh);
    if (threadIdx.x == 0) out[w * 7 + 6] = m;
  }
}

// Modular fixed point: the low 32 bits of round((p - origin) * 2^26), read
// from the mantissa of a single FMA.  With origin a multiple of 2^-26 the
// offset 1.5 * 2^52 - origin * 2^26 is exact, so p * 2^26 + offset is rounded
// once, to nearest even, onto the integer grid of [2^52, 2^53) -- the same
// value a round-to-nearest conversion of the exact product would give, with
// no conversion instruction.  Valid while |p - origin| < 2^25 A.
__device__ __forceinline__ int fixed_coord(double p, double ofixm) {
  return __double2loint(fma(p, kFixedScale, ofixm));
}

// fixed_coord with the range check of the packing kernels (a non-finite or
// far-away coordinate flags the wire and packs a clamped value).
__device__ __forceinline__ int to_fixed(double p, const WireDev& w, int d, uint32_t& bad) {
  const double rel = p - w.origin[d];
  if (!(fabs(rel) < kFixedRange)) {
    bad = 1;
    p = rel != rel ? w.origin[d] : w.origin[d] + fmin(fmax(rel, -kFixedRange), kFixedRange);
  }
  return fixed_coord(p, w.ofixm[d]);
}

template <int PREC>
__device__ __forceinline__ void pack_and_check(int64_t i, uint32_t m, const WireDev& w, double px,
                                               double py, double pz, int4* xq, double4_32a* xd,
                                               const int4* xq_b, const double4_32a* xd_b,
                                               double half_skin2, int check, int32_t* flag,
                                               uint32_t* wire_status, int32_t* any = nullptr) {
  const uint32_t wi = meta_wire(m);
  bool moved = false;
  if (PREC == TBSMA_MIXED) {
    uint32_t bad = 0;
    const int4 q = make_int4(to_fixed(px, w, 0, bad), to_fixed(py, w, 1, bad),
                             to_fixed(pz, w, 2, bad), (int)m);
    if (bad) atomicOr(&wire_status[wi], kWireRange);
    xq[i] = q;
    if (check) {
      const int4 b = xq_b[i];
      const float dx = fixed_diff(q.x, b.x), dy = fixed_diff(q.y, b.y),
                  dz = fixed_diff(q.z, b.z);
      moved = dx * dx + dy * dy + dz * dz > (float)half_skin2;
    }
  } else {
    const double4_32a q = make_double4_32a(px, py, pz, __longlong_as_double((long long)m));
    xd[i] = q;
    if (check) {
      const double4_32a b = xd_b[i];
      const double dx = q.x - b.x, dy = q.y - b.y, dz = q.z - b.z;
      moved = dx * dx + dy * dy + dz * dz > half_skin2;
    }
  }
  if (moved) {
    flag[wi] = 1;
    if (any) *any = 1;
  }
}

// Pack the caller's positions for the pair kernels (both layouts), and, if
// `check`, flag wires whose atoms moved past r_skin/2 since their last build.
template <int PREC>
__global__ void k_pack(int64_t N, const double* __restrict__ x, const uint32_t* __restrict__ meta,
                       const WireDev* __restrict__ wd, int4* xq, double4_32a* xd, const int4* xq_b,
                       const double4_32a* xd_b, double half_skin2, int check, int32_t* flag,
                       uint32_t* wire_status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint32_t m = meta[i];
  const WireDev& w = wd[meta_wire(m)];
  const double px = x[i], py = x[N + i], pz = x[2 * N + i];
  if (!isfinite(px) || !isfinite(py) || !isfinite(pz))
    atomicOr(&wire_status[meta_wire(m)], kWireNonFinite);
  // the context's own layout carries the displacement check; the other is a plain copy
  pack_and_check<PREC>(i, m, w, px, py, pz, xq, xd, xq_b, xd_b, half_skin2, check, flag,
                       wire_status);
  if (PREC == TBSMA_MIXED) {
    xd[i] = make_double4_32a(px, py, pz, __longlong_as_double((long long)m));
  } else {
    uint32_t bad = 0;
    xq[i] = make_int4(to_fixed(px, w, 0, bad), to_fixed(py, w, 1, bad), to_fixed(pz, w, 2, bad),
                      (int)m);
    if (bad) atomicOr(&wire_status[meta_wire(m)], kWireRange);
  }
}

// One step's B(kick) A O A for mobile atoms, rigid shift for grips, then
// pack + displacement check.  KICK = 1: half kick dt/2 (first step of a
// sequence); KICK = 2: the previous step's closing half kick merged with
// this step's opening one (both use the same force).
// Nosé–Hoover (proto.thermo = 1): closing half kick (KICK = 2), the scale s of
// the step boundary's NH half steps (k_nh), opening half kick, drift dt.
// The grips' displacement follows the pull mode and the Langevin noise the
// ramped target temperature (see ProtoDev).  PROTO = false compiles the
// default protocol (Langevin, continuous pull, no ramp) alone.
template <int PREC, int KICK, bool PROTO>
__device__ __forceinline__ void integrate_atom(
    int64_t i, long long step, int64_t N, double* __restrict__ x, double* __restrict__ v,
    const float* __restrict__ f32, const double* __restrict__ f64,
    const uint32_t* __restrict__ meta, const WireDev* __restrict__ wd,
    const WireDyn* __restrict__ wdyn, double dt, double inv_m, int4* xq, double4_32a* xd,
    const int4* __restrict__ xq_b, const double4_32a* __restrict__ xd_b, double half_skin2,
    int32_t* flag, uint32_t* wire_status, double* d_grip, const ProtoDev& proto,
    const NhState* __restrict__ nh, const BaroState* __restrict__ baro, int32_t* any) {
  const uint32_t m = meta[i];
  const uint32_t wi = meta_wire(m), kind = meta_kind(m);
  const WireDev& w = wd[wi];
  const WireDyn dy = wdyn[wi];
  const double delta = PROTO ? grip_delta(proto, dy.delta, step) : dy.delta;
  double px = x[i], py = x[N + i], pz = x[2 * N + i];
  double bc = 0.0, bmu = 1.0;
  if (PROTO && proto.baro) {  // S(dt/2) before the drift (B changes v only)
    bc = baro[wi].c;
    bmu = baro[wi].mu;
    px = bc + (px - bc) * bmu;
  }
  double vx, vy, vz;
  if (kind == 0) {
    vx = v[i];
    vy = v[N + i];
    vz = v[2 * N + i];
    double fx, fy, fz;
    if (PREC == TBSMA_MIXED) {
      fx = f32[i];
      fy = f32[N + i];
      fz = f32[2 * N + i];
    } else {
      fx = f64[i];
      fy = f64[N + i];
      fz = f64[2 * N + i];
    }
    if (PROTO && proto.thermo == 1) {
      const double hk = 0.5 * dt * inv_m;
      if (KICK == 2) {
        vx += hk * fx;
        vy += hk * fy;
        vz += hk * fz;
      }
      const double sc = nh[wi].s;
      vx = sc * vx + hk * fx;
      vy = sc * vy + hk * fy;
      vz = sc * vz + hk * fz;
      px += dt * vx;
      py += dt * vy;
      pz += dt * vz;
    } else {
      const double hk = 0.5 * KICK * dt * inv_m;
      vx += hk * fx;
      vy += hk * fy;
      vz += hk * fz;
      const double hd = 0.5 * dt;
      px += hd * vx;
      py += hd * vy;
      pz += hd * vz;
      double c2sig = dy.c2sig;
      if (PROTO && proto.ramp > 0 && w.temperature > 0.0)
        c2sig *= sqrt(target_temperature(proto, w.temperature, step) / w.temperature);
      if (c2sig != 0.0 || dy.c1 != 1.0) {
        double nx = 0.0, ny = 0.0, nz = 0.0;
        if (c2sig != 0.0) {
          const uint4 b = thermostat_bits(w.seed, (uint32_t)(i - w.offset), (uint64_t)step, 0u);
          if (PREC == TBSMA_MIXED) {
            const float3 g = normals3_f32(b);
            nx = g.x;
            ny = g.y;
            nz = g.z;
          } else {
            const double3 g = normals3_f64(b);
            nx = g.x;
            ny = g.y;
            nz = g.z;
          }
        }
        vx = dy.c1 * vx + c2sig * nx;
        vy = dy.c1 * vy + c2sig * ny;
        vz = dy.c1 * vz + c2sig * nz;
      }
      px += hd * vx;
      py += hd * vy;
      pz += hd * vz;
    }
  } else {
    px += (kind == 1) ? -delta : delta;
    vx = vy = vz = 0.0;
  }
  if (PROTO && proto.baro) px = bc + (px - bc) * bmu;  // S(dt/2) after the drift
  x[i] = px;
  x[N + i] = py;
  x[2 * N + i] = pz;
  v[i] = vx;
  v[N + i] = vy;
  v[2 * N + i] = vz;
  if (!isfinite(px + py + pz + vx + vy + vz)) atomicOr(&wire_status[wi], kWireNonFinite);
  pack_and_check<PREC>(i, m, w, px, py, pz, xq, xd, xq_b, xd_b, half_skin2, 1, flag, wire_status,
                       any);
  if (i == w.offset) d_grip[wi] += delta;
}

template <int PREC, int KICK, bool PROTO>
__global__ void __launch_bounds__(256)
    k_integrate(int64_t N, double* __restrict__ x, double* __restrict__ v,
                const float* __restrict__ f32, const double* __restrict__ f64,
                const uint32_t* __restrict__ meta, const WireDev* __restrict__ wd,
                const WireDyn* __restrict__ wdyn, double dt, double inv_m,
                const int64_t* __restrict__ step_counter, int4* xq, double4_32a* xd,
                const int4* __restrict__ xq_b, const double4_32a* __restrict__ xd_b, double half_skin2,
                int32_t* flag, uint32_t* wire_status, double* d_grip, ProtoDev proto,
                const NhState* __restrict__ nh, const BaroState* __restrict__ baro) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  integrate_atom<PREC, KICK, PROTO>(i, step_counter[0], N, x, v, f32, f64, meta, wd, wdyn, dt, inv_m,
                                    xq, xd, xq_b, xd_b, half_skin2, flag, wire_status, d_grip, proto,
                                    nh, baro, nullptr);
}

// Non-finite test on the exponent bits (integer ops, no FP64 pipe).
__device__ __forceinline__ bool finite_bits(double a) {
  return ((__double2hiint(a) >> 20) & 0x7ff) != 0x7ff;
}

// float -> double by re-biasing the exponent field on the integer pipe (exact
// for normal numbers; zero and subnormals give a signed zero, Inf/NaN stay
// Inf/NaN).  B300 runs double conversions on its small FP64 pipe.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned ex = e == 0xffu ? 0x7ff00000u : ((e + 896u) << 20);
  const unsigned hi = (u & 0x80000000u) | (e ? (ex | ((u >> 3) & 0xfffffu)) : 0u);
  const unsigned lo = e ? (u << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}

// double -> float rounded to nearest, ties to even, on the integer pipe: the
// top 23 of the 52 mantissa bits, plus one where the 29 dropped bits are
// above half an ulp, or exactly half with an odd result (a carry out of the
// mantissa steps the exponent, up to Inf).  |d| below the normal float range
// gives a signed 0, above it Inf; non-finite values are caught by
// finite_bits on the double.  This is the value a round-to-nearest
// conversion gives for every normal float result (an unbiased rounding: a
// truncating one would shrink every position increment formed from v by up
// to one ulp).  Used only for FP32 increments of a velocity.
__device__ __forceinline__ float narrow(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned drop = lo & 0x1fffffffu;  // the 29 dropped bits; half an ulp is 1 << 28
  const unsigned up = (drop > 0x10000000u || (drop == 0x10000000u && (m & 1u))) ? 1u : 0u;
  const unsigned body =
      e <= 0 ? 0u : (e >= 255 ? 0x7f800000u : ((((unsigned)e << 23) | m) + up));
  return __uint_as_float((hi & 0x80000000u) | body);
}

// MIXED step: B A O A with the state accumulated in FP64 and each step's
// increments formed in FP32 (they come from FP32 forces and noise; their
// FP32 rounding is ~1e-7 of an increment, far below the force error):
//   B    v1 = v + dv,                 dv = (KICK dt/2m) F
//   O    v2 = v1 + D,                 D  = (c1 - 1) v1 + c2 sqrt(kT/m) n
//   A+A  x2 = x + (dt/2)(v1 + v2) = x + (dt/2)(2 v1 + D)
// so that v and x each take one FP64 add (v2 = v + (dv + D)); the FP32 value
// of v1 is float(v) + dv.  Conversions run on the integer pipe (widen,
// narrow); B300's FP64 pipe is ~1/64 of its FP32 rate.  The packed
// fixed-point position is one FMA per coordinate (fixed_coord); the
// displacement check is integer.
// 40 registers (6 blocks per SM): a streaming kernel needs the warps to keep
// enough loads in flight (measured 19 us per step faster than at 56 registers)
// (The step of atom i, step the 0-based step index; any_flag, if not null,
// is set too when a wire is flagged.  The kernel runs one atom per thread,
// the persistent step kernel strides its threads over the atoms.)
template <int KICK, bool PROTO>
__device__ __forceinline__ void integrate_mixed_atom(
    int64_t i, long long step, int64_t N, double* __restrict__ x, double* __restrict__ v,
    float3 F, const uint32_t* __restrict__ meta,
    const WireDev* __restrict__ wd, const WireDyn* __restrict__ wdyn, float hk, float hd,
    int4* __restrict__ xq, const int4* __restrict__ xq_b, float half_skin2, int32_t* flag,
    int32_t* any_flag, uint32_t* wire_status, double* d_grip, const ProtoDev& proto,
    const NhState* __restrict__ nh, const BaroState* __restrict__ baro) {
  const uint32_t m = meta[i];
  const uint32_t wi = meta_wire(m), kind = meta_kind(m);
  const WireDev& w = wd[wi];
  double px = x[i], py = x[N + i], pz = x[2 * N + i];
  if (PROTO && proto.baro) {  // S(dt/2) before the drift (B changes v only)
    const double bc = baro[wi].c;
    px = bc + (px - bc) * baro[wi].mu;
  }
  double vx = 0.0, vy = 0.0, vz = 0.0;
  if (kind == 0) {
    vx = v[i];
    vy = v[N + i];
    vz = v[2 * N + i];
    if (PROTO && proto.thermo == 1) {
      // Nosé–Hoover: v' = s (v + a) + b with a the closing half kick (KICK = 2)
      // and b the opening one; increments (s - 1)(v + a) + a + b in FP32,
      // drift dt v'.  hk is the half kick here.
      const float bx = hk * F.x, by = hk * F.y, bz = hk * F.z;
      const float ax = KICK == 2 ? bx : 0.f, ay = KICK == 2 ? by : 0.f, az = KICK == 2 ? bz : 0.f;
      const float sm1 = nh[wi].sm1f;
      const float cx = narrow(vx) + ax, cy = narrow(vy) + ay, cz = narrow(vz) + az;
      const float Dx = sm1 * cx, Dy = sm1 * cy, Dz = sm1 * cz;
      vx += widen(ax + Dx + bx);
      vy += widen(ay + Dy + by);
      vz += widen(az + Dz + bz);
      px += widen(2.f * hd * (cx + Dx + bx));
      py += widen(2.f * hd * (cy + Dy + by));
      pz += widen(2.f * hd * (cz + Dz + bz));
    } else {
      const float c1m1 = wdyn[wi].c1m1f;
      float c2sig = wdyn[wi].c2sigf;
      if (PROTO && proto.ramp > 0 && w.temperature > 0.0)
        c2sig *= sqrtf((float)(target_temperature(proto, w.temperature, step) / w.temperature));
      const float dvx = hk * F.x, dvy = hk * F.y, dvz = hk * F.z;
      const float v1x = narrow(vx) + dvx, v1y = narrow(vy) + dvy, v1z = narrow(vz) + dvz;
      float Dx = 0.f, Dy = 0.f, Dz = 0.f;
      if (c2sig != 0.f) {
        const float3 g = normals3_f32(
            thermostat_bits(w.seed, (uint32_t)(i - w.offset), (uint64_t)step, 0u));
        Dx = fmaf(c1m1, v1x, c2sig * g.x);
        Dy = fmaf(c1m1, v1y, c2sig * g.y);
        Dz = fmaf(c1m1, v1z, c2sig * g.z);
      } else if (c1m1 != 0.f) {
        Dx = c1m1 * v1x;
        Dy = c1m1 * v1y;
        Dz = c1m1 * v1z;
      }
      vx += widen(dvx + Dx);
      vy += widen(dvy + Dy);
      vz += widen(dvz + Dz);
      px += widen(hd * fmaf(2.f, v1x, Dx));
      py += widen(hd * fmaf(2.f, v1y, Dy));
      pz += widen(hd * fmaf(2.f, v1z, Dz));
    }
  } else {
    const double delta = PROTO ? grip_delta(proto, wdyn[wi].delta, step) : wdyn[wi].delta;
    px += (kind == 1) ? -delta : delta;
  }
  if (i == w.offset) d_grip[wi] += PROTO ? grip_delta(proto, wdyn[wi].delta, step) : wdyn[wi].delta;
  if (PROTO && proto.baro) {  // S(dt/2) after the drift
    const double bc = baro[wi].c;
    px = bc + (px - bc) * baro[wi].mu;
  }
  x[i] = px;
  x[N + i] = py;
  x[2 * N + i] = pz;
  v[i] = vx;
  v[N + i] = vy;
  v[2 * N + i] = vz;
  if (!(finite_bits(px) & finite_bits(py) & finite_bits(pz) & finite_bits(vx) & finite_bits(vy) &
        finite_bits(vz)))
    atomicOr(&wire_status[wi], kWireNonFinite);
  const int4 q = make_int4(fixed_coord(px, w.ofixm[0]), fixed_coord(py, w.ofixm[1]),
                           fixed_coord(pz, w.ofixm[2]), (int)m);
  xq[i] = q;
  const int4 b = xq_b[i];
  const float ex = fixed_diff(q.x, b.x), ey = fixed_diff(q.y, b.y), ez = fixed_diff(q.z, b.z);
  if (ex * ex + ey * ey + ez * ez > half_skin2) {
    flag[wi] = 1;
    if (any_flag) *any_flag = 1;
  }
}

template <int KICK, bool PROTO>
__global__ void __launch_bounds__(256, 6)
    k_integrate_mixed(int64_t N, double* __restrict__ x, double* __restrict__ v,
                      const float* __restrict__ f32, const uint32_t* __restrict__ meta,
                      const WireDev* __restrict__ wd, const WireDyn* __restrict__ wdyn, float hk,
                      float hd, const int64_t* __restrict__ step_counter, int4* __restrict__ xq,
                      const int4* __restrict__ xq_b, float half_skin2, int32_t* flag,
                      uint32_t* wire_status, double* d_grip, ProtoDev proto,
                      const NhState* __restrict__ nh, const BaroState* __restrict__ baro) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  integrate_mixed_atom<KICK, PROTO>(i, step_counter[0], N, x, v,
                                    make_float3(f32[i], f32[N + i], f32[2 * N + i]), meta, wd, wdyn,
                                    hk, hd, xq,
                                    xq_b, half_skin2, flag, nullptr, wire_status, d_grip, proto, nh,
                                    baro);
}

// Block per wire: the Nosé–Hoover half steps at a step boundary (Methods,
// "Simulation details": Nosé–Hoover thermostat with velocity Verlet).  K is
// the mobile kinetic energy of v + kick F (kick = the closing half kick not
// yet applied to v, or 0), reduced in a fixed order.  mode bit 1: the end
// half step of step c - 1, bit 2: the begin half step of step c (c = the
// step counter).  A half step of length h = dt/2 at target T is
//   xi += (h/2)(2K - g k_B T)/Q;  scale exp(-xi h);  K *= scale^2;
//   eta += h xi;  xi += (h/2)(2K - g k_B T)/Q
// with g = 3 N_mobile and Q = g k_B T_w tau^2.  The product of the scales is
// left in nh[w].s for the integrator (or k_nh_scale); a wire with Q = 0 gets
// s = 1 (NVE).
__global__ void __launch_bounds__(256)
    k_nh(int W, const WireDev* __restrict__ wd, const uint32_t* __restrict__ meta, int64_t N,
         const double* __restrict__ v, const float* __restrict__ f32,
         const double* __restrict__ f64, int prec, double kick, int mode, double dt,
         ProtoDev proto, double m_e, const int64_t* __restrict__ step_counter,
         NhState* __restrict__ nh) {
  __shared__ double sh[256];
  for (int w = blockIdx.x; w < W; w += gridDim.x) {
    const WireDev& wr = wd[w];
    double k2 = 0.0;
    for (int a = threadIdx.x; a < wr.n; a += blockDim.x) {
      const int64_t i = wr.offset + a;
      if (meta_kind(meta[i]) != 0) continue;
      for (int d = 0; d < 3; ++d) {
        const double f = prec == TBSMA_MIXED ? (double)f32[d * N + i] : f64[d * N + i];
        const double u = v[d * N + i] + kick * f;
        k2 += u * u;
      }
    }
    const double K = 0.5 * m_e * block_sum(k2, sh);
    if (threadIdx.x == 0) {
      NhState st = nh[w];
      const double g = 3.0 * (double)wr.n_mobile;
      const double Q = g * kBoltzmann * wr.temperature * proto.tau * proto.tau;
      double scale = 1.0;
      if (Q > 0.0) {
        const long long c = step_counter[0];
        const double h = 0.5 * dt;
        double Kc = K;
        for (int half = 1; half <= 2; half <<= 1) {
          if (!(mode & half)) continue;
          const double T = target_temperature(proto, wr.temperature, half == 1 ? c - 1 : c);
          const double gkT = g * kBoltzmann * T;
          st.xi += 0.5 * h * (2.0 * Kc - gkT) / Q;
          const double sc = exp(-st.xi * h);
          Kc *= sc * sc;
          st.eta += h * st.xi;
          st.xi += 0.5 * h * (2.0 * Kc - gkT) / Q;
          scale *= sc;
        }
      }
      st.s = scale;
      st.sm1f = (float)(scale - 1.0);
      nh[w] = st;
    }
  }
}

// Mobile velocities times their wire's NH scale (the end half step of a
// sequence, after the closing half kick).
__global__ void k_nh_scale(int64_t N, double* __restrict__ v, const uint32_t* __restrict__ meta,
                           const NhState* __restrict__ nh) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint32_t m = meta[i];
  if (meta_kind(m) != 0) return;
  const double sc = nh[meta_wire(m)].s;
  for (int d = 0; d < 3; ++d) v[d * N + i] *= sc;
}

// Axial Nosé–Hoover barostat (Methods: 100 ps at zero pressure along [100]
// with a Nosé–Hoover barostat before the pull).  Hoover's constant-stress
// equations along x about the grips' centre c, per wire:
//   dx/dt = v_x + zeta (x - c),  dv_x/dt = F_x/m - zeta v_x,
//   dzeta/dt = -(sigma_xx - P) / (B tau_b^2) - gamma_b zeta,  dlambda/dt = zeta
// (barostat mass V B tau_b^2, V the Eq. 5 volume), in the symmetric step
//   Z C [NH] B S A S [forces] B [NH] C Z  (each half a step h = dt/2),
// Z: drag and stress kick of zeta, C: v_x *= exp(-zeta h), S: x = c + (x - c)
// exp(zeta h) (in the integrator).  sigma_xx is Eq. 5 as k_observe forms it,
// from the per-atom virial of the last force pass (on these positions).
struct BaroArgs {
  double m_e, v_atom, h, p, inv_btau2, drag;  // drag = exp(-gamma_b h)
};

__device__ __forceinline__ double baro_sigma(double vir, double vx2, const BaroArgs& a, int n) {
  return (vir - a.m_e * vx2) / (a.v_atom * n);
}

// Block per wire, at a step's start: Z (drag, then kick), C; leaves c and mu
// for the integrator's S and advances lambda by both S half steps.
__global__ void __launch_bounds__(256)
    k_baro_begin(int W, const WireDev* __restrict__ wd, const uint32_t* __restrict__ meta,
                 int64_t N, const double* __restrict__ x, double* __restrict__ v,
                 const double* __restrict__ w_atom, BaroArgs a, BaroState* __restrict__ baro) {
  __shared__ double sh[256];
  for (int w = blockIdx.x; w < W; w += gridDim.x) {
    const WireDev& wr = wd[w];
    double vir = 0.0, vx2 = 0.0, cx = 0.0, ng = 0.0;
    for (int t = threadIdx.x; t < wr.n; t += blockDim.x) {
      const int64_t i = wr.offset + t;
      vir += w_atom[i];
      if (meta_kind(meta[i]) == 0) {
        vx2 += v[i] * v[i];
      } else {
        cx += x[i];
        ng += 1.0;
      }
    }
    vir = block_sum(vir, sh);
    vx2 = block_sum(vx2, sh);
    cx = block_sum(cx, sh);
    ng = block_sum(ng, sh);
    BaroState b = baro[w];
    b.zeta *= a.drag;
    b.zeta -= a.h * (baro_sigma(vir, vx2, a, wr.n) - a.p) * a.inv_btau2;
    b.c = ng > 0.0 ? cx / ng : 0.0;
    b.mu = exp(b.zeta * a.h);
    b.lam = (b.lam + b.zeta * a.h) + b.zeta * a.h;
    const double sc = exp(-b.zeta * a.h);
    for (int t = threadIdx.x; t < wr.n; t += blockDim.x) {
      const int64_t i = wr.offset + t;
      if (meta_kind(meta[i]) == 0) v[i] *= sc;
    }
    if (threadIdx.x == 0) baro[w] = b;
    __syncthreads();
  }
}

// Block per wire, at a step's end: C, then Z (kick, then drag).
__global__ void __launch_bounds__(256)
    k_baro_end(int W, const WireDev* __restrict__ wd, const uint32_t* __restrict__ meta,
               int64_t N, double* __restrict__ v, const double* __restrict__ w_atom, BaroArgs a,
               BaroState* __restrict__ baro) {
  __shared__ double sh[256];
  for (int w = blockIdx.x; w < W; w += gridDim.x) {
    const WireDev& wr = wd[w];
    BaroState b = baro[w];
    const double sc = exp(-b.zeta * a.h);
    double vir = 0.0, vx2 = 0.0;
    for (int t = threadIdx.x; t < wr.n; t += blockDim.x) {
      const int64_t i = wr.offset + t;
      vir += w_atom[i];
      if (meta_kind(meta[i]) == 0) {
        const double u = v[i] * sc;
        v[i] = u;
        vx2 += u * u;
      }
    }
    vir = block_sum(vir, sh);
    vx2 = block_sum(vx2, sh);
    b.zeta -= a.h * (baro_sigma(vir, vx2, a, wr.n) - a.p) * a.inv_btau2;
    b.zeta *= a.drag;
    if (threadIdx.x == 0) baro[w] = b;
    __syncthreads();
  }
}

// Closing half kick of the last step of a sequence, MIXED, with the atom's
// FP32 force at hand.
__device__ __forceinline__ void half_kick_atom_f(int64_t i, int64_t N, double* __restrict__ v,
                                                 float3 F, const uint32_t* __restrict__ meta,
                                                 double hk) {
  if (meta_kind(meta[i]) != 0) return;
  v[i] += hk * (double)F.x;
  v[N + i] += hk * (double)F.y;
  v[2 * N + i] += hk * (double)F.z;
}

// Closing half kick of the last step of a sequence.
template <int PREC>
__device__ __forceinline__ void half_kick_atom(int64_t i, int64_t N, double* __restrict__ v,
                                               const float* __restrict__ f32,
                                               const double* __restrict__ f64,
                                               const uint32_t* __restrict__ meta, double hk) {
  if (meta_kind(meta[i]) != 0) return;
  for (int d = 0; d < 3; ++d) {
    const double f = PREC == TBSMA_MIXED ? (double)f32[d * N + i] : f64[d * N + i];
    v[d * N + i] += hk * f;
  }
}

template <int PREC>
__global__ void k_half_kick(int64_t N, double* __restrict__ v, const float* __restrict__ f32,
                            const double* __restrict__ f64, const uint32_t* __restrict__ meta,
                            double hk) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  half_kick_atom<PREC>(i, N, v, f32, f64, meta, hk);
}

// Block per wire: initial velocities (Philox tag 1), mobile COM removed,
// scaled to the exact target temperature.
__global__ void __launch_bounds__(256)
    k_init_velocities(int W, const WireDev* __restrict__ wd, const uint32_t* __restrict__ meta,
                      int64_t N, double* __restrict__ v, double m_e) {
  __shared__ double sh[256];
  for (int w = blockIdx.x; w < W; w += gridDim.x) {
    const WireDev& wr = wd[w];
    const double sig = sqrt(kBoltzmann * wr.temperature / m_e);
    double s[3] = {0.0, 0.0, 0.0}, nm = 0.0;
    for (int a = threadIdx.x; a < wr.n; a += blockDim.x) {
      const int64_t i = wr.offset + a;
      if (meta_kind(meta[i]) != 0) {
        v[i] = v[N + i] = v[2 * N + i] = 0.0;
        continue;
      }
      const double3 g = normals3_f64(thermostat_bits(wr.seed, (uint32_t)a, 0, 1u));
      v[i] = sig * g.x;
      v[N + i] = sig * g.y;
      v[2 * N + i] = sig * g.z;
      s[0] += v[i];
      s[1] += v[N + i];
      s[2] += v[2 * N + i];
      nm += 1.0;
    }
    const double n_mob = block_sum(nm, sh);
    double mean[3];
    for (int d = 0; d < 3; ++d) mean[d] = n_mob > 0 ? block_sum(s[d], sh) / n_mob : 0.0;
    double v2 = 0.0;
    for (int a = threadIdx.x; a < wr.n; a += blockDim.x) {
      const int64_t i = wr.offset + a;
      if (meta_kind(meta[i]) != 0) continue;
      for (int d = 0; d < 3; ++d) {
        const double u = v[d * N + i] - mean[d];
        v[d * N + i] = u;
        v2 += u * u;
      }
    }
    const double ekin = 0.5 * m_e * block_sum(v2, sh);
    const double target = 1.5 * n_mob * kBoltzmann * wr.temperature;
    const double scale = ekin > 0.0 ? sqrt(target / ekin) : 0.0;
    for (int a = threadIdx.x; a < wr.n; a += blockDim.x) {
      const int64_t i = wr.offset + a;
      if (meta_kind(meta[i]) != 0) continue;
      for (int d = 0; d < 3; ++d) v[d * N + i] *= scale;
    }
  }
}

// Block per wire: Eq. 3-5 reductions in FP64 with a fixed summation order.
__global__ void __launch_bounds__(256)
    k_observe(int W, const WireDev* __restrict__ wd, const uint32_t* __restrict__ meta, int64_t N,
              const double* __restrict__ e_atom, const double* __restrict__ w_atom,
              const double* __restrict__ v, const double* __restrict__ d_grip,
              const int32_t* __restrict__ n_rebuilds, const uint32_t* __restrict__ wire_status,
              int64_t steps, double m_e, double v_atom, tbsma_obs* __restrict__ out) {
  __shared__ double sh[256];
  for (int w = blockIdx.x; w < W; w += gridDim.x) {
    const WireDev& wr = wd[w];
    // five FP64 operations per atom (B300's FP64 pipe is the bound): the
    // x and the y + z parts of v^2 apart, the mobile count in an integer
    double e = 0.0, vir = 0.0, vx2 = 0.0, vyz = 0.0;
    int nmob = 0;
    for (int a = threadIdx.x; a < wr.n; a += blockDim.x) {
      const int64_t i = wr.offset + a;
      e += e_atom[i];
      vir += w_atom[i];
      if (meta_kind(meta[i]) == 0) {
        const double ux = v[i], uy = v[N + i], uz = v[2 * N + i];
        vx2 = fma(ux, ux, vx2);
        vyz = fma(uy, uy, fma(uz, uz, vyz));
        ++nmob;
      }
    }
    e = block_sum(e, sh);
    vir = block_sum(vir, sh);
    vx2 = block_sum(vx2, sh);
    vyz = block_sum(vyz, sh);
    const double nm = block_sum((double)nmob, sh);
    const double v2 = vx2 + vyz;
    if (threadIdx.x == 0) {
      tbsma_obs o;
      o.step = steps;
      o.strain = 2.0 * d_grip[w] / wr.L0;
      o.e_pot = e;
      o.e_kin = 0.5 * m_e * v2;
      o.temp = nm > 0 ? 2.0 * o.e_kin / (3.0 * nm * kBoltzmann) : 0.0;
      o.sigma_xx = (vir - m_e * vx2) / (v_atom * wr.n);
      o.virial_xx = vir;
      o.n_rebuilds = n_rebuilds[w];
      o.status = (int32_t)wire_status[w];
      out[w] = o;
    }
  }
}

// Mixed vs FP64 force errors in two kernels, so that one large wire spreads
// over the GPU: k_force_check_tiles takes one block per 256-slot tile (a
// tile never mixes wires) and writes the tile's partials — the largest
// |dF_i| / S_i, |dF_i| / |F_i| and |dF_i|, and the sums of |dF_i|^2 and
// |F_i|^2 — to part[5 * tile]; k_force_check folds a wire's tiles, a block
// per wire.  Sums run in fixed trees in both, so the results are the same on
// every run and for a wire alone or in any batch.
__global__ void __launch_bounds__(256)
    k_force_check_tiles(int64_t NS, int64_t N, const int32_t* __restrict__ perm,
                        const float* __restrict__ f32, const double* __restrict__ f64,
                        const double* __restrict__ s_atom, double* __restrict__ part) {
  __shared__ double sh[256];
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = t < NS ? perm[t] : -1;
  double es = 0.0, er = 0.0, ea = 0.0, dd = 0.0, ff = 0.0;
  if (i >= 0) {
    for (int d = 0; d < 3; ++d) {
      const double r = f64[d * N + i];
      const double e = (double)f32[d * N + i] - r;
      dd += e * e;
      ff += r * r;
    }
    const double de = sqrt(dd), fm = sqrt(ff);
    if (s_atom[i] > 0.0) es = de / s_atom[i];
    if (fm > 0.0) er = de / fm;
    ea = de;
  }
  es = block_max(es, sh);
  er = block_max(er, sh);
  ea = block_max(ea, sh);
  dd = block_sum(dd, sh);
  ff = block_sum(ff, sh);
  if (threadIdx.x == 0) {
    double* p = part + 5 * blockIdx.x;
    p[0] = es;
    p[1] = er;
    p[2] = ea;
    p[3] = dd;
    p[4] = ff;
  }
}

__global__ void __launch_bounds__(256)
    k_force_check(int W, const WireDev* __restrict__ wd, const double* __restrict__ part,
                  tbsma_fcheck* __restrict__ out) {
  __shared__ double sh[256];
  for (int w = blockIdx.x; w < W; w += gridDim.x) {
    const WireDev& wr = wd[w];
    const int64_t t0 = wr.slot_base / 256, nt = (wr.n + 255) / 256;
    double es = 0.0, er = 0.0, ea = 0.0, d2 = 0.0, f2 = 0.0;
    for (int64_t k = threadIdx.x; k < nt; k += blockDim.x) {
      const double* p = part + 5 * (t0 + k);
      es = fmax(es, p[0]);
      er = fmax(er, p[1]);
      ea = fmax(ea, p[2]);
      d2 += p[3];
      f2 += p[4];
    }
    es = block_max(es, sh);
    er = block_max(er, sh);
    ea = block_max(ea, sh);
    d2 = block_sum(d2, sh);
    f2 = block_sum(f2, sh);
    if (threadIdx.x == 0) {
      tbsma_fcheck o;
      o.max_err_scaled = es;
      o.max_err_raw = er;
      o.norm_err = f2 > 0.0 ? sqrt(d2 / f2) : 0.0;
      o.max_abs_err = ea;
      out[w] = o;
    }
  }
}

__global__ void k_philox(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                         int64_t n, uint32_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = philox4x32_10(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]),
                                make_uint2(key[2 * i], key[2 * i + 1]));
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

template <int PREC>
__global__ void k_normals(uint64_t seed, const uint32_t* __restrict__ atoms, int64_t n,
                          uint64_t step, uint32_t tag, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 b = thermostat_bits(seed, atoms[i], step, tag);
  if (PREC == TBSMA_MIXED) {
    const float3 g = normals3_f32(b);
    out[3 * i] = g.x;
    out[3 * i + 1] = g.y;
    out[3 * i + 2] = g.z;
  } else {
    const double3 g = normals3_f64(b);
    out[3 * i] = g.x;
    out[3 * i + 1] = g.y;
    out[3 * i + 2] = g.z;
  }
}

}  // namespace tbsma
