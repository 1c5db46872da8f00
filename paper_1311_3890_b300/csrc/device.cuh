// Device-side building blocks of the TB-SMA wire MD path: layouts shared by
// the kernels, the counter-based generator and its Gaussian transform.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tbsma {

// ---------------------------------------------------------------- constants
// CODATA 2018.  1 amu*A^2/fs^2 in eV = amu[kg] * 1e10 / e[J].
constexpr double kBoltzmann = 8.617333262e-5;  // eV/K
constexpr double kAmuKg = 1.66053906660e-27;
constexpr double kElectronVoltJ = 1.602176634e-19;
constexpr double kMvv2e = kAmuKg * 1.0e10 / kElectronVoltJ;

// Modular fixed-point positions for the FP32 pair kernels: 2^26 units per
// Angstrom relative to the wire centre, kept modulo 2^32 (int32 wrap-around).
// The wrap-around difference of two coordinates is their exact difference
// whenever that is below 2^31 units = 32 A, which holds for every list pair
// and for every displacement check; its conversion to float is the correctly
// rounded FP32 difference.  The grid error (2^-27 A) is ~100x below an FP32
// ulp of a neighbour distance, so positions carry no coherent error.
constexpr double kFixedScale = 67108864.0;                 // 2^26
constexpr float kFixedInv = 1.4901161193847656e-08f;       // 2^-26
constexpr double kFixedRange = 1.0e7;                      // |x - centre| limit of fixed_coord, A
constexpr double kFixedMagic = 6755399441055744.0;          // 1.5 * 2^52

constexpr uint32_t kWireNonFinite = 1u;
constexpr uint32_t kWireNbrOverflow = 2u;
constexpr uint32_t kWireCellOverflow = 4u;
constexpr uint32_t kWireRange = 8u;
// Not a fault: an atom lay outside its wire's cell grid at a list build and
// was binned into an edge cell (the list is still exact while no cell
// overflows).  The host grows the wire's grid and clears the bit.
constexpr uint32_t kWireGridClamp = 16u;

constexpr int kCellCap = 32;  // atoms per cell (one per lane in the sort and build)

// meta word of an atom: wire index << 2 | kind (0 mobile, 1 left grip, 2 right grip)
__host__ __device__ __forceinline__ uint32_t meta_wire(uint32_t m) { return m >> 2; }
__host__ __device__ __forceinline__ uint32_t meta_kind(uint32_t m) { return m & 3u; }

// Static description of one wire (set at init).
struct WireDev {
  int64_t offset;
  int32_t n;
  int32_t n_mobile;
  double origin[3];  // fixed-point origin: centre of the initial bounding box, a multiple of 2^-26
  double ofixm[3];   // 1.5 * 2^52 - origin * 2^26 (exact): the fixed-point offset of fixed_coord
  double glo[3];     // cell-grid lower corner relative to the origin
  double einv[3];    // 1 / cell edge
  int32_t nc[3];     // cells per direction
  int32_t pad;
  int64_t cell_base;  // index of the wire's first cell
  int64_t slot_base;  // first slot of the wire's tiles (a multiple of kSlotTile; see k_slot_order)
  uint64_t seed;
  double L0, strain_rate, temperature, gamma;
};

// Per-wire constants that depend on dt.
struct WireDyn {
  double c1;     // exp(-gamma dt)
  double c2sig;  // sqrt(1 - c1^2) * sqrt(kT/m)  (A/fs)
  double delta;  // grip displacement per step, A
  float c1m1f;   // c1 - 1 (FP32 increment form of the O step)
  float c2sigf;  // c2sig in FP32
};

// Paper protocol mode (Methods, "Simulation details"): the thermostat kind,
// the pull mode and the temperature ramp, as set by tbsma_set_protocol.
struct ProtoDev {
  int thermo;          // 0 Langevin (B A O A B), 1 Nosé–Hoover
  int pull;            // 0 continuous (strain rate), 1 stepwise
  double tau;          // Nosé–Hoover period, fs
  double pull_step;    // stepwise: displacement of each grip per event, A
  long long interval;  // stepwise: steps per event
  double t_start;      // ramp start temperature, K
  long long ramp;      // ramp length in steps, 0 = none
  long long ramp_start;  // first step of the ramp (t_start before it)
  int baro;            // 1: the axial barostat scales x about BaroState::c
};

// One wire's axial Nosé–Hoover barostat: strain rate zeta (1/fs), the
// log-stretch lambda, and for the current step the grips' centre c and the
// half-step scale factor mu = exp(zeta dt/2) that the integrator applies
// to x before and after its drift.
struct BaroState {
  double zeta, lam, c, mu;
};

// One wire's Nosé–Hoover state: xi (1/fs), its integral eta, and the
// velocity scale factor s of the current step boundary (with s - 1 in FP32
// for the mixed integrator's increment form).
struct NhState {
  double xi, eta, s;
  float sm1f;
};

// Target temperature of step s (0-based): t_start until step ramp_start,
// then a linear ramp to the wire's temperature over `ramp` steps, then
// constant (no ramp: the wire's temperature throughout).
__host__ __device__ inline double target_temperature(const ProtoDev& p, double T_w, long long s) {
  if (p.ramp <= 0) return T_w;
  double f = (double)(s - p.ramp_start) / (double)p.ramp;
  if (f < 0.0) f = 0.0;
  if (f > 1.0) f = 1.0;
  return p.t_start + (T_w - p.t_start) * f;
}

// Grip displacement in step s: a stepwise event when (s + 1) is a multiple
// of the interval, else the continuous per-step displacement.
__host__ __device__ inline double grip_delta(const ProtoDev& p, double delta_continuous,
                                             long long s) {
  if (p.pull == 1) return (p.interval > 0 && (s + 1) % p.interval == 0) ? p.pull_step : 0.0;
  return delta_continuous;
}

// Constants of the pair kernels (Eq. 1-2 rewritten with exp2).
struct PairConsts {
  // FP32 path, r in fixed-point units (2^-26 A), s = r / r0 - 1.
  // Density pass: e^{-2q s} = gC 2^(gA r + gB) with gA = -(2q/r0) log2(e) 2^-26
  // and gB = -gA r0 2^26 (the two terms cancel exactly at r = r0; one FMA),
  // gC = 2^(exact - rounded gB) putting back gB's FP32 rounding (in xi2g).
  // Force pass: e^{-2q s} = 2^(-kgf t), e^{-(p-2q) s} = 2^(-khf t) with
  // t = r 2^-26 - r0 (an FMA with a single constant: an FMA may read one).
  float rc2f, r0f, kgf, khf;  // rc2f in fixed-point units^2 (2^52 / A^2)
  float xi2g;                 // xi^2 gC: rho = xi2g sum 2^(gA r + gB)
  float Af, fpf;              // fpf = 2 p A / r0
  float fgf;                  // 2 q xi^2 / r0: the density pass stores a_i = fgf / (2 sqrt(rho_i))
  float gA, gB;
  // FP64 path
  double rc2, r0, A, xi2, p, q, fp, fg;  // fp = 2 p / r0, fg = 2 q / r0
  double inv_r0;                          // 1 / r0: s = r inv_r0 - 1
};

// Tabulated EAM tables on the device (tbsma_set_eam).  Each function is a
// piecewise cubic over its grid's intervals: on interval k, with t = s/h - k
// in [0, 1), value = c0 + t (c1 + t (c2 + t c3)); the coefficients are the
// cubic Hermite interpolant of the samples with finite-difference node
// slopes, formed on the host.  FP32 tables serve the mixed pair passes (r in
// fixed-point units, so the grid scale 2^-26 / d_r comes split in two floats
// for a full-precision t), FP64 tables the FP64 passes and every energy.
struct EamDev {
  const float4* f32;   // [n_r - 1] value coefficients of f (density pass)
  const float4* d32;   // [2 (n_r - 1)] per interval {f'0, f'1, f'2, phi'0}, {phi'1, phi'2, 0, 0},
                       // derivative coefficients per A: f'(t) = f'0 + t (f'1 + t f'2);
                       // 32-byte records, 32-byte aligned (read with one 256-bit load)
  const float4* p32;   // [n_r - 1] value coefficients of phi (pair energy)
  const float4* F32;   // [n_rho - 1] value coefficients of F (embedding slope)
  const double* f64;   // [4 (n_r - 1)] value coefficients of f, c0..c3 per interval
  const double* p64;   // [4 (n_r - 1)] of phi
  const double* F64;   // [4 (n_rho - 1)] of F
  float inv_dr_hi, inv_dr_lo;  // 2^-26 / d_r = hi + lo (r in fixed-point units)
  float inv_drho_hi, inv_drho_lo;
  int kmax_r, kmax_rho;        // last interval: n - 2
  double inv_dr, inv_drho;     // 1 / d_r, 1 / d_rho
};

// Neighbour lists hold int16 offsets j - i, by slot, warp-tiled and grouped
// by four: entries 4g..4g+3 of slot t form one 8-byte group, and the groups g
// of 32 consecutive slots are contiguous (256 bytes), so a warp reads four
// entries of each of its atoms with one coalesced load.  cap is a multiple of 4.
constexpr int kMaxOffset = 32767;  // |j - i| an entry can hold

__host__ __device__ __forceinline__ int64_t nbr_group(int64_t i, int g, int cap) {
  return ((i >> 5) * (cap >> 2) + g) * 32 + (i & 31);  // in units of 4 entries
}
__host__ __device__ __forceinline__ int64_t nbr_slot(int64_t i, int k, int cap) {
  return nbr_group(i, k >> 2, cap) * 4 + (k & 3);  // in entries
}

// Exact wrap-around difference of two modular fixed-point coordinates, in A.
__device__ __forceinline__ float fixed_diff(int a, int b) {
  return (float)(int)((unsigned)a - (unsigned)b) * kFixedInv;
}

// ----------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// -> 64-bit multiplies on counter words 0 and 2, the high halves xored into
// the other two words with the round key, the key advanced by the Weyl
// increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += W0;
    k.y += W1;
  }
  return c;
}

__device__ __forceinline__ uint4 thermostat_bits(uint64_t seed, uint32_t atom, uint64_t step,
                                                 uint32_t tag) {
  return philox4x32_10(make_uint4(atom, (uint32_t)step, (uint32_t)(step >> 32), tag),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Box-Muller: u = (bits + 1/2) 2^-32 in (0,1); (u0,u1) -> n0, n1; (u2,u3) -> n2.
__device__ __forceinline__ double3 normals3_f64(uint4 b) {
  const double s = 2.3283064365386962890625e-10;  // 2^-32
  const double two_pi = 6.283185307179586476925286766559;
  const double u0 = ((double)b.x + 0.5) * s, u1 = ((double)b.y + 0.5) * s;
  const double u2 = ((double)b.z + 0.5) * s, u3 = ((double)b.w + 0.5) * s;
  const double a = sqrt(-2.0 * log(u0)), c = sqrt(-2.0 * log(u2));
  double sn, cs, sn2, cs2;
  sincos(two_pi * u1, &sn, &cs);
  sincos(two_pi * u3, &sn2, &cs2);
  return make_double3(a * cs, a * sn, c * cs2);
}

// -ln(u) for u = (b + 1/2) 2^-32 in FP32.  Above u = 1/2 the complement
// 1 - u = (~b + 1/2) 2^-32 is formed from the integer and passed to log1pf, so
// u never rounds to 1 and -ln(u) keeps full relative precision near 0.
__device__ __forceinline__ float neg_log_u32(uint32_t b) {
  const float s = 2.3283064365386963e-10f, h = 1.16415321826934814e-10f;  // 2^-32, 2^-33
  if (b < 0x80000000u) return -logf(fmaf((float)b, s, h));
  return -log1pf(-fmaf((float)(0xFFFFFFFFu - b), s, h));
}

__device__ __forceinline__ float3 normals3_f32(uint4 b) {
  const float s = 2.3283064365386963e-10f, h = 1.16415321826934814e-10f;
  const float u1 = fmaf((float)b.y, s, h), u3 = fmaf((float)b.w, s, h);
  const float a = sqrtf(2.0f * neg_log_u32(b.x)), c = sqrtf(2.0f * neg_log_u32(b.z));
  float sn, cs, sn2, cs2;
  sincospif(2.0f * u1, &sn, &cs);
  sincospif(2.0f * u3, &sn2, &cs2);
  return make_float3(a * cs, a * sn, c * cs2);
}

}  // namespace tbsma
