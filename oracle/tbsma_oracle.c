/*
 * Plain FP64 CPU oracle of the TB-SMA nanowire MD step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, constant or helper with the CUDA library: it has its own
 * copy of the physical constants and its own Philox4x32-10.
 *
 * Everything is double precision, written for clarity, not speed:
 *   - pair sets are rebuilt from scratch at every force call (no skin);
 *   - every pair's exponentials are recomputed in both passes;
 *   - per-atom neighbour sets are held in ascending order of j.
 *
 * Layout: positions and velocities are (n, 3) row-major (x0 y0 z0 x1 ...).
 *
 * Potential (Methods, "TB-SMA potential", Eq. 1-3):
 *   E_B^i = -sqrt(rho_i),  rho_i = sum_j xi^2 exp(-2 q (r_ij/r0 - 1))      (Eq. 1)
 *   E_R^i = sum_j A exp(-p (r_ij/r0 - 1))                                  (Eq. 2)
 *   E_C   = sum_i (E_B^i + E_R^i)                                          (Eq. 3)
 * sums over j != i with r_ij <= r_cut (hard cutoff, 5.8 A).  Each pair enters
 * E_R twice, once from each side (Eq. 2 summed by Eq. 3).
 * Force (derivative of Eq. 3; the text after Eq. 3 notes it needs rho_i and rho_j):
 *   F_i = sum_j [2 (p/r0) phi_ij - (2q/r0) g_ij (1/(2 sqrt rho_i) + 1/(2 sqrt rho_j))]
 *               (r_i - r_j) / r_ij
 * with phi = A exp(-p s), g = xi^2 exp(-2 q s), s = r/r0 - 1.  The two passes
 * (density, then force) follow the paper's two-kernel scheme.
 *
 * The last section holds a tabulated EAM (the general form of that scheme)
 * on the same pair sets: or_eam_interp, or_eam_on_pairs, or_eam_energy_forces.
 */

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- physical constants (CODATA 2018) -------------------------------- */
#define OR_KB_EV_PER_K 8.617333262e-5           /* Boltzmann, eV/K */
#define OR_AMU_KG 1.66053906660e-27             /* atomic mass unit, kg */
#define OR_EV_J 1.602176634e-19                 /* electron volt, J */
/* 1 amu*A^2/fs^2 expressed in eV: amu * 1e-20 m^2 / 1e-30 s^2 / eV */
#define OR_MVV2E (OR_AMU_KG * 1.0e10 / OR_EV_J)

/* Tabulated EAM functions (see the last section). */
typedef struct {
  const double* F;   /* n_rho samples of F(rho), eV */
  int n_rho;
  double d_rho;
  const double* f;   /* n_r samples of f(r) */
  const double* phi; /* n_r samples of phi(r), eV */
  int n_r;
  double d_r;
  double r_cut;
} or_eam;

/* The potential: TB-SMA (Eq. 1-3) with these parameters, or, when eam is
 * not NULL, the tabulated EAM it points to (pairs within eam->r_cut; r0 then
 * only sets the hard-sphere volume of Eq. 5). */
typedef struct {
  double A, xi, p, q, r0, r_cut;
  const or_eam* eam;
} or_pot;

typedef struct {
  double mass;   /* amu */
  double r_skin; /* A, only used to count would-be list rebuilds */
} or_md;

/* One wire's driving parameters. */
typedef struct {
  double L0;          /* initial length, A */
  double strain_rate; /* 1/s */
  double temperature; /* K */
  double gamma;       /* 1/fs, 0 = NVE */
  uint64_t seed;
} or_wire;

double or_mvv2e(void) { return OR_MVV2E; }
double or_kb(void) { return OR_KB_EV_PER_K; }

/* ======================================================================
 * Pair sets.  Output is CSR: start[n+1], nbr[start[i]..start[i+1]) holds
 * every j != i with |r_i - r_j|^2 <= rc^2, in ascending j.  Returns the
 * number of entries, or -1 if it would exceed cap.
 * ==================================================================== */

static double dist2(const double* x, int i, int j) {
  double dx = x[3 * j + 0] - x[3 * i + 0];
  double dy = x[3 * j + 1] - x[3 * i + 1];
  double dz = x[3 * j + 2] - x[3 * i + 2];
  return dx * dx + dy * dy + dz * dz;
}

long or_pairs_brute(int n, const double* x, double rc, int* start, int* nbr, long cap) {
  double rc2 = rc * rc;
  long k = 0;
  for (int i = 0; i < n; ++i) {
    start[i] = (int)k;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      if (dist2(x, i, j) <= rc2) {
        if (k >= cap) return -1;
        nbr[k++] = j;
      }
    }
  }
  start[n] = (int)k;
  return k;
}

static int cmp_int(const void* a, const void* b) {
  int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

/* Same pair set found through a cell grid of edge >= rc over the bounding box:
 * each atom only tests the 27 cells around its own.  Lists are sorted so the
 * result is identical to or_pairs_brute. */
long or_pairs_cells(int n, const double* x, double rc, int* start, int* nbr, long cap) {
  if (n == 0) {
    start[0] = 0;
    return 0;
  }
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) lo[d] = hi[d] = x[d];
  for (int i = 1; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      if (x[3 * i + d] < lo[d]) lo[d] = x[3 * i + d];
      if (x[3 * i + d] > hi[d]) hi[d] = x[3 * i + d];
    }
  int nc[3];
  double edge[3];
  for (int d = 0; d < 3; ++d) {
    double ext = hi[d] - lo[d];
    nc[d] = (int)floor(ext / rc);
    if (nc[d] < 1) nc[d] = 1;
    edge[d] = ext / nc[d];
    if (edge[d] < rc) edge[d] = rc; /* keep edge >= rc */
  }
  long ncell = (long)nc[0] * nc[1] * nc[2];
  int* head = (int*)malloc(sizeof(int) * ncell);
  int* next = (int*)malloc(sizeof(int) * n);
  int* cell = (int*)malloc(sizeof(int) * 3 * n);
  for (long c = 0; c < ncell; ++c) head[c] = -1;
  for (int i = n - 1; i >= 0; --i) {
    int ci[3];
    for (int d = 0; d < 3; ++d) {
      int v = (int)floor((x[3 * i + d] - lo[d]) / edge[d]);
      if (v < 0) v = 0;
      if (v >= nc[d]) v = nc[d] - 1;
      ci[d] = v;
      cell[3 * i + d] = v;
    }
    long c = ((long)ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
    next[i] = head[c];
    head[c] = i;
  }
  double rc2 = rc * rc;
  long k = 0;
  int overflow = 0;
  for (int i = 0; i < n && !overflow; ++i) {
    start[i] = (int)k;
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b)
        for (int c = -1; c <= 1; ++c) {
          int cx = cell[3 * i] + a, cy = cell[3 * i + 1] + b, cz = cell[3 * i + 2] + c;
          if (cx < 0 || cy < 0 || cz < 0 || cx >= nc[0] || cy >= nc[1] || cz >= nc[2]) continue;
          for (int j = head[((long)cx * nc[1] + cy) * nc[2] + cz]; j >= 0; j = next[j]) {
            if (j == i) continue;
            if (dist2(x, i, j) <= rc2) {
              if (k >= cap) {
                overflow = 1;
                break;
              }
              nbr[k++] = j;
            }
          }
        }
    qsort(nbr + start[i], (size_t)(k - start[i]), sizeof(int), cmp_int);
  }
  start[n] = (int)k;
  free(head);
  free(next);
  free(cell);
  return overflow ? -1 : k;
}

/* ======================================================================
 * TB-SMA energy and forces on a given pair set (Eq. 1-3), two passes.
 * Outputs are optional (NULL skips): rho[n], F[n][3], eB[n], eR[n],
 * w[n] = 1/2 sum_j (x_j - x_i) F_ij,x  (per-atom axial pair virial, Eq. 5),
 * S[n] = sum_j |f_ij| (scale of the pair forces acting on i).
 * Returns E_C.
 * ==================================================================== */
double or_tbsma(const or_pot* P, int n, const double* x, const int* start, const int* nbr,
                double* rho, double* F, double* eB, double* eR, double* w, double* S) {
  double* rh = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* inv = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double E = 0.0;
  /* pass 1: density rho_i (Eq. 1) */
  for (int i = 0; i < n; ++i) {
    double r_i = 0.0;
    for (int k = start[i]; k < start[i + 1]; ++k) {
      int j = nbr[k];
      double r = sqrt(dist2(x, i, j));
      double s = r / P->r0 - 1.0;
      r_i += P->xi * P->xi * exp(-2.0 * P->q * s);
    }
    rh[i] = r_i;
    /* 1/(2 sqrt(rho)); an atom without neighbours has no band energy and no force */
    inv[i] = r_i > 0.0 ? 1.0 / (2.0 * sqrt(r_i)) : 0.0;
    double e_b = -sqrt(r_i);
    if (rho) rho[i] = r_i;
    if (eB) eB[i] = e_b;
    E += e_b;
  }
  /* pass 2: forces, repulsive energy (Eq. 2), virial */
  for (int i = 0; i < n; ++i) {
    double fx = 0.0, fy = 0.0, fz = 0.0, e_r = 0.0, wi = 0.0, si = 0.0;
    for (int k = start[i]; k < start[i + 1]; ++k) {
      int j = nbr[k];
      double dx = x[3 * i + 0] - x[3 * j + 0];
      double dy = x[3 * i + 1] - x[3 * j + 1];
      double dz = x[3 * i + 2] - x[3 * j + 2];
      double r = sqrt(dx * dx + dy * dy + dz * dz);
      double s = r / P->r0 - 1.0;
      double phi = P->A * exp(-P->p * s);
      double g = P->xi * P->xi * exp(-2.0 * P->q * s);
      double f = 2.0 * (P->p / P->r0) * phi - (2.0 * P->q / P->r0) * g * (inv[i] + inv[j]);
      fx += f * dx / r;
      fy += f * dy / r;
      fz += f * dz / r;
      e_r += phi;
      /* r_x,ij = x_j - x_i = -dx ; F_x,ij = f dx / r */
      wi += 0.5 * (-dx) * (f * dx / r);
      si += fabs(f);
    }
    if (F) {
      F[3 * i + 0] = fx;
      F[3 * i + 1] = fy;
      F[3 * i + 2] = fz;
    }
    if (eR) eR[i] = e_r;
    if (w) w[i] = wi;
    if (S) S[i] = si;
    E += e_r;
  }
  free(rh);
  free(inv);
  return E;
}

double or_eam_energy_forces(const or_eam* T, int n, const double* x, int brute_max, double* F,
                            double* rho, double* eB, double* eR, double* w, double* S,
                            long* n_pairs_out);

/* Convenience: pair set (brute force if n <= brute_max, else cells) + Eq. 1-3
 * (or the tabulated EAM when P->eam is set). */
double or_energy_forces(const or_pot* P, int n, const double* x, int brute_max, double* F,
                        double* rho, double* eB, double* eR, double* w, double* S,
                        long* n_pairs_out) {
  if (P->eam) return or_eam_energy_forces(P->eam, n, x, brute_max, F, rho, eB, eR, w, S, n_pairs_out);
  long cap = 64L * n + 64;
  int* start = (int*)malloc(sizeof(int) * (n + 1));
  int* nbr = NULL;
  long k;
  for (;;) {
    nbr = (int*)malloc(sizeof(int) * cap);
    k = (n <= brute_max) ? or_pairs_brute(n, x, P->r_cut, start, nbr, cap)
                         : or_pairs_cells(n, x, P->r_cut, start, nbr, cap);
    if (k >= 0) break;
    free(nbr);
    cap *= 2;
  }
  double E = or_tbsma(P, n, x, start, nbr, rho, F, eB, eR, w, S);
  if (n_pairs_out) *n_pairs_out = k;
  free(start);
  free(nbr);
  return E;
}

/* ======================================================================
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): a 10-round bijection of
 * a 128-bit counter under a 64-bit key.  Each round multiplies counter words
 * 0 and 2 by the constants M0, M1 (full 64-bit products), and forms
 *   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
 * the key is advanced by the Weyl constants W0, W1 between rounds.
 * ==================================================================== */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += OR_PHILOX_W0;
      k1 += OR_PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

void or_philox_many(long n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  for (long i = 0; i < n; ++i) or_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* Three standard normals for one atom and one draw.
 * key = (seed lo, seed hi); counter = (atom index in wire, step lo, step hi, tag),
 * tag 0 = thermostat, tag 1 = initial velocities.
 * u_k = (x_k + 1/2) 2^-32 lies in (0, 1); Box-Muller on (u0,u1) gives n0, n1
 * and on (u2,u3) gives n2. */
void or_normals3(uint64_t seed, uint32_t atom, uint64_t step, uint32_t tag, double out[3]) {
  uint32_t ctr[4] = {atom, (uint32_t)step, (uint32_t)(step >> 32), tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  or_philox4x32_10(ctr, key, r);
  const double two_m32 = 1.0 / 4294967296.0;
  const double two_pi = 6.283185307179586476925286766559;
  double u0 = ((double)r[0] + 0.5) * two_m32;
  double u1 = ((double)r[1] + 0.5) * two_m32;
  double u2 = ((double)r[2] + 0.5) * two_m32;
  double u3 = ((double)r[3] + 0.5) * two_m32;
  double a = sqrt(-2.0 * log(u0));
  double b = sqrt(-2.0 * log(u2));
  out[0] = a * cos(two_pi * u1);
  out[1] = a * sin(two_pi * u1);
  out[2] = b * cos(two_pi * u3);
}

void or_normals_many(long n, uint64_t seed, const uint32_t* atom, uint64_t step, uint32_t tag,
                     double* out) {
  for (long i = 0; i < n; ++i) or_normals3(seed, atom[i], step, tag, out + 3 * i);
}

/* ======================================================================
 * Initial velocities (Methods: Gaussian velocities at the start of each
 * trajectory).  Mobile atoms draw Gaussian velocities at T from Philox tag 1,
 * the mobile centre-of-mass velocity is removed, and the velocities are
 * scaled so that T = 2 E_kin / (3 N_mobile k_B) exactly.  Grip atoms get 0.
 * ==================================================================== */
void or_init_velocities(const or_md* M, int n, const uint8_t* kind, uint64_t seed, double T,
                        double* v) {
  double sig = sqrt(OR_KB_EV_PER_K * T / (M->mass * OR_MVV2E)); /* A/fs */
  double sum[3] = {0, 0, 0};
  long nm = 0;
  for (int i = 0; i < n; ++i) {
    if (kind[i] != 0) {
      v[3 * i] = v[3 * i + 1] = v[3 * i + 2] = 0.0;
      continue;
    }
    double g[3];
    or_normals3(seed, (uint32_t)i, 0, 1, g);
    for (int d = 0; d < 3; ++d) {
      v[3 * i + d] = sig * g[d];
      sum[d] += v[3 * i + d];
    }
    ++nm;
  }
  if (nm == 0) return;
  double v2 = 0.0;
  for (int i = 0; i < n; ++i) {
    if (kind[i] != 0) continue;
    for (int d = 0; d < 3; ++d) {
      v[3 * i + d] -= sum[d] / (double)nm;
      v2 += v[3 * i + d] * v[3 * i + d];
    }
  }
  double ekin = 0.5 * M->mass * OR_MVV2E * v2;
  double target = 1.5 * (double)nm * OR_KB_EV_PER_K * T;
  double scale = (ekin > 0.0) ? sqrt(target / ekin) : 0.0;
  for (int i = 0; i < n; ++i)
    if (kind[i] == 0)
      for (int d = 0; d < 3; ++d) v[3 * i + d] *= scale;
}

/* ======================================================================
 * MD steps for one wire (Methods, "Simulation details"):
 * velocity-Verlet with dt, split as B A O A B (Langevin "BAOAB"):
 *   B: v += (dt/2) F/m          A: x += (dt/2) v
 *   O: v  = c1 v + c2 sqrt(kT/m) n,  c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2)
 * gamma = 0 gives plain velocity Verlet (NVE).  Grip atoms (kind 1, 2) are
 * rigid: not integrated, v = 0, and moved by -/+ delta per step with
 * delta = strain_rate * L0 * dt / 2 (each end moves half the elongation).
 * F is the force at the input positions on entry and at the output positions
 * on exit.  `d_grip` accumulates delta.  `n_rebuild` counts the steps at
 * which some atom moved more than r_skin/2 from its position at the last
 * count (the Verlet-list rebuild rule with skin r_skin); x_build holds those
 * positions.  `step0` is the index of the first step (thermostat counter).
 * ==================================================================== */
void or_md_steps(const or_pot* P, const or_md* M, const or_wire* W, int n, double* x, double* v,
                 const uint8_t* kind, double* F, double* x_build, int64_t step0, int64_t n_steps,
                 double dt, double* d_grip, int64_t* n_rebuild, int brute_max) {
  double inv_m = 1.0 / (M->mass * OR_MVV2E); /* (A/fs^2) per (eV/A) */
  double c1 = exp(-W->gamma * dt);
  double c2 = sqrt(1.0 - c1 * c1);
  double sig = sqrt(OR_KB_EV_PER_K * W->temperature * inv_m);
  double delta = W->strain_rate * 1.0e-15 * W->L0 * dt / 2.0;
  double half_skin2 = 0.25 * M->r_skin * M->r_skin;
  for (int64_t s = 0; s < n_steps; ++s) {
    int64_t step = step0 + s;
    for (int i = 0; i < n; ++i) {
      if (kind[i] == 0) {
        for (int d = 0; d < 3; ++d) v[3 * i + d] += 0.5 * dt * F[3 * i + d] * inv_m; /* B */
        for (int d = 0; d < 3; ++d) x[3 * i + d] += 0.5 * dt * v[3 * i + d];         /* A */
        double g[3];
        or_normals3(W->seed, (uint32_t)i, (uint64_t)step, 0, g);
        for (int d = 0; d < 3; ++d) v[3 * i + d] = c1 * v[3 * i + d] + c2 * sig * g[d]; /* O */
        for (int d = 0; d < 3; ++d) x[3 * i + d] += 0.5 * dt * v[3 * i + d];              /* A */
      } else {
        x[3 * i + 0] += (kind[i] == 1) ? -delta : delta;
        v[3 * i + 0] = v[3 * i + 1] = v[3 * i + 2] = 0.0;
      }
    }
    *d_grip += delta;
    if (x_build) {
      int need = 0;
      for (int i = 0; i < n && !need; ++i) {
        double dx = x[3 * i] - x_build[3 * i], dy = x[3 * i + 1] - x_build[3 * i + 1],
               dz = x[3 * i + 2] - x_build[3 * i + 2];
        if (dx * dx + dy * dy + dz * dz > half_skin2) need = 1;
      }
      if (need) {
        memcpy(x_build, x, sizeof(double) * 3 * n);
        if (n_rebuild) ++*n_rebuild;
      }
    }
    or_energy_forces(P, n, x, brute_max, F, NULL, NULL, NULL, NULL, NULL, NULL);
    for (int i = 0; i < n; ++i)
      if (kind[i] == 0)
        for (int d = 0; d < 3; ++d) v[3 * i + d] += 0.5 * dt * F[3 * i + d] * inv_m; /* B */
  }
}

/* Many independent wires: wire w owns atoms offset[w] .. offset[w]+count[w].
 * Wires are independent, so they run in parallel over the host's threads. */
void or_md_batch(const or_pot* P, const or_md* M, int n_wires, const or_wire* W,
                 const long* offset, const int* count, double* x, double* v, const uint8_t* kind,
                 double* F, double* x_build, int64_t step0, int64_t n_steps, double dt,
                 double* d_grip, int64_t* n_rebuild, int brute_max) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int w = 0; w < n_wires; ++w) {
    long o = offset[w];
    or_md_steps(P, M, &W[w], count[w], x + 3 * o, v + 3 * o, kind + o, F + 3 * o,
                x_build ? x_build + 3 * o : NULL, step0, n_steps, dt, &d_grip[w],
                n_rebuild ? &n_rebuild[w] : NULL, brute_max);
  }
}

/* ======================================================================
 * Paper protocol mode (Methods, "Simulation details": Nosé–Hoover
 * thermostat, velocity Verlet with dt = 2 fs, grips displaced by 0.05 A
 * every 20 ps, temperature ramped from 0.01 K to the target).
 *
 * Thermostat (thermostat = 1).  One Nosé–Hoover variable xi per wire with
 * g = 3 N_mobile degrees of freedom and mass Q = g k_B T_w tau^2 (T_w the
 * wire's target temperature, tau the thermostat period).  Equations of
 * motion for the mobile atoms:
 *   dx/dt = v,  dv/dt = F/m - xi v,  dxi/dt = (2K - g k_B T)/Q,  deta/dt = xi
 * with K = 1/2 m sum v^2.  A step of length dt is the symmetric splitting
 *   NH(dt/2)  B(dt/2)  A(dt)  [forces]  B(dt/2)  NH(dt/2)
 * where B: v += (dt/2) F/m, A: x += dt v, and NH(h) is
 *   xi += (h/2) (2K - g k_B T)/Q;  v *= exp(-xi h);  eta += h xi;
 *   xi += (h/2) (2K' - g k_B T)/Q   (K' the kinetic energy after scaling)
 * (the single-thermostat case of the Martyna–Tuckerman–Klein factorisation).
 * The extended energy E_pot + K + Q xi^2/2 + g k_B T eta is conserved when
 * T is constant.  A wire with T_w = 0 or no mobile atom runs NVE (xi = 0).
 * thermostat = 0 keeps the Langevin B A O A B step of or_md_steps.
 *
 * Target temperature at step index s (0-based): T(s) = t_start +
 * (T_w - t_start) clamp((s - ramp_start) / ramp_steps, 0, 1), or T_w when
 * ramp_steps = 0 (the paper holds 0.01 K during its barostat phase, then
 * ramps: ramp_start is the first step of the ramp).  The
 * NH half step at the start of step s and the one at its end use T(s).
 *
 * Pull (pull = 1, stepwise): in step s each grip moves by -/+ pull_step
 * (rigidly) when (s + 1) is a multiple of pull_interval, else not at all;
 * pull = 0 keeps the continuous delta = strain_rate L0 dt / 2 per step.
 *
 * Axial Nosé–Hoover barostat (baro_tau > 0; Methods: the wire is first
 * equilibrated for 100 ps at zero pressure along [100] with a Nosé–Hoover
 * barostat).  One strain-rate variable zeta (1/fs) per wire, the wire's
 * axial log-stretch lambda, and Hoover's constant-stress equations along x
 * about the centre c of the grips (the mean x of the grip atoms):
 *   dx/dt = v_x + zeta (x - c)            (every atom; grips have v = 0)
 *   dv_x/dt = F_x/m - zeta v_x            (mobile atoms)
 *   dzeta/dt = -V (sigma_xx - P) / W_b - gamma_b zeta,  dlambda/dt = zeta,
 * sigma_xx the wire's axial stress (Eq. 5, tension positive, V = N (4/3)
 * pi (r0/2)^3), P = baro_pressure and barostat mass W_b = V B tau_b^2
 * (B = baro_modulus, tau_b = baro_tau: a wire of axial modulus B oscillates
 * with angular frequency 1/tau_b) and drag gamma_b = baro_drag / tau_b.
 * Because V sigma_xx = -sum_i F_x,i (x_i - c) - m sum v_x^2, these conserve
 * (with the grips held, no thermostat and no drag) H = E_pot + K +
 * W_b zeta^2/2 - P V lambda.  At the paper's 0.01 K nothing else damps the
 * barostat's oscillation, so the drag (a reading: the paper names the
 * barostat only) is what lets the length settle.  A step is the symmetric
 * splitting (h = dt/2)
 *   Z(h) C(h) [NH(h)] B(h) S(h) A(dt) S(h) [forces] B(h) [NH(h)] C(h) Z(h)
 * with Z(h): zeta *= exp(-gamma_b h), then zeta -= h V (sigma_xx - P)/W_b
 * at the current state (at the step's end: the kick, then the drag), C(h):
 * mobile v_x *= exp(-zeta h), S(h): x = c + (x - c) exp(zeta h) for every
 * atom and lambda += zeta h; A(dt) is the thermostat's drift (A, or A O A
 * under Langevin) with the grip displacement, and c is taken once per step,
 * at its start (the scaling and the symmetric grip moves leave it fixed).
 * ==================================================================== */
typedef struct {
  int thermostat;        /* 0 Langevin (B A O A B), 1 Nosé–Hoover */
  int pull;              /* 0 continuous, 1 stepwise */
  double tau;            /* Nosé–Hoover period, fs */
  double pull_step;      /* stepwise: displacement of each grip per event, A */
  int64_t pull_interval; /* stepwise: steps per event */
  double t_start;        /* ramp start temperature, K */
  int64_t ramp_steps;    /* 0: no ramp */
  double baro_tau;       /* axial barostat time tau_b, fs; 0: off */
  double baro_modulus;   /* its reference modulus B, eV/A^3 */
  double baro_pressure;  /* its target sigma_xx, eV/A^3 */
  double baro_drag;      /* its drag gamma_b in units of 1/tau_b */
  int64_t ramp_start;    /* first step of the ramp */
} or_protocol;

double or_target_temperature(const or_protocol* R, double T_w, int64_t s) {
  if (R->ramp_steps <= 0) return T_w;
  if (s < R->ramp_start) return R->t_start;
  double f = (double)(s - R->ramp_start) / (double)R->ramp_steps;
  if (f > 1.0) f = 1.0;
  return R->t_start + (T_w - R->t_start) * f;
}

static double kinetic(int n, const double* v, const uint8_t* kind, double m_e) {
  double v2 = 0.0;
  for (int i = 0; i < n; ++i)
    if (kind[i] == 0)
      v2 += v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
  return 0.5 * m_e * v2;
}

/* One NH half step of length h on the mobile velocities (see above). */
static void nh_half(int n, double* v, const uint8_t* kind, double m_e, double g, double kT,
                    double Q, double h, double* xi, double* eta) {
  double K = kinetic(n, v, kind, m_e);
  *xi += 0.5 * h * (2.0 * K - g * kT) / Q;
  double sc = exp(-*xi * h);
  for (int i = 0; i < n; ++i)
    if (kind[i] == 0)
      for (int d = 0; d < 3; ++d) v[3 * i + d] *= sc;
  *eta += h * *xi;
  K = kinetic(n, v, kind, m_e);
  *xi += 0.5 * h * (2.0 * K - g * kT) / Q;
}

/* Axial stress of a wire (Eq. 5 with D7's hard-sphere volume). */
static double axial_stress(const or_pot* P, const or_md* M, int n, const double* x,
                           const double* v, const uint8_t* kind, int brute_max) {
  double* w = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  or_energy_forces(P, n, x, brute_max, NULL, NULL, NULL, NULL, w, NULL, NULL);
  double vir = 0.0, mv2x = 0.0;
  for (int i = 0; i < n; ++i) {
    vir += w[i];
    if (kind[i] == 0) mv2x += v[3 * i] * v[3 * i];
  }
  free(w);
  const double pi = 3.141592653589793238462643383279;
  double rhs = 0.5 * P->r0;
  double V = (double)n * (4.0 / 3.0) * pi * rhs * rhs * rhs;
  return (vir - M->mass * OR_MVV2E * mv2x) / V;
}

/* Z(h): the drag zeta *= exp(-gamma_b h) and the kick zeta -= h V (sigma_xx
 * - P) / W_b = h (sigma_xx - P) / (B tau_b^2); drag first at a step's start
 * (end = 0), kick first at its end (end = 1). */
static void baro_z(const or_pot* P, const or_md* M, const or_protocol* R, int n, const double* x,
                   const double* v, const uint8_t* kind, int brute_max, double h, int end,
                   double* zeta) {
  double drag = exp(-R->baro_drag / R->baro_tau * h);
  if (!end) *zeta *= drag;
  double sig = axial_stress(P, M, n, x, v, kind, brute_max);
  *zeta -= h * (sig - R->baro_pressure) / (R->baro_modulus * R->baro_tau * R->baro_tau);
  if (end) *zeta *= drag;
}

/* C(h): mobile v_x *= exp(-zeta h). */
static void baro_c(int n, double* v, const uint8_t* kind, double zeta, double h) {
  double sc = exp(-zeta * h);
  for (int i = 0; i < n; ++i)
    if (kind[i] == 0) v[3 * i] *= sc;
}

/* S(h): every atom's x = c + (x - c) exp(zeta h); lambda += zeta h. */
static void baro_s(int n, double* x, double c, double zeta, double h, double* lambda) {
  double mu = exp(zeta * h);
  for (int i = 0; i < n; ++i) x[3 * i] = c + (x[3 * i] - c) * mu;
  *lambda += zeta * h;
}

/* Protocol-mode MD steps for one wire; arguments as or_md_steps, plus the
 * protocol and the wire's state nh = {xi, eta, lambda, zeta} (in/out: the
 * Nosé–Hoover variable, its integral, the barostat's log-stretch and its
 * strain rate). */
void or_md_steps_protocol(const or_pot* P, const or_md* M, const or_wire* W, const or_protocol* R,
                          int n, double* x, double* v, const uint8_t* kind, double* F,
                          double* x_build, int64_t step0, int64_t n_steps, double dt,
                          double* d_grip, int64_t* n_rebuild, double nh[4], int brute_max) {
  double m_e = M->mass * OR_MVV2E;
  double inv_m = 1.0 / m_e;
  double c1 = exp(-W->gamma * dt);
  double c2 = sqrt(1.0 - c1 * c1);
  double half_skin2 = 0.25 * M->r_skin * M->r_skin;
  long nm = 0;
  for (int i = 0; i < n; ++i) nm += kind[i] == 0;
  double g = 3.0 * (double)nm;
  double Q = g * OR_KB_EV_PER_K * W->temperature * R->tau * R->tau;
  int nh_on = R->thermostat == 1 && Q > 0.0;
  int baro_on = R->baro_tau > 0.0;
  for (int64_t s = 0; s < n_steps; ++s) {
    int64_t step = step0 + s;
    double c = 0.0;
    if (baro_on) {
      long ng = 0;
      for (int i = 0; i < n; ++i)
        if (kind[i] != 0) c += x[3 * i], ++ng;
      c = ng > 0 ? c / (double)ng : 0.0;
      baro_z(P, M, R, n, x, v, kind, brute_max, 0.5 * dt, 0, &nh[3]); /* Z(h) */
      baro_c(n, v, kind, nh[3], 0.5 * dt);                             /* C(h) */
    }
    double T = or_target_temperature(R, W->temperature, step);
    double kT = OR_KB_EV_PER_K * T;
    double delta;
    if (R->pull == 1)
      delta = (R->pull_interval > 0 && (step + 1) % R->pull_interval == 0) ? R->pull_step : 0.0;
    else
      delta = W->strain_rate * 1.0e-15 * W->L0 * dt / 2.0;
    if (R->thermostat == 1) {
      if (nh_on) nh_half(n, v, kind, m_e, g, kT, Q, 0.5 * dt, &nh[0], &nh[1]);
      for (int i = 0; i < n; ++i)
        if (kind[i] == 0)
          for (int d = 0; d < 3; ++d) v[3 * i + d] += 0.5 * dt * F[3 * i + d] * inv_m; /* B */
      if (baro_on) baro_s(n, x, c, nh[3], 0.5 * dt, &nh[2]);                       /* S(h) */
      for (int i = 0; i < n; ++i) {
        if (kind[i] == 0) {
          for (int d = 0; d < 3; ++d) x[3 * i + d] += dt * v[3 * i + d]; /* A */
        } else {
          x[3 * i + 0] += (kind[i] == 1) ? -delta : delta;
          v[3 * i + 0] = v[3 * i + 1] = v[3 * i + 2] = 0.0;
        }
      }
    } else {
      double sig = sqrt(kT * inv_m);
      for (int i = 0; i < n; ++i)
        if (kind[i] == 0)
          for (int d = 0; d < 3; ++d) v[3 * i + d] += 0.5 * dt * F[3 * i + d] * inv_m; /* B */
      if (baro_on) baro_s(n, x, c, nh[3], 0.5 * dt, &nh[2]);                       /* S(h) */
      for (int i = 0; i < n; ++i) {
        if (kind[i] == 0) {
          for (int d = 0; d < 3; ++d) x[3 * i + d] += 0.5 * dt * v[3 * i + d];         /* A */
          double gn[3];
          or_normals3(W->seed, (uint32_t)i, (uint64_t)step, 0, gn);
          for (int d = 0; d < 3; ++d) v[3 * i + d] = c1 * v[3 * i + d] + c2 * sig * gn[d]; /* O */
          for (int d = 0; d < 3; ++d) x[3 * i + d] += 0.5 * dt * v[3 * i + d];               /* A */
        } else {
          x[3 * i + 0] += (kind[i] == 1) ? -delta : delta;
          v[3 * i + 0] = v[3 * i + 1] = v[3 * i + 2] = 0.0;
        }
      }
    }
    if (baro_on) baro_s(n, x, c, nh[3], 0.5 * dt, &nh[2]); /* S(h) */
    *d_grip += delta;
    if (x_build) {
      int need = 0;
      for (int i = 0; i < n && !need; ++i) {
        double dx = x[3 * i] - x_build[3 * i], dy = x[3 * i + 1] - x_build[3 * i + 1],
               dz = x[3 * i + 2] - x_build[3 * i + 2];
        if (dx * dx + dy * dy + dz * dz > half_skin2) need = 1;
      }
      if (need) {
        memcpy(x_build, x, sizeof(double) * 3 * n);
        if (n_rebuild) ++*n_rebuild;
      }
    }
    or_energy_forces(P, n, x, brute_max, F, NULL, NULL, NULL, NULL, NULL, NULL);
    for (int i = 0; i < n; ++i)
      if (kind[i] == 0)
        for (int d = 0; d < 3; ++d) v[3 * i + d] += 0.5 * dt * F[3 * i + d] * inv_m; /* B */
    if (nh_on) nh_half(n, v, kind, m_e, g, kT, Q, 0.5 * dt, &nh[0], &nh[1]);
    if (baro_on) {
      baro_c(n, v, kind, nh[3], 0.5 * dt);                             /* C(h) */
      baro_z(P, M, R, n, x, v, kind, brute_max, 0.5 * dt, 1, &nh[3]); /* Z(h) */
    }
  }
}

/* Many wires in protocol mode; nh is [n_wires][4]. */
void or_md_batch_protocol(const or_pot* P, const or_md* M, const or_protocol* R, int n_wires,
                          const or_wire* W, const long* offset, const int* count, double* x,
                          double* v, const uint8_t* kind, double* F, double* x_build,
                          int64_t step0, int64_t n_steps, double dt, double* d_grip,
                          int64_t* n_rebuild, double* nh, int brute_max) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int w = 0; w < n_wires; ++w) {
    long o = offset[w];
    or_md_steps_protocol(P, M, &W[w], R, count[w], x + 3 * o, v + 3 * o, kind + o, F + 3 * o,
                         x_build ? x_build + 3 * o : NULL, step0, n_steps, dt, &d_grip[w],
                         n_rebuild ? &n_rebuild[w] : NULL, nh + 4 * w, brute_max);
  }
}

/* ======================================================================
 * Wire topology: rupture and neck (Results, "Nanowire elongation": a wire
 * fails when it separates into two pieces; the final neck is its thinnest
 * cross-section before that; the paper gives no formal definition).
 *
 * Clusters: connected components of the graph whose edges are the pairs
 * with r_ij <= r_cut (the interacting pairs), found by union-find; every
 * component is labelled by its smallest atom index.  connected = 1 when a
 * left-grip atom (kind 1) and a right-grip atom (kind 2) share a component.
 * Neck: between the largest x of the left grip (x_lo) and the smallest x of
 * the right grip (x_hi), slab k covers x_lo + (k + 1/2) w <= x < x_lo +
 * (k + 3/2) w, k = 0 .. n_slabs - 1 with n_slabs = floor((x_hi - x_lo) / w
 * - 1/2) and w = a/2, the spacing of the (100) planes, so that each (100) plane
 * of the unstrained wire lies at the centre of one slab; the neck is the
 * smallest count of atoms in a slab and its index (the first one on ties).
 * out[0] connected, out[1] n_clusters, out[2] neck count, out[3] neck slab,
 * out[4] n_slabs; label[n] (may be NULL) receives the component labels.
 * Returns -1 if a grip is missing or the pair set does not fit in `cap`.
 * ==================================================================== */
static int uf_find(int* parent, int a) {
  while (parent[a] != a) a = parent[a];
  return a;
}

long or_topology(int n, const double* x, const uint8_t* kind, double rc, double w, long cap,
                 int* label, long out[5]) {
  int* start = (int*)malloc(sizeof(int) * (n + 1));
  int* nbr = (int*)malloc(sizeof(int) * (cap > 0 ? cap : 1));
  int* parent = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  long k = or_pairs_cells(n, x, rc, start, nbr, cap);
  if (k < 0) {
    free(start), free(nbr), free(parent);
    return -1;
  }
  for (int i = 0; i < n; ++i) parent[i] = i;
  for (int i = 0; i < n; ++i)
    for (int e = start[i]; e < start[i + 1]; ++e) {
      int ra = uf_find(parent, i), rb = uf_find(parent, nbr[e]);
      if (ra == rb) continue;
      if (ra < rb) parent[rb] = ra; /* the smaller index stays the root */
      else parent[ra] = rb;
    }
  long n_clusters = 0;
  int left = -1, right = -1;
  double x_lo = -1e300, x_hi = 1e300;
  for (int i = 0; i < n; ++i) {
    int r = uf_find(parent, i);
    if (label) label[i] = r;
    if (r == i) ++n_clusters;
    if (kind[i] == 1) {
      if (left < 0) left = i;
      if (x[3 * i] > x_lo) x_lo = x[3 * i];
    } else if (kind[i] == 2) {
      if (right < 0) right = i;
      if (x[3 * i] < x_hi) x_hi = x[3 * i];
    }
  }
  if (left < 0 || right < 0) {
    free(start), free(nbr), free(parent);
    return -1;
  }
  long n_slabs = (x_hi > x_lo) ? (long)floor((x_hi - x_lo) / w - 0.5) : 0;
  if (n_slabs < 0) n_slabs = 0;
  long neck = 0, neck_slab = -1;
  if (n_slabs > 0) {
    long* cnt = (long*)calloc((size_t)n_slabs, sizeof(long));
    for (int i = 0; i < n; ++i) {
      double u = (x[3 * i] - x_lo) / w - 0.5;
      if (u >= 0.0 && u < (double)n_slabs) cnt[(long)floor(u)] += 1;
    }
    neck = cnt[0];
    neck_slab = 0;
    for (long s = 1; s < n_slabs; ++s)
      if (cnt[s] < neck) neck = cnt[s], neck_slab = s;
    free(cnt);
  }
  out[0] = uf_find(parent, left) == uf_find(parent, right);
  out[1] = n_clusters;
  out[2] = neck;
  out[3] = neck_slab;
  out[4] = n_slabs;
  free(start), free(nbr), free(parent);
  return 0;
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ======================================================================
 * Per-wire observables (Eq. 4-5):
 *   strain   = (L - L0)/L0 with L = L0 + 2 d_grip                        (Eq. 4)
 *   virial   = sum_i 1/2 sum_j r_x,ij F_x,ij,  r_x,ij = x_j - x_i,
 *              F_ij the force on i due to j (tension positive)
 *   sigma_xx = (virial - m sum_mobile v_x,i^2) / V,
 *              V = N (4/3) pi (r0/2)^3  (hard-sphere volume, constant)  (Eq. 5)
 *   E_pot = E_C, E_kin = 1/2 m sum_mobile |v|^2, T = 2 E_kin/(3 N_mob k_B)
 * out = {e_pot, e_kin, temp, sigma_xx (eV/A^3), virial (eV), strain}
 * ==================================================================== */
void or_observables(const or_pot* P, const or_md* M, const or_wire* W, int n, const double* x,
                    const double* v, const uint8_t* kind, double d_grip, int brute_max,
                    double out[6]) {
  double* w = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double E = or_energy_forces(P, n, x, brute_max, NULL, NULL, NULL, NULL, w, NULL, NULL);
  double vir = 0.0, mv2x = 0.0, v2 = 0.0;
  long nm = 0;
  for (int i = 0; i < n; ++i) {
    vir += w[i];
    if (kind[i] == 0) {
      mv2x += v[3 * i] * v[3 * i];
      v2 += v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
      ++nm;
    }
  }
  double m_e = M->mass * OR_MVV2E;
  double ekin = 0.5 * m_e * v2;
  const double pi = 3.141592653589793238462643383279;
  double rhs = 0.5 * P->r0;
  double V = (double)n * (4.0 / 3.0) * pi * rhs * rhs * rhs;
  out[0] = E;
  out[1] = ekin;
  out[2] = nm > 0 ? 2.0 * ekin / (3.0 * (double)nm * OR_KB_EV_PER_K) : 0.0;
  out[3] = (vir - m_e * mv2x) / V;
  out[4] = vir;
  out[5] = 2.0 * d_grip / W->L0;
  free(w);
}

/* ======================================================================
 * Tabulated embedded-atom method (EAM) on the same pair sets.
 *
 * The paper builds its TB-SMA force on the two-stage structure of the EAM
 * implementation it cites (Introduction; Methods, "TB-SMA potential"): a
 * density loop over i's neighbours, then a force loop that needs the
 * embedding derivative of both i and j.  EAM in its general form:
 *   rho_i = sum_j f(r_ij),   E = sum_i [ F(rho_i) + 1/2 sum_j phi(r_ij) ],
 *   F_i   = -sum_j [ phi'(r_ij) + (F'(rho_i) + F'(rho_j)) f'(r_ij) ] (r_i - r_j)/r_ij,
 * pairs j != i with r_ij <= r_cut.  TB-SMA is the case f = xi^2 e^{-2qs},
 * phi = 2 A e^{-ps}, F = -sqrt(rho).
 *
 * F, f and phi are given as samples on uniform grids (F at rho = k d_rho,
 * f and phi at r = k d_r, k = 0..n-1).  Between samples each is the cubic
 * Hermite interpolant whose node slopes are finite differences of the
 * samples: central (y[k+1] - y[k-1]) / 2h inside, the one-sided second-order
 * forms (-3 y0 + 4 y1 - y2) / 2h and (3 y[n-1] - 4 y[n-2] + y[n-3]) / 2h at
 * the ends (all exact for quadratics, so a quadratic is reproduced exactly).
 * Beyond the last sample (or below 0) a function continues as the straight
 * line through its end sample with its end slope.
 * ==================================================================== */
static double node_slope(const double* y, int n, double h, int k) {
  if (k == 0) return (-3.0 * y[0] + 4.0 * y[1] - y[2]) / (2.0 * h);
  if (k == n - 1) return (3.0 * y[n - 1] - 4.0 * y[n - 2] + y[n - 3]) / (2.0 * h);
  return (y[k + 1] - y[k - 1]) / (2.0 * h);
}

/* Value and derivative of the interpolant of y[0..n) (spacing h) at s. */
double or_eam_interp(const double* y, int n, double h, double s, double* dyds) {
  const double s_max = (n - 1) * h;
  if (s < 0.0 || s > s_max) {
    const int k = s < 0.0 ? 0 : n - 1;
    const double m = node_slope(y, n, h, k);
    if (dyds) *dyds = m;
    return y[k] + m * (s - k * h);
  }
  int k = (int)floor(s / h);
  if (k > n - 2) k = n - 2;
  const double u = s / h - k;
  const double m0 = node_slope(y, n, h, k), m1 = node_slope(y, n, h, k + 1);
  /* Hermite basis on [0, 1] and its derivative.  h00 = 1 - h01 and
   * d00 = -d01, so the two sample terms are grouped through the sample
   * difference (exact in floating point for neighbouring samples): summing
   * h00 y_k and h01 y_{k+1} separately would cancel to a few ulp of y, not of
   * the derivative. */
  const double h01 = -2 * u * u * u + 3 * u * u, h10 = u * u * u - 2 * u * u + u;
  const double h11 = u * u * u - u * u;
  const double d01 = -6 * u * u + 6 * u, d10 = 3 * u * u - 4 * u + 1, d11 = 3 * u * u - 2 * u;
  const double dy = y[k + 1] - y[k];
  if (dyds) *dyds = d01 * dy / h + d10 * m0 + d11 * m1;
  return y[k] + h01 * dy + h10 * h * m0 + h11 * h * m1;
}

/* EAM energy and forces on a given pair set, two passes.  Outputs as in
 * or_tbsma (NULL skips): rho, F, eB[i] = F(rho_i), eR[i] = 1/2 sum_j phi,
 * w[i] = 1/2 sum_j (x_j - x_i) F_ij,x, S[i] = sum_j |f_ij| with f_ij the
 * bracket's magnitude along (r_i - r_j)/r.  Returns E. */
double or_eam_on_pairs(const or_eam* T, int n, const double* x, const int* start, const int* nbr,
                       double* rho, double* F, double* eB, double* eR, double* w, double* S) {
  double* dF = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double E = 0.0;
  /* pass 1: densities and embedding energies */
  for (int i = 0; i < n; ++i) {
    double r_i = 0.0;
    for (int k = start[i]; k < start[i + 1]; ++k)
      r_i += or_eam_interp(T->f, T->n_r, T->d_r, sqrt(dist2(x, i, nbr[k])), NULL);
    const double e_b = or_eam_interp(T->F, T->n_rho, T->d_rho, r_i, &dF[i]);
    if (rho) rho[i] = r_i;
    if (eB) eB[i] = e_b;
    E += e_b;
  }
  /* pass 2: forces, pair energy, virial */
  for (int i = 0; i < n; ++i) {
    double fx = 0.0, fy = 0.0, fz = 0.0, e_r = 0.0, wi = 0.0, si = 0.0;
    for (int k = start[i]; k < start[i + 1]; ++k) {
      const int j = nbr[k];
      const double dx = x[3 * i + 0] - x[3 * j + 0];
      const double dy = x[3 * i + 1] - x[3 * j + 1];
      const double dz = x[3 * i + 2] - x[3 * j + 2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      double dphi, df;
      const double phi = or_eam_interp(T->phi, T->n_r, T->d_r, r, &dphi);
      or_eam_interp(T->f, T->n_r, T->d_r, r, &df);
      /* -dE/dr_ij, the pair's force along (r_i - r_j)/r */
      const double f = -(dphi + (dF[i] + dF[j]) * df);
      fx += f * dx / r;
      fy += f * dy / r;
      fz += f * dz / r;
      e_r += 0.5 * phi;
      wi += 0.5 * (-dx) * (f * dx / r);
      si += fabs(f);
    }
    if (F) {
      F[3 * i + 0] = fx;
      F[3 * i + 1] = fy;
      F[3 * i + 2] = fz;
    }
    if (eR) eR[i] = e_r;
    if (w) w[i] = wi;
    if (S) S[i] = si;
    E += e_r;
  }
  free(dF);
  return E;
}

/* Pair set (brute force if n <= brute_max, else cells) + EAM. */
double or_eam_energy_forces(const or_eam* T, int n, const double* x, int brute_max, double* F,
                            double* rho, double* eB, double* eR, double* w, double* S,
                            long* n_pairs_out) {
  long cap = 64L * n + 64;
  int* start = (int*)malloc(sizeof(int) * (n + 1));
  int* nbr = NULL;
  long k;
  for (;;) {
    nbr = (int*)malloc(sizeof(int) * cap);
    k = (n <= brute_max) ? or_pairs_brute(n, x, T->r_cut, start, nbr, cap)
                         : or_pairs_cells(n, x, T->r_cut, start, nbr, cap);
    if (k >= 0) break;
    free(nbr);
    cap *= 2;
  }
  double E = or_eam_on_pairs(T, n, x, start, nbr, rho, F, eB, eR, w, S);
  if (n_pairs_out) *n_pairs_out = k;
  free(start);
  free(nbr);
  return E;
}
