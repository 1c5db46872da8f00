/*
 * tbsma.h -- C ABI of the B300 (sm_103a) TB-SMA nanowire MD hot path.
 *
 * The library advances many independent fcc Au nanowires ("wires") at once:
 * a per-wire cell-list / Verlet neighbour-list build, the two-pass TB-SMA
 * force (density pass, then force pass), an FP64 velocity-Verlet step with a
 * Langevin thermostat and a rigid-grip pull, and per-wire FP64 observables.
 *
 * Method (French, Pervaje, Santos, Iacovella, Cummings, arXiv:1311.3890):
 *   Eq. 1   E_B^i = -sqrt(rho_i),  rho_i = sum_j xi^2 exp(-2q (r_ij/r0 - 1))
 *   Eq. 2   E_R^i = sum_j A exp(-p (r_ij/r0 - 1))
 *   Eq. 3   E_C   = sum_i (E_B^i + E_R^i), pairs with r_ij <= r_cut only
 *   Methods "TB-SMA potential": the force needs rho_i and rho_j, so it is
 *           computed in two passes over each atom's neighbours.
 *   Methods "Simulation details": velocity Verlet, dt = 2 fs, two rigid
 *           gripping layers per end pulled apart along [100].
 *   Eq. 4   strain = (L - L0)/L0;  Eq. 5  virial stress sigma_xx.
 *   Results "TB-SMA benchmarks": Verlet list with a buffer (skin) radius.
 *   Introduction: the two-stage force follows the EAM implementation the
 *           paper cites; tbsma_set_eam runs a tabulated EAM through the
 *           same two passes.
 *
 * Units: Angstrom, eV, amu, fs.  Strain rate in 1/s, temperature in K,
 * Langevin friction gamma in 1/fs.
 *
 * Layout conventions:
 *   - Positions x and velocities v are caller-owned DEVICE arrays of
 *     3*N doubles in SoA order: x[0..N) = x-coordinates, x[N..2N) = y,
 *     x[2N..3N) = z, N = total atoms of all wires.
 *   - Wire w owns atoms [atom_offset, atom_offset + n_atoms); wires are
 *     packed back to back in wire order (offset[0] = 0, offset[w+1] =
 *     offset[w] + n[w]).  The library never reorders atoms.
 *   - kind[i] (device uint8): 0 mobile, 1 left grip, 2 right grip.
 *
 * Ownership: the caller owns x, v, kind and the CUDA stream; the library
 * keeps the pointers and never frees them, so they must outlive the
 * context.  The library owns all other device memory (neighbour lists,
 * cell lists, packed positions, forces), allocated in tbsma_init and freed
 * in tbsma_destroy.
 *
 * Errors: every call returns a tbsma_status; nothing aborts, traps or
 * prints.  tbsma_last_error() returns a text for the last failure.  Calls
 * are enqueued on the context's stream and are asynchronous unless stated
 * otherwise.  Per-wire faults (non-finite coordinates, list or cell
 * overflow, fixed-point range) are recorded in a per-wire status word; the
 * calls that synchronise (tbsma_step_nvt_pull, tbsma_build_neighbors with a
 * counter, tbsma_reduce_observables, tbsma_force_check) return TBSMA_EWIRE
 * or TBSMA_EOVERFLOW when any wire is flagged.
 */
#ifndef TBSMA_H
#define TBSMA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tbsma_ctx tbsma_ctx; /* opaque, owned by the library */

typedef enum {
  TBSMA_OK = 0,
  TBSMA_EINVAL = 1,    /* bad argument (null pointer, size, layout) */
  TBSMA_ENOMEM = 2,    /* device allocation failed */
  TBSMA_ECUDA = 3,     /* a CUDA runtime call failed */
  TBSMA_EOVERFLOW = 4, /* neighbour-list or cell capacity exceeded */
  TBSMA_ETIMEOUT = 5,  /* a bounded device-side wait ran out */
  TBSMA_EWIRE = 6,     /* at least one wire has a non-zero status word */
  TBSMA_ESTATE = 7     /* call not valid in the context's current state */
} tbsma_status;

/* Arithmetic of the pair kernels.  FP64: every pair term in double.  MIXED:
 * pair geometry, exponentials, density and force accumulation in FP32 on
 * exact fixed-point coordinate differences; positions, velocities,
 * integration and all reductions stay FP64. */
typedef enum { TBSMA_FP64 = 0, TBSMA_MIXED = 1 } tbsma_precision;

/* Per-wire status bits. */
#define TBSMA_WIRE_NONFINITE 1u     /* NaN/Inf position or velocity */
#define TBSMA_WIRE_NBR_OVERFLOW 2u  /* an atom has more neighbours than the list holds, or a
                                       neighbour more than 32767 positions away in the atom order */
#define TBSMA_WIRE_CELL_OVERFLOW 4u /* a cell holds more atoms than its capacity */
#define TBSMA_WIRE_RANGE 8u         /* an atom is more than 1e7 A from its wire's centre */
#define TBSMA_WIRE_GRID_CLAMP 16u   /* not a fault: an atom lay outside its wire's cell grid at a
                                       list build (the list is still exact while no cell
                                       overflows); the next call that synchronises grows the
                                       grid and clears the bit */

/* TB-SMA parameters (Table 1; r_cut after Eq. 3), list skin and mass.
 * Au: A = 0.2061 eV, xi = 1.790 eV, p = 10.229, q = 4.036, r0 = 2.884 A
 * (the nearest-neighbour distance; Table 1 prints the lattice constant
 * 4.079 A in that column), r_cut = 5.8 A, r_skin = 0.29 A, mass = 196.966569.
 * r_skin changes only speed, never results: lists hold the pairs within
 * r_cut + r_skin and every pass tests r_cut itself.  The list row length
 * follows the list radius (1.25 x the fcc sites of a sphere of that radius
 * for nearest-neighbour distance r0, 64 to 128 entries:
 * tbsma_nbr_capacity); an atom with more neighbours sets
 * TBSMA_WIRE_NBR_OVERFLOW. */
typedef struct {
  double A, xi, p, q, r0, r_cut, r_skin, mass;
} tbsma_params;

/* One wire of the batch (host array passed to tbsma_init). */
typedef struct {
  int64_t atom_offset; /* first atom */
  int32_t n_atoms;     /* atoms in the wire (>= 1) */
  int32_t reserved;    /* must be 0 */
  double L0;           /* initial length, A (Eq. 4) */
  double strain_rate;  /* 1/s; each grip moves strain_rate*L0*dt/2 per step */
  double temperature;  /* K, Langevin target */
  double gamma;        /* 1/fs Langevin friction; 0 = NVE velocity Verlet */
  uint64_t seed;       /* Philox key of the wire's thermostat */
} tbsma_wire;

/* Per-wire observables (Eq. 3-5), FP64 reductions. */
typedef struct {
  int64_t step;       /* steps done since init */
  double strain;      /* Eq. 4 */
  double e_pot;       /* E_C of the wire, eV (Eq. 3; or the EAM energy) */
  double e_kin;       /* 1/2 m sum_mobile |v|^2, eV */
  double temp;        /* 2 E_kin / (3 N_mobile k_B), K */
  double sigma_xx;    /* Eq. 5, eV/A^3 (x 160.2177 for GPa) */
  double virial_xx;   /* sum_i 1/2 sum_j r_x,ij F_x,ij, eV */
  int32_t n_rebuilds; /* neighbour-list rebuilds of this wire during steps */
  int32_t status;     /* TBSMA_WIRE_* bits */
} tbsma_obs;

/* Mixed-precision vs FP64 force comparison of one wire (same positions, same list). */
typedef struct {
  double max_err_scaled; /* max_i |F_i^mixed - F_i^fp64| / S_i, S_i = sum_j |f_ij| */
  double max_err_raw;    /* max_i |F_i^mixed - F_i^fp64| / |F_i^fp64| */
  double norm_err;       /* ||F^mixed - F^fp64||_2 / ||F^fp64||_2 over the wire */
  double max_abs_err;    /* max_i |F_i^mixed - F_i^fp64|, eV/A */
} tbsma_fcheck;

/* Create a context for n_wires wires packed in x, v, kind (device, see
 * layout above) and enqueue on `cuda_stream` (a cudaStream_t; NULL = the
 * legacy default stream).  Allocates every device buffer, sizes a fixed
 * cell grid per wire from its initial bounding box (margins for strain up to
 * 1.0 along x; atoms outside are clamped into edge cells), builds all
 * neighbour lists and computes the initial forces.  Synchronises.
 * Errors: EINVAL (null pointers, n_wires < 1, wires not packed back to back,
 * bad parameters, non-finite positions, a wire centred 1e7 A or more from
 * the coordinate origin), ENOMEM, ECUDA: *out is NULL.  EWIRE / EOVERFLOW (a wire
 * was flagged by the initial build): *out is a valid context that the
 * caller inspects (tbsma_get_wire_status) and destroys. */
tbsma_status tbsma_init(const tbsma_params* params, tbsma_precision precision, int32_t n_wires,
                        const tbsma_wire* wires, double* x, double* v, const uint8_t* kind,
                        void* cuda_stream, tbsma_ctx** out);

/* Draw initial velocities (Methods: random Gaussian velocities per
 * trajectory): mobile atoms get Philox4x32-10 Gaussians at the wire's
 * temperature (key = seed, counter = (atom index in wire, 0, 0, 1)), the
 * mobile centre-of-mass velocity is removed and the velocities are scaled
 * to the exact target temperature; grip atoms get 0.  Writes v. */
tbsma_status tbsma_init_velocities(tbsma_ctx* ctx);

/* Re-read x (after the caller changed positions), then rebuild the lists of
 * the wires whose atoms moved more than r_skin/2 since their last build, or
 * of all wires if force_all != 0.  If n_rebuilt is non-NULL it receives the
 * number of wires rebuilt and the call synchronises. */
tbsma_status tbsma_build_neighbors(tbsma_ctx* ctx, int32_t force_all, int32_t* n_rebuilt);

/* Forces at the current positions (rebuilding lists first if needed), in
 * SoA 3*N device arrays.  f32_out (nullable) receives the MIXED-precision
 * forces, f64_out (nullable) the FP64 forces, both on the same list; either
 * precision can be asked of any context.  The context's own force buffer
 * (used by the next step) is refreshed in the context's precision.  After
 * tbsma_set_eam every pass (here and in the other calls) uses the EAM. */
tbsma_status tbsma_compute_forces(tbsma_ctx* ctx, float* f32_out, double* f64_out);

/* Per-atom energies E_B^i + E_R^i (Eq. 1-2; EAM: F(rho_i) + 1/2 sum_j phi) and axial pair virials
 * 1/2 sum_j r_x,ij F_x,ij at the current positions, context precision,
 * into device arrays of N doubles (either nullable). */
tbsma_status tbsma_atom_energies(tbsma_ctx* ctx, double* e_out, double* w_out);

/* Advance every wire by n_steps steps of dt_fs: B A O A (mobile atoms; grips
 * shifted rigidly), displacement check, list rebuild of flagged wires,
 * density pass, force pass, B (under the Nosé–Hoover protocol: NH B A,
 * ..., B NH; see tbsma_set_protocol).  Replays a captured CUDA graph; the first
 * call with a new dt captures it.  Synchronises at the end to read the
 * wires' status words (and, in a call of more than 1000 steps, every 1000
 * steps).
 * Cell grids grow: each wire's cell grid is planned at init with room for
 * the wire to double its length; an atom outside it at a list build is
 * binned into an edge cell and marks the wire (TBSMA_WIRE_GRID_CLAMP), and
 * at the next status read the library re-plans that wire's grid around
 * its current extent (again with room to double), growing its cell
 * storage if needed, and rebuilds its list.  Forces are unaffected unless
 * an edge cell overflowed before that (TBSMA_WIRE_CELL_OVERFLOW): then the
 * grid is grown all the same, the forces are recomputed, the bit is
 * cleared, and the call returns EOVERFLOW at once (the steps since that
 * wire's previous list build used a list that missed atoms; repeat them
 * from saved state: the retry runs on the grown grid).
 * Errors: EINVAL (n_steps < 0, dt_fs <= 0), EWIRE, EOVERFLOW, ECUDA. */
tbsma_status tbsma_step_nvt_pull(tbsma_ctx* ctx, int64_t n_steps, double dt_fs);

/* Paper protocol mode (Methods, "Simulation details": Nosé–Hoover
 * thermostat with velocity Verlet, dt = 2 fs; grips displaced by 0.05 A
 * every 20 ps; temperature ramped from 0.01 K to the target).  Applies to
 * every wire of the context from the next tbsma_step_nvt_pull on.
 *   thermostat  TBSMA_THERMO_LANGEVIN (default; the wire's gamma, B A O A B)
 *               or TBSMA_THERMO_NOSE_HOOVER: one thermostat per wire, g =
 *               3 N_mobile degrees of freedom, mass Q = g k_B T_w tau^2 (T_w
 *               the wire's temperature, tau = tau_fs), the step
 *               NH(dt/2) B(dt/2) A(dt) [forces] B(dt/2) NH(dt/2) with
 *               NH(h): xi += (h/2)(2K - g k_B T)/Q; v *= exp(-xi h);
 *               eta += h xi; xi += (h/2)(2K' - g k_B T)/Q.  A wire with
 *               T_w = 0 or no mobile atom runs NVE.
 *   pull        TBSMA_PULL_CONTINUOUS (default; each grip moves by
 *               strain_rate L0 dt / 2 per step) or TBSMA_PULL_STEPWISE:
 *               in step s (0-based, counted from tbsma_init) each grip
 *               moves by -/+ pull_step when (s + 1) is a multiple of
 *               pull_interval, else not at all.
 *   ramp        the thermostat's target at step s is t_start + (T_w -
 *               t_start) clamp((s - ramp_start) / ramp_steps, 0, 1): t_start
 *               until step ramp_start (counted from tbsma_init), then the
 *               linear ramp; ramp_steps = 0: T_w throughout.  The paper's
 *               equilibration (100 ps of barostat at 0.01 K, 400 ps of ramp,
 *               400 ps at T_w) is ramp_start 50000, ramp_steps 200000.
 *   barostat    (baro_tau_fs > 0; Methods: 100 ps at zero pressure along
 *               [100] with a Nosé–Hoover barostat before the pull) Hoover's
 *               constant-stress equations along x about the mean x, c, of
 *               the wire's grip atoms: dx/dt = v_x + zeta (x - c) (every
 *               atom), dv_x/dt = F_x/m - zeta v_x (mobile atoms), dzeta/dt =
 *               -(sigma_xx - P)/(B tau_b^2) - gamma_b zeta, dlambda/dt =
 *               zeta, with sigma_xx the wire's axial stress (Eq. 5, as
 *               tbsma_reduce_observables), P = baro_pressure, B =
 *               baro_modulus, tau_b = baro_tau_fs (barostat mass V B
 *               tau_b^2: a wire of axial modulus B oscillates with angular
 *               frequency 1/tau_b) and drag gamma_b = baro_drag / tau_b.
 *               Without drag and thermostat E_pot + K + V B tau_b^2 zeta^2/2
 *               - P V lambda is conserved.  Step (h = dt/2): Z C [NH] B S
 *               A S [forces] B [NH] C Z, with Z the drag and stress kick of
 *               zeta (kick first at the step's end), C: v_x *= exp(-zeta h),
 *               S: x = c + (x - c) exp(zeta h), lambda += zeta h; c is
 *               taken at the step's start.  The default sequence's merged
 *               kicks are not used and every force pass also forms the
 *               per-atom virial; the grips keep their pull (d_grip is not
 *               changed by the scaling).
 * The paper's values: Nosé–Hoover (tau is not given; 1000 fs is this
 * library's reading), pull_step 0.05 A, pull_interval 10000, t_start
 * 0.01 K, ramp_steps 200000 (400 ps).  Resets every wire's thermostat
 * state (xi = eta = 0; lambda is kept) and drops captured graphs.  Errors:
 * EINVAL (unknown thermostat or pull, tau_fs <= 0 under Nosé–Hoover,
 * pull_interval < 1 or non-finite pull_step under stepwise pull, t_start < 0,
 * ramp_steps < 0 or ramp_start < 0, baro_tau_fs < 0 or non-finite, and with
 * the barostat on baro_modulus <= 0, baro_drag < 0, or any of them or
 * baro_pressure non-finite). */
typedef enum { TBSMA_THERMO_LANGEVIN = 0, TBSMA_THERMO_NOSE_HOOVER = 1 } tbsma_thermostat;
typedef enum { TBSMA_PULL_CONTINUOUS = 0, TBSMA_PULL_STEPWISE = 1 } tbsma_pull;
typedef struct {
  int32_t thermostat;    /* tbsma_thermostat */
  int32_t pull;          /* tbsma_pull */
  double tau_fs;         /* Nosé–Hoover period, fs */
  double pull_step;      /* stepwise: displacement of each grip per event, A */
  int64_t pull_interval; /* stepwise: steps per event */
  double t_start;        /* ramp start temperature, K */
  int64_t ramp_steps;    /* ramp length in steps, 0 = no ramp */
  double baro_tau_fs;    /* axial barostat time, fs; 0 = no barostat */
  double baro_modulus;   /* its reference modulus, eV/A^3 */
  double baro_pressure;  /* its target sigma_xx (tension positive), eV/A^3 */
  double baro_drag;      /* its drag gamma_b in units of 1/baro_tau_fs */
  int64_t ramp_start;    /* first step of the ramp (target t_start before it) */
} tbsma_protocol;

tbsma_status tbsma_set_protocol(tbsma_ctx* ctx, const tbsma_protocol* protocol);

/* Each wire's Nosé–Hoover state into host arrays of n_wires doubles (either
 * nullable): xi (1/fs) and its time integral eta, so that the extended
 * energy E_pot + E_kin + Q xi^2/2 + g k_B T eta can be formed.  Zeros under
 * the Langevin thermostat.  Synchronises. */
tbsma_status tbsma_get_thermostat(tbsma_ctx* ctx, double* xi, double* eta);

/* Each wire's barostat state into host arrays of n_wires doubles (either
 * nullable): the axial log-stretch lambda (the integral of zeta since
 * tbsma_init or tbsma_restore_state: a wire of length L then has length
 * L e^lambda, less its grips' pull) and the strain rate zeta (1/fs).  Kept
 * across tbsma_set_protocol.  Synchronises. */
tbsma_status tbsma_get_barostat(tbsma_ctx* ctx, double* lambda, double* zeta);

/* Wire topology: rupture and neck (Results, "Nanowire elongation"; the paper
 * gives no formal definition).  Clusters are the connected components of
 * the graph of interacting pairs (r_ij <= r_cut under the context's
 * precision rule: the FP32 rule on fixed-point positions for MIXED, FP64
 * distances for FP64), each labelled by its smallest atom index.  A wire is
 * connected while a left-grip and a right-grip atom share a cluster (the
 * failure strain is the strain of the first report at which it is not).
 * Neck: with x_lo the largest x of the left grip and x_hi the smallest x of
 * the right grip, slab k = 0 .. n_slabs - 1 covers x_lo + (k + 1/2) w <= x <
 * x_lo + (k + 3/2) w, n_slabs = floor((x_hi - x_lo)/w - 1/2), w = a/2 =
 * 2.0395 A (the (100) plane spacing), so each plane of the unstrained wire
 * sits at a slab centre; neck = the fewest atoms in a slab, neck_slab its
 * index (first on ties; without slabs neck = 0 and neck_slab = -1).  status: 0, 1 if the wire has
 * more than 4096 slabs (neck not computed), 2 if a bounded union-find loop
 * gave up.  Re-packs positions and rebuilds the lists of wires that moved
 * past the skin first.  out[n_wires] host; labels (nullable) device, N int32.
 * Synchronises.  Errors: EINVAL (null out), ETIMEOUT (a status 2), ECUDA. */
typedef struct {
  int32_t connected;  /* 1: the grips are in one cluster */
  int32_t n_clusters; /* components of the interacting-pair graph */
  int32_t neck;       /* fewest atoms in an axial slab between the grips */
  int32_t neck_slab;  /* its index, -1 without slabs */
  int32_t n_slabs;
  int32_t status;
} tbsma_topology;

tbsma_status tbsma_wire_topology(tbsma_ctx* ctx, tbsma_topology* out, int32_t* labels);

/* Test hook for failure detection: the bound of every union-find walk of
 * tbsma_wire_topology (default 1048576 steps), and of every wait of the
 * persistent step kernel at a grid barrier (4 (steps - 1) polls; 1 makes
 * every block that is not the last to arrive give up at once).  A bound too
 * small for the graph makes tbsma_wire_topology give up: status 2 and
 * TBSMA_ETIMEOUT; a barrier wait that gives up ends the step kernel in every
 * block and tbsma_step_nvt_pull returns TBSMA_ETIMEOUT (the wires' state
 * is then part-way through a step: restore it before going on).  The
 * context stays usable.  Errors: EINVAL (steps < 1). */
tbsma_status tbsma_set_wait_limit(tbsma_ctx* ctx, int32_t steps);

/* How tbsma_step_nvt_pull runs the steps.
 *   TBSMA_STEPS_AUTO        the persistent step kernel when the context can
 *                           run it, else graph replays (default);
 *   TBSMA_STEPS_GRAPH       always replays of captured step graphs;
 *   TBSMA_STEPS_PERSISTENT  the persistent step kernel (tbsma_step_nvt_pull
 *                           returns EINVAL if the context cannot run it).
 * The persistent step kernel runs a call's steps (up to 1000 per launch) in
 * one cooperative launch, one block per 256-atom tile, its blocks meeting at
 * bounded grid-wide barriers between the phases of a step (two per step
 * without a rebuild: the force pass also integrates each atom's next step):
 * the same kernels' code per atom and per tile, so bitwise the same
 * trajectories as the graph replays, without a launch per phase.  It serves small contexts:
 * the default protocol (Langevin, continuous pull), 256-atom tiles
 * (tbsma_set_launch), and every tile of the batch resident on the GPU at
 * once; MIXED and FP64 contexts alike (FP64: 128-thread blocks, the FP64
 * passes 16 lanes per slot over the grid, three barriers per step).
 * blocks (host, nullable) receives the blocks it would use in this context
 * (0: it cannot run it).  Errors: EINVAL (unknown mode). */
/* Threads per atom in the MIXED pair passes, graph replays and the
 * persistent step kernel alike: 1 (default; one thread walks the atom's
 * list), 2 or 4 (each thread evaluating every second or fourth entry of
 * every group of four, the terms added in list order through shuffles:
 * bitwise the same forces and energies; a tile then holds 128 or 64
 * atoms).  Invalidates captured graphs.  Errors: EINVAL (other values). */
tbsma_status tbsma_set_pair_lanes(tbsma_ctx* ctx, int32_t lanes);

#define TBSMA_STEPS_AUTO 0
#define TBSMA_STEPS_GRAPH 1
#define TBSMA_STEPS_PERSISTENT 2
tbsma_status tbsma_set_step_mode(tbsma_ctx* ctx, int32_t mode, int32_t* blocks);

/* Tabulated embedded-atom method (EAM), the general form of the two-stage
 * many-body force the paper builds TB-SMA on (Introduction; Methods,
 * "TB-SMA potential": the force is computed in two kernels, each looping
 * over atom i's neighbours, as in the EAM implementation it cites):
 *   rho_i = sum_j f(r_ij),   E = sum_i [F(rho_i) + 1/2 sum_j phi(r_ij)],
 *   F_i = -sum_j [phi'(r_ij) + (F'(rho_i) + F'(rho_j)) f'(r_ij)] (r_i - r_j)/r_ij,
 * over pairs j != i with r_ij <= params.r_cut.  TB-SMA (Eq. 1-3) is the case
 * f = xi^2 e^{-2q s}, phi = 2 A e^{-p s}, F = -sqrt(rho).
 *
 * The functions are given as samples on uniform grids: F[k] = F(k d_rho)
 * for k < n_rho, f[k] = f(k d_r) and phi[k] = phi(k d_r) for k < n_r (host
 * arrays of doubles, read during the call only).  Between samples each is
 * the cubic Hermite interpolant whose node slopes are the finite
 * differences (y[k+1] - y[k-1]) / 2h inside and (-3 y0 + 4 y1 - y2) / 2h,
 * (3 y[n-1] - 4 y[n-2] + y[n-3]) / 2h at the two ends; F continues past
 * either end of its grid as the tangent line at the end sample. */
typedef struct {
  const double* F;   /* n_rho samples of the embedding energy F(rho), eV */
  int32_t n_rho;
  double d_rho;      /* rho grid spacing (rho in the units of f) */
  const double* f;   /* n_r samples of the density function f(r) */
  const double* phi; /* n_r samples of the pair energy phi(r), eV */
  int32_t n_r;
  double d_r;        /* r grid spacing, A */
} tbsma_eam;

/* Switch the context's potential to the tabulated EAM (tables != NULL) or
 * back to TB-SMA with the context's parameters (tables == NULL).  The
 * tables are copied to library-owned device memory (any earlier EAM tables
 * are freed, after the context's stream has drained).  The neighbour lists,
 * r_cut and r_skin are unchanged; the forces of the current positions are
 * recomputed (enqueued), so the next step starts from the new potential.
 * Both precisions use the tables: MIXED in FP32 (coefficients rounded once
 * from the FP64 ones), FP64 in FP64; energies (tbsma_atom_energies,
 * tbsma_reduce_observables) are FP64 sums.  A checkpoint holds no tables:
 * set the same tables before tbsma_restore_state.  Errors: EINVAL (null
 * arrays, n_rho or n_r < 3 or > 2^22, spacings not positive and finite, a
 * non-finite sample, (n_r - 1) d_r < r_cut: nothing changed), ENOMEM or
 * ECUDA (the earlier tables are gone: the context is left on TB-SMA). */
tbsma_status tbsma_set_eam(tbsma_ctx* ctx, const tbsma_eam* tables);

/* The interpolant tbsma_set_eam builds from one sample table, as cubic
 * coefficients per interval (host only: no context, no GPU): for interval
 * k = 0 .. n-2, with t = s/h - k, y(t) = c[4k] + t (c[4k+1] + t (c[4k+2] +
 * t c[4k+3])) in units of y per grid step (divide derivatives in t by h).
 * samples: n doubles (host); coeffs: 4 (n - 1) doubles (host, caller-owned).
 * Errors: EINVAL (null pointers, n < 3 or > 2^22). */
tbsma_status tbsma_eam_cubics(const double* samples, int32_t n, double* coeffs);

/* Checkpoint / resume.  A wire's counters: grip displacement (A), the
 * Nosé–Hoover state, the barostat's log-stretch and strain rate, the number
 * of list rebuilds and its status word. */
typedef struct {
  double d_grip;
  double xi, eta;
  double log_stretch, stretch_rate; /* barostat lambda and zeta */
  int32_t n_rebuilds;
  uint32_t status;
} tbsma_wire_state;

/* Save: rebuild every wire's list from the current positions and recompute
 * the forces (so that the state is a function of what is saved), then copy
 * x, v (host, 3*N doubles SoA each), the wires' counters (host, n_wires) and
 * the step count.  Restore into a context made by tbsma_init on the same
 * batch layout and parameters (and the same tbsma_set_protocol, which must
 * come first): the continuation of the restored context equals the
 * continuation of the saved one bit for bit.  Both synchronise.  Errors:
 * EINVAL (null pointers, step < 0), ESTATE (the counts disagree), ECUDA. */
tbsma_status tbsma_save_state(tbsma_ctx* ctx, double* x_host, double* v_host,
                              tbsma_wire_state* wires, int64_t* step);
tbsma_status tbsma_restore_state(tbsma_ctx* ctx, const double* x_host, const double* v_host,
                                 const tbsma_wire_state* wires, int64_t step);

/* Per-wire observables at the current state into out[n_wires] (host).
 * Synchronises.  Returns EWIRE if any wire's status is non-zero (out is
 * still filled). */
tbsma_status tbsma_reduce_observables(tbsma_ctx* ctx, tbsma_obs* out);

/* n_steps steps as tbsma_step_nvt_pull, then the observables of the final
 * state as tbsma_reduce_observables (Eq. 3-5): bitwise the same trajectory
 * and the same out[n_wires] (host) as the two calls.  In graph replays
 * under the default protocol the last step's pair passes also form the
 * per-atom energy and virial terms (their forces are the same), so the
 * report does not run the passes again (a whole last graph chunk replays a
 * second captured graph, kept until the graphs are dropped); the
 * persistent step kernel and the protocol mode make the two calls.
 * Synchronises.  Errors: as tbsma_step_nvt_pull, and EINVAL for a null out;
 * EWIRE as tbsma_reduce_observables (out is still filled). */
tbsma_status tbsma_step_observe(tbsma_ctx* ctx, int64_t n_steps, double dt_fs, tbsma_obs* out);

/* Compare MIXED and FP64 forces at the current positions on the same list,
 * per wire, into out[n_wires] (host).  Whether a pair is inside r_cut is
 * decided once, by the MIXED path's FP32 rule, for both arms (a pair within
 * ~1e-6 A of r_cut may fall either way in different precisions; both are
 * valid), so the comparison measures the pair arithmetic alone.  The
 * context's own force buffer is left in the context's precision.
 * Synchronises. */
tbsma_status tbsma_force_check(tbsma_ctx* ctx, tbsma_fcheck* out);

/* Copy the state from / to host buffers of 3*N doubles (SoA, as x and v).
 * Either pointer may be NULL to skip it.  Upload re-packs positions,
 * rebuilds the lists of wires that moved past the skin and recomputes the
 * forces; download synchronises.  Pinned host memory makes the copies
 * asynchronous DMA. */
tbsma_status tbsma_upload_state(tbsma_ctx* ctx, const double* x_host, const double* v_host);
tbsma_status tbsma_download_state(tbsma_ctx* ctx, double* x_host, double* v_host);

/* Per-wire status words (TBSMA_WIRE_* bits) into status_host[n_wires].
 * Synchronises. */
tbsma_status tbsma_get_wire_status(tbsma_ctx* ctx, int32_t* status_host);

/* Neighbour lists (device): n_nbr[N] and nbr[N * cap] (row i holds atom i's
 * neighbours within r_cut + r_skin, in the library's deterministic order;
 * unused entries -1).  cap must equal tbsma_nbr_capacity(ctx). */
int32_t tbsma_nbr_capacity(const tbsma_ctx* ctx);

/* Launch accounting: how many times the kernels of the list-rebuild chain
 * (cell clear, bin, sort, cell build, and in MIXED contexts the two envelope
 * passes and the slab build) were launched since tbsma_init: once
 * per step and per position refresh (they return at once when no wire is
 * flagged).  Synchronises.  Errors: EINVAL (null). */
tbsma_status tbsma_get_rebuild_chains(tbsma_ctx* ctx, int64_t* n);

/* List-build accounting since tbsma_init (host out[3]): out[0] launches of
 * the rebuild chain (as tbsma_get_rebuild_chains), out[1] wires whose lists
 * were built, out[2] atoms whose lists were built (both summed over every
 * build: step loop, refreshes, init).  The difference of two reads gives
 * the rebuilds inside a stretch of steps (Results, "TB-SMA benchmarks": the
 * list rebuild rate is what separates the 10 K and 298 K timings).
 * Synchronises.  Errors: EINVAL (null). */
tbsma_status tbsma_get_rebuild_stats(tbsma_ctx* ctx, int64_t* out);
tbsma_status tbsma_get_neighbors(tbsma_ctx* ctx, int32_t* n_nbr, int32_t* nbr, int32_t cap);

/* Launch shape of the pair passes: threads per block (64, 128 or 256; one
 * atom per thread, a block is a tile of consecutive atoms of one wire) and the tile's
 * shared-memory window in atoms (0..4096, 0 = read neighbours from global
 * memory): a tile whose neighbours span at most that many consecutive atoms
 * stages their packed positions in shared memory.  Invalidates captured
 * graphs.  Defaults: 256, 1280 (the window of a 256-atom tile of a 4 nm wire;
 * 8 blocks of 256 threads still fit an SM). */
tbsma_status tbsma_set_launch(tbsma_ctx* ctx, int32_t block_threads, int32_t window_atoms);

/* Enqueue `reps` launches of one pair pass on the context's stream, on the
 * current packed positions and lists, in the context's precision and launch
 * shape: pass 1 = density (Eq. 1), pass 2 = force.  Both are idempotent, so a
 * caller can bracket this call with CUDA events on the same stream to time a
 * pass alone.  Errors: EINVAL (pass not 1 or 2, reps < 1). */
tbsma_status tbsma_run_pass(tbsma_ctx* ctx, int32_t pass, int32_t reps);

/* Phases of one MD step, as tbsma_step_profile splits its time. */
#define TBSMA_PHASE_INTEGRATE 0 /* thermostat half steps + B A O A + pack + displacement check */
#define TBSMA_PHASE_PLAN 1      /* flagged wires -> rebuild work list, step counter */
#define TBSMA_PHASE_REBUILD 2   /* cell clear, bin, sort, list build of the flagged wires */
#define TBSMA_PHASE_DENSITY 3   /* pass 1 (Eq. 1) */
#define TBSMA_PHASE_FORCE 4     /* pass 2 (Eq. 2-3 derivative) */
#define TBSMA_PHASE_KICK 5      /* closing half kick (+ thermostat end half step) */
#define TBSMA_N_PHASES 6

/* The same steps as tbsma_step_nvt_pull (identical kernels, order and
 * results), enqueued directly instead of through the graph, with a CUDA
 * event after every phase; phase_ms (host, TBSMA_N_PHASES doubles) receives
 * the summed milliseconds of each phase over the n_steps steps.  For
 * measurement: the events between phases serialise nothing that the graph
 * overlaps (the step is one stream), but each launch pays its own launch
 * latency.  Synchronises.  Errors: EINVAL (n_steps outside [1, 2^20],
 * dt_fs <= 0, a barostat protocol), and those of tbsma_step_nvt_pull. */
tbsma_status tbsma_step_profile(tbsma_ctx* ctx, int64_t n_steps, double dt_fs, double* phase_ms);

/* Philox4x32-10 (Salmon et al., SC'11) on the device, as the thermostat
 * uses it: out[4i..4i+4) = philox(ctr[4i..4i+4), key[2i..2i+2)).  Device
 * arrays; enqueued on cuda_stream. */
tbsma_status tbsma_philox4x32_10(const uint32_t* ctr, const uint32_t* key, int64_t n,
                                 uint32_t* out, void* cuda_stream);

/* The thermostat's Gaussian triples on the device: for each atoms[i],
 * out[3i..3i+3) = Box-Muller normals of philox(counter = (atoms[i], step lo,
 * step hi, tag), key = (seed lo, seed hi)); precision selects the
 * FP64 or FP32 Box-Muller used by that path. */
tbsma_status tbsma_normals(uint64_t seed, const uint32_t* atoms, int64_t n, int64_t step,
                           uint32_t tag, tbsma_precision precision, double* out,
                           void* cuda_stream);

/* Allocation-free forces.  The paper has no counterpart to this call; it
 * exists for callers that may not allocate device memory when they need
 * forces: a host program that gives its plug-ins a fixed, pre-reserved slice
 * of the GPU's memory, or code inside a latency-critical loop where a
 * cudaMalloc would stall the whole device.  It needs no context and no
 * device allocation (no cudaMalloc or cudaFree, no allocating library call).
 *
 * FP64 TB-SMA forces (Eq. 1-3, two passes, hard cutoff) of ONE cluster of
 * n_atoms <= TBSMA_NOALLOC_MAX_ATOMS atoms; every pair is tested (no list),
 * so the cost grows as n_atoms^2.  x: device, 3*n_atoms doubles, SoA as
 * everywhere in this header; f_out: device, 3*n_atoms doubles, written.
 * The per-atom density scratch lives in one file-scope device array of
 * TBSMA_NOALLOC_MAX_ATOMS doubles (128 KiB) that every GPU loading this
 * library holds until the process exits.
 *   - Every call looks that array's device address up with the caller's
 *     device current (a CUDA runtime query, no allocation, no host-side
 *     cache: the address is right for whichever device and context is
 *     current, and concurrent calls from several host threads share no
 *     host state).  The first lookup on a device may load the library's
 *     module there, so make the first call on each device before any
 *     stream capture.
 *   - All calls share the array: two calls whose kernels overlap on the GPU
 *     (e.g. issued on different streams) race and give wrong forces.
 *     Calls on one stream are ordered and safe.  Each call rewrites every
 *     slot it reads, so nothing carries over between calls.
 * Errors: EOVERFLOW if n_atoms > TBSMA_NOALLOC_MAX_ATOMS (nothing launched),
 * EINVAL for null pointers, n_atoms < 0 or bad parameters, ECUDA if the
 * lookup or one of this call's two launches fails.  A launch error left
 * pending by an earlier, unrelated CUDA call also gives ECUDA: it is left
 * pending for its owner (not cleared) and nothing is launched.  n_atoms == 0
 * is a no-op.  Asynchronous on cuda_stream. */
#define TBSMA_NOALLOC_MAX_ATOMS 16384
tbsma_status tbsma_forces_noalloc(const tbsma_params* params, int32_t n_atoms, const double* x,
                                  double* f_out, void* cuda_stream);

const char* tbsma_last_error(const tbsma_ctx* ctx);
void tbsma_destroy(tbsma_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* TBSMA_H */
