/*
 * gcme.h -- C ABI of libgcme, a CUDA (sm_103a) library for the per-step
 * nonbonded force and energy of GCMe, the Gaussian core model with smeared
 * electrostatics (Ye, Chen & Wang, arXiv 2403.08148).
 *
 * Model (reduced units: kT = 1, length d, charge e, Coulomb prefactor lB):
 *   Gaussian core (Eq. u_ex):
 *     u_ex(r) = A (3 / (2 pi s))^{3/2} exp(-3 r^2 / (2 s)),  s = sigma_i^2 + sigma_j^2
 *   smeared Coulomb (Eq. u_elec):
 *     u_elec(r) = lB z_i z_j erf(beta r) / r,  beta = sqrt(pi) / (sqrt(2) a_ij)
 *   Ewald split of the electrostatics (Eq. ewald):
 *     real  = sum_{pairs, r < rc} lB z_i z_j [erfc(kappa r) - erfc(beta r)] / r
 *     recip = smooth PME (Essmann et al. 1995) of the point-charge sum
 *     corr  = -lB kappa / sqrt(pi) sum z_i^2,   self = lB sum z_i^2 / (2 a)
 *   Boundaries (Method of image charges section; Illustrative example):
 *     BULK          periodic box
 *     SLAB_NONMETAL real beads in 0 < z < H, box Lz = 3 H, Yeh-Berkowitz term
 *                   2 pi lB M_z^2 / V and electrode walls at z = 0, H
 *     SLAB_IMAGE    real beads in 0 < z < H, box Lz = 2 H; every charged bead
 *                   has a mirror image (x, y, -z) with charge -z_i; reported
 *                   electrostatic energies are those of the physical system
 *                   (half of the doubled one), walls at z = 0, H
 *   Harmonic bonds (Illustrative example): u = k/2 (r - r0)^2.
 *
 * Conventions for every entry point:
 *   - return 0 on success or a negative GCME_ERR_* code; nothing throws,
 *     exits or traps; gcme_last_error() gives a message for the calling
 *     thread's last failure;
 *   - pointers named d_* are device pointers owned by the caller (the
 *     library never frees them); pointers named h_* are host pointers read
 *     during the call only;
 *   - positions are (n, 3) row-major FP64; velocities (n, 3) row-major FP32;
 *     forces are 64-bit fixed point, value = F * 2^32, in structure-of-arrays
 *     layout: fx[0..n), fy[n..2n), fz[2n..3n);
 *   - energies are FP64 arrays of GCME_NTERMS entries (index GCME_E_*);
 *     the virial is 9 FP64 values, W_ab = sum_pairs r_ij,a F_ij,b of the
 *     pair, reciprocal and bond terms; it is the virial of the physical
 *     forces in the bulk geometry only (the pressure's); the slab geometries
 *     return these sums without the wall and Yeh-Berkowitz terms (the
 *     image-charge geometry's reciprocal part halved like its energy), which
 *     is not a pressure there;
 *   - work is enqueued on the caller's CUDA stream (NULL = legacy default
 *     stream) and ordered with the caller's other work on that stream.
 */
#ifndef GCME_H
#define GCME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gcme_ctx gcme_ctx;
typedef struct gcme_sys gcme_sys;
typedef struct gcme_batch gcme_batch;
typedef struct gcme_server gcme_server;
typedef void *gcme_stream_t; /* a cudaStream_t */

enum {
  GCME_OK = 0,
  GCME_ERR_INVALID = -1,   /* bad argument, rejected before any GPU work */
  GCME_ERR_OOM = -2,       /* device allocation failed or budget exceeded */
  GCME_ERR_CUDA = -3,      /* a CUDA runtime call failed */
  GCME_ERR_TIMEOUT = -4,   /* a bounded device-side wait ran out */
  GCME_ERR_NONFINITE = -5, /* a force or energy became NaN/Inf */
  GCME_ERR_FULL = -6,      /* server queue full */
  GCME_ERR_NOTFOUND = -7   /* unknown ticket */
};

enum { GCME_BULK = 0, GCME_SLAB_NONMETAL = 1, GCME_SLAB_IMAGE = 2 };

enum { GCME_FP32 = 0, GCME_FP64 = 1 };

/* Energy terms (FP64, kT). */
enum {
  GCME_E_GC = 0,      /* Gaussian core, Eq. u_ex                        */
  GCME_E_REAL = 1,    /* real-space electrostatics, Eq. ewald line 3    */
  GCME_E_RECIP = 2,   /* reciprocal (PME), Eq. ewald line 5             */
  GCME_E_CORR = 3,    /* -lB kappa/sqrt(pi) sum z^2, Eq. ewald line 6   */
  GCME_E_SELF = 4,    /* Born self energy, Eq. ewald line 7             */
  GCME_E_SLAB = 5,    /* Yeh-Berkowitz slab term                        */
  GCME_E_WALL = 6,    /* electrode wall term                            */
  GCME_E_BOND = 7,    /* harmonic bonds                                 */
  GCME_E_POTENTIAL = 8, /* sum of the above                             */
  GCME_E_KINETIC = 9,   /* 1/2 sum v^2 (unit masses), set by gcme_step  */
  GCME_NTERMS = 10
};

#define GCME_FORCE_SCALE 4294967296.0 /* 2^32: fixed-point force scale */
#define GCME_MAX_TYPES 8               /* species per system */

/* Parameters of one system.  All lengths in d, energies in kT. */
typedef struct gcme_params {
  double box[3];      /* periodic box (for slabs: the doubled/tripled box) */
  int32_t geometry;   /* GCME_BULK / GCME_SLAB_NONMETAL / GCME_SLAB_IMAGE  */
  int32_t precision;  /* GCME_FP32 (default) or GCME_FP64 (plain path)     */
  double A;           /* Gaussian-core amplitude A_ij, uniform               */
  double sigma;       /* mass smearing radius sigma_i, uniform               */
  double a;           /* charge smearing radius a_i, uniform                 */
  double lB;          /* Bjerrum length                                      */
  double rc;          /* real-space cutoff                                   */
  double kappa;       /* Ewald splitting parameter, kappa = 1/(sqrt(2) G)    */
  int32_t K[3];       /* PME grid, each 2^a 3^b 5^c, 4 <= K <= 1024          */
  int32_t order;      /* B-spline order p, 3..8                              */
  double dt;          /* velocity-Verlet time step                           */
  double H;           /* slab height (slab geometries)                       */
  double wall_A;      /* wall amplitude A n_s (slab geometries; 0 = none)    */
  double wall_sigma2; /* wall width sigma_w^2                                */
  double bond_k;      /* harmonic bond constant                              */
  double bond_r0;     /* harmonic bond rest length                           */
  int32_t cell_factor; /* cells of side >= rc / cell_factor: 1 (27-cell
                          stencil) or 2 (blocks of 2^3 cells with culling);
                          0 lets the library choose                        */
  int32_t pair_path;   /* GCME_PAIR_AUTO (0), GCME_PAIR_LIST or GCME_PAIR_CELLS */
  double gamma;        /* Langevin friction (1/tau); 0 = velocity Verlet (NVE) */
  double kT;           /* Langevin temperature (kT units; 1 = the reduced unit) */
  uint64_t seed;       /* Langevin noise key                                    */
  /* Several species (0 = one species with A, sigma, a above).  Species t of
   * ntypes <= GCME_MAX_TYPES has sigma_tab[t] and a_tab[t]; species t and u
   * interact with A_tab[t * GCME_MAX_TYPES + u] (symmetric).  Beads get
   * their species from h_types at creation. */
  int32_t ntypes;
  int32_t frozen_mask; /* bit t set: beads of species t never move (electrodes) */
  double A_tab[GCME_MAX_TYPES * GCME_MAX_TYPES];
  double sigma_tab[GCME_MAX_TYPES];
  double a_tab[GCME_MAX_TYPES];
} gcme_params;

/* Several species (Supporting Information, Flory-Huggins section: A/B
 * monomers with A_AB = A_AA + Delta A; species may also differ in sigma_i
 * and a_i).  Per pair of species: s = sigma_i^2 + sigma_j^2 in Eq. u_ex,
 * a_ij^2 = a_i^2 + a_j^2 and beta_ij = sqrt(pi) / (sqrt(2) a_ij) in the
 * real-space term of Eq. ewald, the Born self energy lB z_i^2 / (2 a_i) per
 * bead; image beads keep their source's species (a_i, no Gaussian core).
 * Supported by the 27-cell FP32 kernel (graph and persistent launches) and
 * the FP64 kernel; the fine-cell and neighbour-list paths reject it.
 *
 * Frozen species (frozen_mask): explicit electrodes as in the performance
 * table's slab systems, close-packed layers of beads of size d/2 with a
 * fixed charge per bead.  Their beads interact like any other but the
 * integrators leave their positions and velocities unchanged and the
 * kinetic energy omits them. */

/* Langevin dynamics (gamma > 0).  The paper integrates Langevin equations of
 * motion in the canonical ensemble (method of image charges and illustrative
 * example sections) without naming a splitting; this library takes BAOAB
 * (Leimkuhler-Matthews), unit masses:
 *   v += dt/2 F;  x += dt/2 v;  v = c1 v + c2 z;  x += dt/2 v;  F = F(x);
 *   v += dt/2 F,  c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kT).
 * z of bead i (index within its system) at step n is counter-based:
 * Philox4x64-10 with counter (n, i, 0, 0) and key (seed, 0) gives four
 * words w_k, u_k = (floor(w_k / 2^40) + 1/2) / 2^24, and Box-Muller
 *   z = (sqrt(-2 ln u0) cos 2pi u1, sqrt(-2 ln u0) sin 2pi u1, sqrt(-2 ln u2) cos 2pi u3).
 * n is the system's own step counter (0 at creation, +1 per step; see
 * gcme_system_set_step_count), so a system's trajectory is the same alone,
 * in a batch or in the server. */

/* Pair-kernel path of the FP32 precision (the FP64 path always scans cells):
 * LIST keeps a Verlet neighbour list of every (j, image) within rc + 0.4
 * (the skin), rebuilt from the cell list when some bead has moved more than
 * half the skin since the last build, and evaluates the pair terms over it;
 * CELLS scans the 27 neighbour cells every step.  Both give the same pair
 * set (the FP32 in-cutoff rule on the wrapped positions of the step); the
 * FP32 sums differ in order, hence in rounding.  The list sums each bead's
 * terms in an order fixed by the pairs, so results do not depend on when
 * the list was rebuilt.  AUTO takes CELLS (the faster path on dense
 * soft-core fluids, where a bead has ~340 neighbours within rc and the
 * list is rebuilt every few steps).  A system
 * whose neighbour count exceeds the list capacity (about 1024 within
 * rc + skin) is evaluated by the cell kernel instead, step by step. */
#define GCME_PAIR_AUTO 0
#define GCME_PAIR_LIST 1
#define GCME_PAIR_CELLS 2

/* Fill p with the paper's defaults (A = 25, sigma = a = 0.5, lB = 1.2053,
 * rc = 3, kappa = 0.87609, p = 5, dt = 0.01, k = 100, r0 = 1) and a cubic
 * box of side L with grid K^3. */
void gcme_params_default(gcme_params *p, double L, int32_t K);

/* Message of the calling thread's last error ("" if none). */
const char *gcme_last_error(void);

/* Library version string. */
const char *gcme_version(void);

/* Host-only check of a system description, without a device: the same
 * validation gcme_system_create performs.  Returns 0 or GCME_ERR_INVALID
 * (message in gcme_last_error). */
int gcme_validate(const gcme_params *p, int64_t n, const double *h_q, const int32_t *h_types,
                  const int32_t *h_bonds, int64_t nbonds);

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device` (the library makes it current
 * for its own calls).  *out is owned by the caller; free with
 * gcme_ctx_destroy. */
int gcme_ctx_create(gcme_ctx **out, int device);
void gcme_ctx_destroy(gcme_ctx *ctx);

/* ---- single system ------------------------------------------------------- */

/* Create a system of n real beads with charges h_q[n] (charge numbers z_i),
 * species h_types[n] (in [0, p->ntypes); NULL = all of species 0) and an
 * optional bond list h_bonds[2*nbonds] (bead index pairs).  Validates:
 *   - net charge zero (|sum z| < 1e-6), n >= 1;
 *   - the non-collapse condition of the Gaussian core model section,
 *     A_ij / sigma_ij^3 > 4 pi^{3/2} |z_i z_j| lB / (3^{3/2} a_ij), for every
 *     pair of species present with their largest charges;
 *   - species tables: A_ij symmetric and >= 0, sigma_i, a_i > 0;
 *   - every box side >= rc (27-cell stencil) and, for slabs, the box height
 *     3 H (nonmetal) or 2 H (image charges);
 *   - grid sizes 2^a 3^b 5^c within [4, 1024], order within [3, 8].
 * Allocates the library's scratch memory for the system (cell lists, PME
 * grids, accumulators).  Errors: INVALID, OOM, CUDA. */
int gcme_system_create(gcme_ctx *ctx, const gcme_params *p, int64_t n,
                       const double *h_q, const int32_t *h_types, const int32_t *h_bonds,
                       int64_t nbonds, gcme_sys **out);
void gcme_system_destroy(gcme_sys *sys);

/* Build the cell list of the positions d_pos[n*3] (K1 + K2): wrap into the
 * box in FP64 (x - L floor(x/L)), cell c_a = floor(x_a n_a / L_a), cells of
 * side >= rc / cell_factor (n_a = floor(L_a / ((rc / cell_factor) (1 + 1e-4)))),
 * beads of a cell in (class, index) order with class 0 = image,
 * 1 = charged, 2 = neutral.  Outputs (caller-owned, may be NULL):
 *   d_cell_start[ncell+1], d_sorted_idx[n_ext]  (n_ext = n + images).
 * ncell and n_ext are returned by gcme_system_info. */
int gcme_build_cells(gcme_sys *sys, const double *d_pos, int32_t *d_cell_start,
                     int32_t *d_sorted_idx, gcme_stream_t stream);

/* Cell-list build that allocates no device memory (no counterpart in the
 * paper: an interface for callers that cannot call cudaMalloc, such as a
 * host program whose device memory belongs to another runtime's pool, or a
 * latency-bound loop that cannot afford cudaMalloc's implicit device
 * synchronisation).  Same result as gcme_build_cells for a system of n real
 * beads with parameters *p, positions d_pos[n*3] and charges d_q[n] (FP64,
 * device), written to the caller's d_cell_start[ncell+1] and
 * d_sorted_idx[n].  Scratch comes from one fixed file-scope device array
 * of about 3.9 MB, held by every GPU that loads the library until exit:
 *   - n <= 65536 beads and ncell <= 32768 cells, else INVALID with a message;
 *   - bulk and nonmetal-slab geometries only (no image charges), else INVALID;
 *   - the first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture;
 *   - every call shares the array and leaves its contents behind: calls
 *     whose work overlaps on the GPU (other streams, other threads) race,
 *     so serialise them;
 *   - no cudaMalloc, cudaFree or other allocating routine is called, and
 *     nothing is copied from host memory (the call's constants travel as a
 *     kernel argument).
 * ncell follows the rule of gcme_build_cells with cells of side
 * >= rc / f (f = p->cell_factor, 0 meaning 1):
 *   ncell = prod_a max(1, floor(box[a] / ((rc / f) (1 + 1e-4)))),
 * and gcme_cells_noalloc_size returns it without touching the GPU. */
int gcme_build_cells_noalloc(const gcme_params *p, int64_t n, const double *d_pos,
                             const double *d_q, int32_t *d_cell_start,
                             int32_t *d_sorted_idx, gcme_stream_t stream);

/* Host-only size query for gcme_build_cells_noalloc (no counterpart in the
 * paper): writes to *ncell the number of cells that call would use for n
 * beads with parameters *p, so that a caller that cannot create a system
 * (creating one allocates) can size d_cell_start[ncell + 1].  Applies the
 * same checks as the build (maxima, geometry, cell_factor) and returns
 * INVALID with the same messages; no CUDA call is made. */
int gcme_cells_noalloc_size(const gcme_params *p, int64_t n, int64_t *ncell);

/* Forces, energies and virial at positions d_pos[n*3] (FP64, any image).
 * d_force[3n] (fixed point, SoA), d_energy[GCME_NTERMS], d_virial[9]; any
 * output may be NULL.  Errors: INVALID, CUDA. */
int gcme_forces(gcme_sys *sys, const double *d_pos, int64_t *d_force,
                double *d_energy, double *d_virial, gcme_stream_t stream);

/* Convert fixed-point forces to FP64 (d_out[3n] in the same SoA layout). */
int gcme_forces_to_f64(gcme_sys *sys, const int64_t *d_force, double *d_out,
                       gcme_stream_t stream);

/* nsteps of NVE velocity Verlet with unit masses:
 *   v += dt/2 F;  x += dt v;  F = F(x);  v += dt/2 F.
 * Updates d_pos[n*3] (FP64, not wrapped) and d_vel[n*3] (FP32) in place and
 * writes the energies of the final state to d_energy (may be NULL).  Steps
 * run as replays of a captured CUDA graph (one per (d_pos, d_vel) pair). */
int gcme_step(gcme_sys *sys, double *d_pos, float *d_vel, int64_t nsteps,
              double *d_energy, gcme_stream_t stream);

/* Continue the trajectory of the last gcme_step / gcme_step_f64 call on the
 * same buffers for nsteps more steps, reusing the forces that call left at
 * the current positions (d_vel is float* or double* by the system's
 * precision).  The caller must not change d_pos or d_vel in between; calls
 * on other buffers return INVALID. */
int gcme_step_continue(gcme_sys *sys, double *d_pos, void *d_vel, int64_t nsteps,
                       double *d_energy, gcme_stream_t stream);

/* The same for FP64 systems (the plain FP64 path), FP64 velocities. */
int gcme_step_f64(gcme_sys *sys, double *d_pos, double *d_vel, int64_t nsteps,
                  double *d_energy, gcme_stream_t stream);

#define GCME_STEP_CONTINUE 1 /* gcme_step_host: reuse the last call's forces */

/* nsteps of velocity Verlet, as gcme_step, on a state held
 * on the host: h_pos[n*3] (FP64, not wrapped) and h_vel[n*3] (FP32) are
 * copied to device copies the system keeps, stepped, and copied back in
 * place, with the energies of the final state to h_energy[GCME_NTERMS] (may
 * be NULL).  The buffers must be page-locked (cudaHostAlloc, or
 * cudaHostRegister'ed); others return INVALID.  The copies and the steps are
 * enqueued on `stream` (for nsteps = 1 as one captured graph per set of host
 * buffers) and the call returns at once: synchronise the stream before
 * reading or changing the host buffers.  Without flags the forces at the
 * copied-in positions are evaluated first (as gcme_step); with
 * GCME_STEP_CONTINUE they are the forces the previous call on the same host
 * buffers left, valid when the caller has not changed the state since (as
 * gcme_step_continue; other buffers return INVALID).  The first call on a
 * system allocates its device copies (OOM on failure); FP64 systems return
 * INVALID.  Results are those of gcme_step on the same state bit for bit. */
int gcme_step_host(gcme_sys *sys, double *h_pos, float *h_vel, int64_t nsteps, double *h_energy,
                   int32_t flags, gcme_stream_t stream);

/* Phase timing on (on != 0) or off (the default).  With it on, later step
 * graphs carry CUDA event nodes between the phases, which lengthen a step
 * (by ~20 us per step on a GB300 at N = 32,000): for profiling only.  The
 * setting takes effect at the next gcme_step / gcme_step_continue call.
 * Errors: INVALID for a NULL system. */
int gcme_step_phase_timing(gcme_sys *sys, int32_t on);

/* Device time of the phases of the most recent completed step (the caller
 * synchronises first), measured by CUDA events captured in the step graph:
 * h_ms[0] half kick + drift, [1] cell list, [2] pair kernel (with the
 * harmonic bonds on the FP32 27-cell path), [3] PME (a branch on a side
 * stream concurrent with [2] and [4]), [4] bonds (other paths) and walls,
 * [5] Yeh-Berkowitz + half kick + energies after the join (nphase >= 6);
 * with nphase >= 8 also [6] binning alone (part of [1]) and [7] the second
 * half kick alone (part of [5]).
 * INVALID unless the most recent step ran with phase timing on
 * (gcme_step_phase_timing); h_ms may be NULL to query only *kernels (may be
 * NULL), the number of kernel launches in one step. */
#define GCME_NPHASE 8
int gcme_step_phase_ms(gcme_sys *sys, float *h_ms, int32_t nphase, int32_t *kernels);

/* Sizes of the system: n, n_ext, ncell, number of charged beads incl.
 * images, cells per axis. */
typedef struct gcme_sys_info {
  int64_t n, n_ext, n_charged_ext, ncell, nbonds;
  int32_t nc[3];
  int32_t cell_factor;
  int64_t scratch_bytes;
  int32_t pair_path;    /* path in use: GCME_PAIR_LIST or GCME_PAIR_CELLS */
  int32_t list_stride;  /* list entries per bead and lane (4 lanes), 0 without list */
  int64_t list_builds;  /* neighbour-list builds so far (synchronises the device) */
  int64_t steps;        /* the system's step counter (synchronises the device)   */
  double box[3];        /* current box (changes with gcme_system_set_box)       */
} gcme_sys_info;
int gcme_system_info(const gcme_sys *sys, gcme_sys_info *out);

/* ---- pressure and NpT (Parametrization section) ---------------------------
 * Bulk systems only.  gcme_pressure: the configuration's Eq. pres_virial,
 * p = (N kT + tr W / 3) / V, with W the virial of all forces (pair,
 * reciprocal, bonds) at d_pos; synchronises the stream.
 * gcme_system_set_box: change the periodic box (sides >= rc); the cell grid
 * is kept when its cell counts do not change, else the system's device
 * scratch is rebuilt (launch shapes kept).  Positions are not touched.
 * gcme_barostat_move: one Monte Carlo volume move of the NpT ensemble (the
 * paper's NpT runs name no barostat; reading: isotropic ln V moves),
 *   V' = V exp((2 u0 - 1) dlnv),  x' = x (V'/V)^{1/3}  (d_pos scaled in place),
 *   accepted iff dW <= 0 or u1 < exp(-dW / kT),
 *   dW = U(x', V') - U(x, V) + pressure (V' - V) - (N + 1) kT ln(V'/V),
 * u0, u1 = floor(w / 2^11) / 2^53 of the first two words of Philox4x64-10
 * at counter (move, 0, 0, 0) with key (seed, 1).  A rejected move restores
 * positions and box exactly.  *h_accepted = 1 or 0.  Velocities are not
 * scaled.  Two force evaluations and two synchronisations per move. */
int gcme_pressure(gcme_sys *sys, const double *d_pos, double kT, double *h_pressure,
                  gcme_stream_t stream);
int gcme_system_set_box(gcme_sys *sys, const double *box, gcme_stream_t stream);
int gcme_barostat_move(gcme_sys *sys, double *d_pos, double pressure, double kT, double dlnv,
                       uint64_t seed, uint64_t move, int32_t *h_accepted, gcme_stream_t stream);

/* Set the system's step counter (the Langevin noise counter of the next
 * step), e.g. to continue a trajectory from a checkpoint taken after
 * `steps` steps.  Enqueued on the stream; GCME_ERR_INVALID if steps < 0. */
int gcme_system_set_step_count(gcme_sys *sys, int64_t steps, gcme_stream_t stream);

/* Debug: every ordered in-cutoff triple (i, j, image code) found by the
 * pair kernel at d_pos, code = (nx+1) + 3 (ny+1) + 9 (nz+1).  Writes up to
 * cap triples to d_triples[3*cap] and the total to d_count[1].  Indices are
 * into the extended bead set (reals, then images). */
int gcme_debug_pairs(gcme_sys *sys, const double *d_pos, int32_t *d_triples,
                     int64_t cap, int64_t *d_count, gcme_stream_t stream);

/* Debug: the smooth-PME grids of the reciprocal part of Eq. ewald (Essmann
 * et al. 1995) at d_pos, for checking the FFT passes on their own: d_q[G]
 * the spread charge grid Q (FP64 from the fixed-point grid), d_phi[G] the
 * convolution theta * Q = F^-1[B C F(Q)] after the forward transform, the
 * influence function and the backward transform (transforms unnormalised,
 * so d_phi is K0 K1 K2 times the normalised convolution).  G = K0 K1 K2,
 * index kx + K0 (ky + K1 kz); either output may be NULL, not both.  Uses
 * the system's accumulators: a following gcme_step_continue needs a
 * gcme_step first.  Errors: INVALID, CUDA. */
int gcme_debug_pme_grids(gcme_sys *sys, const double *d_pos, double *d_q, double *d_phi,
                         gcme_stream_t stream);

/* Debug: launch a grid barrier that one CTA never reaches, so every other
 * CTA's bounded wait (timeout_s seconds, at most 10) runs out; returns
 * GCME_ERR_TIMEOUT when the kernel reported the timeout as designed.  Used
 * to test the failure path of the persistent launch without hanging. */
int gcme_debug_barrier_timeout(gcme_ctx *ctx, double timeout_s, gcme_stream_t stream);

/* ---- autotuner ------------------------------------------------------------ */

/* Tuned launch shapes: work items per home cell of the pair kernel (3: 9
 * neighbour cells each; 9: 3 each), pair block size (128, 160 or 192
 * threads) of which pair_nelec (1 to 3) electrostatics warps and the rest
 * Gaussian-core warps, resident pair
 * CTAs per SM fetching work items dynamically (0: one CTA per item), FFT
 * lines per tile per axis, x-y plane passes (1) or per-axis passes (0);
 * forces_ms: device time of one whole step (the step graph, on which the
 * candidates are timed) and pme_ms of the PME branch alone, with the chosen
 * shapes.
 * pair_nelec = 0 selects one warp per work item instead (both terms by the
 * same warp, 64, 96 or 128 threads per CTA, pair_ctas_per_sm >= 1 resident
 * CTAs with at most 28 warps per SM); its items are split by chunks of 32
 * home beads into pair_chunks items per (home cell, part): 1 to 4, or 0 for
 * the median real-bead count of the system's non-empty cells / 32.
 * pair_nelec = -1 to -3 (CTA items, 128, 160 or 192 threads) lets every warp
 * of a CTA take the item's tasks in turn: chunks of 32 home beads for the
 * Gaussian core, then chunks of 32 charged home beads in -pair_nelec parts
 * of the charged candidates (the sums of the static split with that many
 * electrostatics warps, which a cell with many beads would leave partly
 * idle).
 * spread_cells = 1 spreads the charges (FP32, 27-cell path without lists)
 * cell by cell through a brick of the grid in shared memory, the PME branch
 * then starting after the cell sort; 0 spreads each charge straight to the
 * grid in global memory, the branch starting after binning.
 * pair_group = 2 or 3 (split 9 CTA items only) lets one work item take
 * that many consecutive home cells along x in every system with at least
 * pair_group + 2 cells along x (others keep one home cell per item): the
 * pair_group + 2 cells of a neighbour row are staged once for all of them;
 * 1 (or 0 when applying) one home cell per item. */
typedef struct gcme_tuning {
  int32_t pair_split, pair_threads, pair_ctas_per_sm, fft_lpb[3], fft_plane, from_cache,
      cell_factor, pair_nelec, pair_chunks, spread_cells, pair_group;
  double forces_ms, pme_ms;
} gcme_tuning;

#define GCME_TUNE_REMEASURE 1 /* ignore a cached entry, time again       */
#define GCME_TUNE_NO_CACHE 2  /* neither read nor write the cache file   */

/* Time the candidate shapes on this system at positions d_pos (CUDA events
 * on `stream`; replays of the step graph on a scratch copy of the state
 * started from rest, the system's step counter restored afterwards), keep
 * the fastest and record it in the tuning cache
 * (GCME_TUNE_CACHE, else $HOME/.cache/gcme_tune.jsonl) keyed by GPU name and
 * workload shape; a cached entry is applied without timing.  Results of
 * later calls are unchanged except for FP32 summation order.  A following
 * gcme_step_continue must be preceded by gcme_step.  out may be NULL. */
int gcme_autotune(gcme_sys *sys, const double *d_pos, int32_t flags, gcme_tuning *out,
                  gcme_stream_t stream);

/* Apply given launch shapes without timing (e.g. a tuning recorded
 * elsewhere, or to pin one path): pair_split, pair_threads, pair_nelec,
 * pair_chunks, pair_group, spread_cells and pair_ctas_per_sm (27-cell path
 * of cell_factor 1 only; ignored otherwise),
 * fft_lpb[3] and fft_plane are read, every other field ignored.  A shape out
 * of range (see gcme_tuning), lines per tile or x-y planes that do not fit in
 * shared memory return GCME_ERR_INVALID and leave the shapes unchanged.
 * Results are unchanged except for FP32 summation order. */
int gcme_apply_tuning(gcme_sys *sys, const gcme_tuning *t);
int gcme_batch_apply_tuning(gcme_batch *b, const gcme_tuning *t);

/* ---- batch of independent systems ---------------------------------------- */

/* A batch of nsys independent systems stepped together: every phase of the
 * step is one launch over all systems (or one persistent cooperative launch
 * for all phases), replayed from a captured CUDA graph.  params[s], n[s],
 * charges h_q and species h_types (concatenated; h_types may be NULL), bonds
 * are per system as in gcme_system_create;
 * h_bond_count[s] gives the number of bonds of system s (concatenated in
 * h_bonds, indices local to the system).  The batch owns pooled device state:
 * positions, velocities, forces. */
int gcme_batch_create(gcme_ctx *ctx, int32_t nsys, const gcme_params *params,
                      const int64_t *n, const double *h_q, const int32_t *h_types,
                      const int32_t *h_bonds, const int64_t *h_bond_count, gcme_batch **out);
void gcme_batch_destroy(gcme_batch *b);

/* Copy state in/out (host, concatenated over systems in batch order). */
int gcme_batch_set_state(gcme_batch *b, const double *h_pos, const float *h_vel,
                         gcme_stream_t stream);
int gcme_batch_get_state(gcme_batch *b, double *h_pos, float *h_vel,
                         double *h_energy /* nsys * GCME_NTERMS */,
                         gcme_stream_t stream);

/* Step every system nsteps times.  mode 0: one launch per phase, the whole
 * step captured in a CUDA graph; mode 1: one persistent cooperative launch
 * running all phases of all steps with grid-wide barriers. */
int gcme_batch_step(gcme_batch *b, int64_t nsteps, int32_t mode, gcme_stream_t stream);

/* Autotune a batch on its current state (as gcme_autotune). */
int gcme_batch_autotune(gcme_batch *b, int32_t flags, gcme_tuning *out, gcme_stream_t stream);

/* Phase timing of a batch's step graphs (mode 0), as gcme_step_phase_timing. */
int gcme_batch_phase_timing(gcme_batch *b, int32_t on);

/* Phase times of the last batch step, as gcme_step_phase_ms. */
int gcme_batch_phase_ms(gcme_batch *b, float *h_ms, int32_t nphase, int32_t *kernels);

/* Device pointers to the pooled state (positions [3 N_tot] FP64, velocities
 * [3 N_tot] FP32, energies [nsys * GCME_NTERMS] FP64) and bead offsets. */
int gcme_batch_pointers(gcme_batch *b, double **d_pos, float **d_vel,
                        double **d_energy, const int64_t **h_bead_off);

/* ---- serving -------------------------------------------------------------- */

/* A continuous-batching request server.  A host thread owns a pool of
 * hbm_budget bytes; requests are admitted when their footprint fits, their
 * state stays on the device, and every chunk of `chunk_steps` steps (fewer
 * when every admitted request ends sooner) runs all admitted systems in one
 * batched launch sequence; a request with fewer steps left than the chunk
 * is held at its own count (its state unchanged) while the others step on.
 * Requests that arrive while others run are admitted at the next chunk
 * boundary.  Each result is the same bit for bit as the request run alone. */
typedef struct gcme_request {
  gcme_params params;
  int64_t n;
  const double *h_pos;   /* n*3, copied on submit */
  const float *h_vel;    /* n*3, copied on submit */
  const double *h_q;     /* n, copied on submit */
  const int32_t *h_bonds; /* 2*nbonds, may be NULL */
  int64_t nbonds;
  int64_t nsteps;
  const int32_t *h_types; /* n species, may be NULL (all species 0); copied on submit */
} gcme_request;

typedef struct gcme_result {
  int32_t status;        /* 0 done, 1 queued, 2 running, <0 error code */
  int64_t steps_done;
  double energy[GCME_NTERMS];
  double t_submit, t_admit, t_done; /* seconds, monotonic clock */
} gcme_result;

int gcme_server_create(gcme_ctx *ctx, size_t hbm_budget, int32_t chunk_steps,
                       int32_t max_active, gcme_server **out);
void gcme_server_destroy(gcme_server *srv);
/* Submit a request; copies all host inputs before returning. */
int gcme_submit(gcme_server *srv, const gcme_request *req, uint64_t *ticket);
/* Poll a ticket; when done, copies the final state to h_pos/h_vel if not
 * NULL (n*3 each).  Returns NOTFOUND for unknown or already-released tickets. */
int gcme_poll(gcme_server *srv, uint64_t ticket, gcme_result *out, double *h_pos,
              float *h_vel);
/* Release a finished ticket's host copy, or cancel a queued/running one. */
int gcme_cancel(gcme_server *srv, uint64_t ticket);
/* Block until every submitted request has finished (or timeout_s passes). */
int gcme_server_drain(gcme_server *srv, double timeout_s);
/* Counters: [0] admitted, [1] completed, [2] rejected, [3] chunks run,
 * [4] bead-steps done, [5] peak active, [6] peak bytes in use, [7] pooled
 * engines built for a new active set, [8] host microseconds spent building
 * them (overlapping the running chunk except for the first), [9] host
 * microseconds waiting for chunks to finish. */
int gcme_server_stats(gcme_server *srv, int64_t *out10);

#ifdef __cplusplus
}
#endif
#endif /* GCME_H */
