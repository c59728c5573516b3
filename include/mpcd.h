/*
 * mpcd.h -- C ABI of libmpcd, a single-GPU (NVIDIA GB300, sm_103a)
 * implementation of the per-step hot path of multiparticle collision dynamics
 * with the stochastic rotation dynamics (SRD) collision rule.
 *
 * Method: Howard, Panagiotopoulos & Nikoubashman, "Efficient mesoscale
 * hydrodynamics: multiparticle collision dynamics with massively parallel GPU
 * acceleration", arXiv:1801.10187.  One step is (Sec. 3, step flow):
 *   [solute velocity-Verlet substeps]           Sec. 2 / Sec. 3.6 (solute)
 *   ballistic streaming r <- r + v dt           Sec. 2, Eq. (stream)
 *   random grid shift, binning into cells       Sec. 2, Sec. 3.4
 *     (each particle record is appended to the row of its new cell, so the
 *      particles are grouped by cell every step: the reorder of Sec. 3.8 is
 *      part of binning)
 *   per-cell mass / momentum / kinetic energy   Sec. 3.5
 *   per-cell random axis [+ MB thermostat]      Sec. 3.6, Eq. (thermo)
 *   v <- u + xi R(alpha) (v - u)                Sec. 2, Eq. (srd); Sec. 3.6 algorithm
 * or, with the Andersen-thermostat collision rule (collision = MPCD_AT):
 *   v <- u + dv - <dv>_m, dv Gaussian per       Sec. 2, Eq. (at); Sec. 3.7
 *   particle, <dv>_m the cell's mass-weighted
 *   mean of dv
 *
 * Conventions
 *   - Lengths are in units of the cell edge a: the cell edge is 1 and the box
 *     is [0, n_x) x [0, n_y) x [0, n_z).  Positions outside are wrapped.
 *   - Host arrays are caller owned, row major (x, y, z per particle), and are
 *     only read or written during the call.  "_device" variants take device
 *     pointers to memory on the context's device; the call orders itself on
 *     the context's stream and does not synchronise unless stated.
 *   - Particles keep their input order (their tag) in every output.
 *   - Every call returns MPCD_OK (0) or a negative code below; the message of
 *     the last failure on the calling thread is mpcd_last_error().
 *   - Nothing here falls back to the CPU: without a usable CUDA device the
 *     creating calls fail with MPCD_ECUDA.
 */
#ifndef MPCD_H
#define MPCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPCD_OK 0
#define MPCD_EINVAL (-1)   /* invalid argument                                */
#define MPCD_ENOMEM (-2)   /* device memory exhausted                         */
#define MPCD_ECUDA (-3)    /* CUDA runtime error (message in mpcd_last_error) */
#define MPCD_EDEVICE (-4)  /* a device-side limit was hit (thermostat sampler  */
                           /* gave up after 64 attempts, or a cell id left the */
                           /* grid because a position was not finite)          */
#define MPCD_ESTATE (-5)   /* no state has been set                           */

typedef enum { MPCD_FP64 = 0, MPCD_MIXED = 1 } mpcd_precision;

/* Collision rules: stochastic rotation (Eq. srd, Sec. 3.6) or the Andersen
 * thermostat (Eq. at, Sec. 3.7).  The Andersen rule draws, for every member
 * of a cell, a velocity dv with Gaussian components of variance kT/m_i
 * (Box-Muller on Philox keyed by seed, step and the particle's tag) and sets
 * v_i <- u + dv_i - sum_j m_j dv_j / sum_j m_j, which is the paper's
 * (1/N_c) sum_j dv_j when all masses are equal; solute beads take part with
 * their mass.  It thermostats by itself, so it takes neither the thermostat
 * flag nor walls, and it needs a row capacity of at most 448 records
 * (a density below about 300 per cell) when beads take part.
 *
 * Angular-momentum conservation (angular = 1; the constraint the paper cites
 * after Eqs. srd and at, Sec. 2): after either rule every member of a cell
 * receives omega x r_c, r_c its position relative to the cell's centre of
 * mass and Pi omega = sum m r_c x (v - v') with the cell's inertia tensor Pi
 * about that centre (v before, v' after the rule), so each cell keeps its
 * angular momentum; a two-member or collinear cell takes omega = 2 dL /
 * tr(Pi).  The mixed model sums in int64 fixed point and solves in float.
 * Not with walls or solute (EINVAL).  Mixed-model SRD boxes take it in the
 * fused warp-spread pass; the Andersen rule and FP64 on a kernel with one
 * thread per cell (slower; same results). */
typedef enum { MPCD_SRD = 0, MPCD_AT = 1 } mpcd_collision;

/* SRD parameters (Sec. 2; Sec. 4 benchmark values in brackets).  Plain
 * values, copied at create time. */
typedef struct {
  int32_t n[3];          /* cells per axis                                   */
  int32_t precision;     /* mpcd_precision: FP64, or MIXED = float particles, */
                         /* int64 fixed-point cell sums (Sec. 4.1 model)     */
  double a;              /* cell edge; must be 1.0                           */
  double dt;             /* collision time Delta t [0.1]                      */
  double alpha;          /* rotation angle in radians [130 degrees]          */
  double kT;             /* thermal energy [1]                               */
  double mass;           /* solvent particle mass m [1]                      */
  uint64_t seed;         /* seed of all random draws                         */
  int32_t thermostat;    /* 1: Maxwell-Boltzmann cell thermostat (Eq. thermo)*/
  int32_t sort_period;   /* accepted for the reorder period of Sec. 3.8 [25]; */
                         /* records are grouped by cell every step here, so  */
                         /* it does not change the work or the results       */
  int32_t walls_z;       /* 1: no-slip bounce-back walls at z = 0, z = n_z   */
  int32_t collision;     /* mpcd_collision [MPCD_SRD]; alpha is unused by AT */
  double body_force[3];  /* constant acceleration g; g_z must be 0 w/ walls  */
  double virt_density;   /* density of virtual wall particles; 0 = N / V     */
  int32_t chain_len;     /* solute: beads per linear chain (0 = no solute)   */
  int32_t md_substeps;   /* solute: velocity-Verlet substeps per collision   */
  double solute_mass;    /* solute: bead mass M                              */
  double bond_k;         /* solute: harmonic bond constant k                 */
  double bond_r0;        /* solute: harmonic bond rest length r0             */
  int32_t angular;       /* 1: conserve each cell's angular momentum (below) */
  int32_t reserved1;
  double lj_epsilon;     /* solute: non-bonded WCA repulsion epsilon (0 off) */
  double lj_sigma;       /* solute: WCA sigma; cutoff 2^(1/6) sigma; needs    */
                         /* 2^(1/6) sigma + 0.4 <= 1 (neighbour-list buffer)  */
} mpcd_params;

/* Non-bonded solute forces (Sec. 4.3: the paper's polymer benchmark uses
 * pair forces from a neighbour list with a 0.4 a buffer and cites the
 * bead-spring potential): with lj_epsilon > 0 every pair of beads repels by
 * the Weeks-Chandler-Andersen potential U(r) = 4 eps ((sigma/r)^12 -
 * (sigma/r)^6) + eps for r < 2^(1/6) sigma (minimum-image distances), added
 * to the bond forces in every velocity-Verlet substep.  The neighbour list
 * (buffer 0.4) is built every collision step and rebuilt within it as soon as
 * a bead has moved more than half the buffer; a bead with more than 64
 * neighbours is reported as MPCD_EDEVICE.  Needs n_k >= 3 and
 * 2^(1/6) sigma + 0.4 <= 1 (EINVAL).  The list is built through a hash grid
 * filled by atomic exchange, so the order in which a bead's pair forces are
 * added, and with it the last bits of the bead states, may differ between
 * runs; without the repulsion the mixed model is reproducible bit for bit. */

/* Observables of the current state (Sec. 3.5, last paragraph). */
typedef struct {
  double P[3];           /* total momentum sum m v                           */
  double KE;             /* total kinetic energy sum m v^2 / 2               */
  double T_kin;          /* 2 (KE - |P|^2 / 2M) / (3 (N - 1))                */
  double T_cell_mean;    /* mean over cells of the unshifted grid with >= 2   */
                         /* members of 2 Ek / (3 (Nc - 1))                    */
  double mass;           /* total mass                                        */
  int64_t n;             /* particles (solvent + solute)                      */
  int64_t occupied_cells;/* cells of the unshifted grid with >= 1 member      */
  uint64_t step;         /* step counter                                      */
} mpcd_obs;

typedef struct mpcd_ctx mpcd_ctx;

/* Create a context for one box on the current CUDA device.  stream: a
 * cudaStream_t to order all work on (NULL = a stream the library creates).
 * Allocates the cell arrays; particle arrays are sized by set_state.
 * Errors: EINVAL (bad parameters, a != 1), ENOMEM, ECUDA. */
int mpcd_create(const mpcd_params* params, void* stream, mpcd_ctx** out);

/* Load the state (Sec. 3.2 particle data).  pos/vel: n_solvent x 3 doubles
 * (in MIXED mode rounded to float); solute_pos/solute_vel: n_solute x 3
 * doubles or NULL when n_solute == 0 (n_solute a multiple of chain_len).
 * step: the step counter t that keys the random draws.  Synchronises.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int mpcd_set_state(mpcd_ctx* ctx, int64_t n_solvent, const double* pos, const double* vel,
                   int64_t n_solute, const double* solute_pos, const double* solute_vel,
                   uint64_t step);

/* Same, from device memory: pos/vel are n_solvent x 3 arrays of float
 * (MIXED) or double (FP64) on the context's device. */
int mpcd_set_state_device(mpcd_ctx* ctx, int64_t n_solvent, const void* pos, const void* vel,
                          uint64_t step);

/* Thermal initial state drawn on the device (input generation, Sec. 4 /
 * Sec. 4.1 set-up): positions uniform in the box, velocity components
 * Gaussian with variance kT/m, mean velocity removed; reproducible from
 * init_seed.  No solute.  Synchronises.  Errors: EINVAL, ENOMEM, ECUDA. */
int mpcd_set_state_thermal(mpcd_ctx* ctx, int64_t n_solvent, uint64_t init_seed, uint64_t step);

/* Advance nsteps SRD steps.  Enqueued on the context's stream (replays of a
 * captured CUDA graph); returns without synchronising.  A device-side limit
 * hit during these steps is reported by the next synchronising call.
 * Errors: ESTATE, EINVAL (nsteps < 0), ECUDA. */
int mpcd_step(mpcd_ctx* ctx, int64_t nsteps);

/* Launch tuner (the paper tunes its kernels' launch parameters, among them
 * the threads per cell, on real steps at run time, Sec. 3.5 and Sec. 4): each
 * candidate of the fused step kernel -- its grid (1 up to the occupancy limit
 * of blocks per SM, and one block per span part) times, for mixed boxes with
 * the SRD rule and no angular correction, the cells each warp owns and the
 * depth of pass 2: 32 cells per warp with 2, 3 or 4 windows of 32 members
 * whose record loads and slot requests are in flight together, and 16 or 8
 * cells per warp with 3 (a 256-cell span is then taken in 2 or 4 parts, one
 * block each: more blocks for a small box, idle lanes in the per-cell work)
 * -- runs steps_per_candidate real steps, timed with CUDA events; the fastest
 * is kept for later steps.  The simulation advances by *steps_taken steps (one
 * more when the first step must stream and bin).  Results do not depend on
 * the candidate (mixed model bit for bit; FP64 to rounding).  Outputs may be
 * NULL: *blocks_per_sm (-1 = one block per span part), *ms_per_step of the
 * winner, *pass2_chunk (windows per chunk), *cells_per_warp (32, 16 or 8).
 * Synchronises.  Errors: EINVAL, ESTATE, ECUDA, EDEVICE. */
int mpcd_tune(mpcd_ctx* ctx, int64_t steps_per_candidate, int32_t* blocks_per_sm,
              double* ms_per_step, int64_t* steps_taken, int32_t* pass2_chunk,
              int32_t* cells_per_warp);

/* Copy the state out in input (tag) order; arrays as for set_state (solute
 * arrays may be NULL).  Synchronises.  Errors: ESTATE, ECUDA, EDEVICE. */
int mpcd_get_state(mpcd_ctx* ctx, double* pos, double* vel, double* solute_pos,
                   double* solute_vel, uint64_t* step);

/* Same into device arrays of the storage type (float for MIXED, double for
 * FP64), in input (tag) order.  Synchronises. */
int mpcd_get_state_device(mpcd_ctx* ctx, void* pos, void* vel);

/* Observables of the current state, computed on the device.  Synchronises. */
int mpcd_observables(mpcd_ctx* ctx, mpcd_obs* out);

/* Mean solvent v_x in nbins equal slabs of z in [0, n_z) (Poiseuille
 * profile), computed on the device.  out: nbins doubles.  Synchronises. */
int mpcd_profile(mpcd_ctx* ctx, int32_t nbins, double* out);

/* Allocation-free mpcd_profile, for callers that cannot allocate device
 * memory when they ask for a profile: a service that runs inside a fixed,
 * pre-reserved device-memory budget (every byte is handed out up front, so a
 * library allocation could fail or push the process over its budget), or a
 * job server that keeps nearly all of the GPU's memory filled with resident
 * boxes, where an allocation at query time could fail with out-of-memory.
 * Same result as mpcd_profile (nbins doubles, mean solvent v_x per z slab).
 * The per-bin scratch is a static device array of 4096 bins (64 KiB) that
 * every GPU loading the library holds until the process exits; nbins outside
 * [1, 4096] is rejected with MPCD_EINVAL.  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress, once per device), so
 * make the first call before any stream capture.  All calls share the array
 * and it keeps the last call's contents (each call clears the bins it uses):
 * calls whose work overlaps on the GPU (several threads, or contexts on
 * different streams) race and must be serialised by the caller.  Needs the
 * box on the device already: after set_state, call mpcd_step once (0 steps
 * is enough), else MPCD_ESTATE.  A pending collision is completed first.
 * Synchronises the box's stream: it waits for the box's work and copies the
 * result to the host.  The paper has no counterpart: this is an allocation
 * policy of the library, not part of the method. */
int mpcd_profile_noalloc(mpcd_ctx* ctx, int32_t nbins, double* out);

/* Per-particle cell ids and per-cell member counts of the LAST completed
 * step (diagnostics and tests).  cell_out: n_solvent + n_solute int32 in tag
 * order (may be NULL); count_out: mpcd_num_cells entries (may be NULL).
 * Synchronises. */
int mpcd_last_cells(mpcd_ctx* ctx, int32_t* cell_out, int32_t* count_out);

/* Internal profiler: advance nsteps SRD steps with plain launches and a CUDA
 * event between phases; ms[i] receives the mean time of phase i per step
 * (phases: md_bin, stream_bin, scan, scatter, permute, collide, end_step;
 * see mpcd_phase_name).  nmax: capacity of ms (>= 7).  Synchronises.  The
 * steps are real steps: the state advances. */
int mpcd_phase_times(mpcd_ctx* ctx, int64_t nsteps, double* ms, int32_t nmax, int32_t* nphases);
const char* mpcd_phase_name(int32_t i);

/* Number of collision cells (n_z + 2 layers when walls_z is set). */
int64_t mpcd_num_cells(const mpcd_ctx* ctx);

/* Release everything.  NULL is allowed. */
void mpcd_destroy(mpcd_ctx* ctx);

/* Message of the last failure on the calling thread ("" if none). */
const char* mpcd_last_error(void);

/* ---------------------------------------------------------------------- */
/* Batched ensembles: many independent boxes advanced by the same launches */
/* (one launch per phase covers every resident box).  Boxes differ in size, */
/* density, rotation angle, seed and thermostat; one precision per batch.   */
/* A box gives the same result alone and in any batch (counter-based draws  */
/* keyed by the box's own seed, step and cell).                             */
/* ---------------------------------------------------------------------- */
typedef struct mpcd_batch mpcd_batch;

/* Create an empty batch.  max_bytes: device-memory budget for admitted boxes
 * (0 = no limit beyond the device).  Errors: EINVAL, ECUDA. */
int mpcd_batch_create(int32_t precision, void* stream, int64_t max_bytes, mpcd_batch** out);

/* Device bytes a box of these parameters and n_solvent particles occupies. */
int64_t mpcd_box_footprint(const mpcd_params* params, int64_t n_solvent);

/* Admit a box with its initial state (host arrays, as mpcd_set_state; no
 * solute in batches).  *slot receives its handle.  Errors: EINVAL, ENOMEM
 * (over the budget or the device), ECUDA. */
int mpcd_batch_add(mpcd_batch* b, const mpcd_params* params, int64_t n_solvent,
                   const double* pos, const double* vel, uint64_t step, int32_t* slot);

/* Admit a box with a thermal initial state drawn on the device (as
 * mpcd_set_state_thermal). */
int mpcd_batch_add_thermal(mpcd_batch* b, const mpcd_params* params, int64_t n_solvent,
                           uint64_t init_seed, uint64_t step, int32_t* slot);

/* Advance every resident box by nsteps.  Asynchronous like mpcd_step. */
int mpcd_batch_step(mpcd_batch* b, int64_t nsteps);

/* mpcd_tune for every resident box together (one choice for the batch). */
int mpcd_batch_tune(mpcd_batch* b, int64_t steps_per_candidate, int32_t* blocks_per_sm,
                    double* ms_per_step, int64_t* steps_taken, int32_t* pass2_chunk,
                    int32_t* cells_per_warp);

/* Copy one box's state out (tag order).  Synchronises. */
int mpcd_batch_get_state(mpcd_batch* b, int32_t slot, double* pos, double* vel,
                         uint64_t* step);

/* Observables of one box.  Synchronises. */
int mpcd_batch_observables(mpcd_batch* b, int32_t slot, mpcd_obs* out);

/* Remove a box and free its memory. */
int mpcd_batch_remove(mpcd_batch* b, int32_t slot);

/* Wait until the batch's queued work is done; reports device-side limits
 * hit meanwhile (MPCD_EDEVICE). */
int mpcd_batch_sync(mpcd_batch* b);

/* Number of resident boxes and device bytes they hold. */
int mpcd_batch_info(const mpcd_batch* b, int32_t* n_boxes, int64_t* bytes_used);

void mpcd_batch_destroy(mpcd_batch* b);

#ifdef __cplusplus
}
#endif
#endif
