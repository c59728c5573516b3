/*
 * mpcd_oracle.h -- plain, slow CPU oracle for one SRD (stochastic rotation
 * dynamics) step of multiparticle collision dynamics.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The GPU product path never
 * links, calls or includes anything from this directory, and this code
 * includes nothing from the product.
 *
 * What it computes (Howard, Panagiotopoulos & Nikoubashman, arXiv:1801.10187):
 *   Sec. 2, Eq. (stream) : ballistic streaming r <- r + v dt
 *   Sec. 2 / Sec. 3.4    : random grid shift, cubic cells of edge a = 1
 *   Sec. 3.5             : per-cell mass, momentum and kinetic energy
 *   Sec. 2, Eq. (srd)    : v <- u + R(alpha) (v - u), random axis per cell
 *   Sec. 2, Eq. (thermo) : Maxwell-Boltzmann cell thermostat, xi = sqrt(E^/Ek)
 *   Sec. 2, Eq. (at)     : Andersen-thermostat collision rule (Sec. 3.7):
 *                          v <- u + dv_i - <dv>, dv_i Gaussian per particle
 *   Sec. 2 (after Eqs. srd and at): optional angular-momentum conservation,
 *                          a rigid rotation of each cell's relative velocities
 *                          that restores its angular momentum
 *   Sec. 3.6             : cylindrical-projection axis, Marsaglia-Tsang Gamma
 *                          draw with a Box-Muller normal, xi = 1 if Nc < 2
 *   Sec. 2 / Sec. 3.6    : solute beads (velocity Verlet, harmonic bonds, and
 *                          optionally a non-bonded pair repulsion, Sec. 4.3)
 *                          binned and collided with the solvent
 *   Sec. 3.5 (last par.) : net momentum / energy / temperature observables
 * Walls with bounce-back and a body force are not given in the paper (Sec. 5
 * lists them as future extensions); the reading implemented here is the one
 * the design notes state.
 *
 * Arithmetic modes:
 *   ORACLE_FP64  : every quantity in double; sums in particle-index order.
 *   ORACLE_MIXED : positions/velocities rounded to float after every store,
 *                  cell momentum/energy sums in int64 fixed point (scale 2^32),
 *                  rotation and the thermostat's Gamma draw in float with the
 *                  operation order fixed below; the thermostat factor
 *                  xi = sqrt(E^/E_k) in double (then rounded to float);
 *                  solute beads stay double.
 *   ORACLE_FP64_FSTREAM : the FP64 model of one mixed-model step.  The float
 *                  state streams as in ORACLE_MIXED (float fmaf, float wrap,
 *                  positions and velocities stored as floats); binning, cell
 *                  sums, the draws, xi and the collision are those of
 *                  ORACLE_FP64.  From the same float state both modes see the
 *                  same cells, so the velocities after one step measure the
 *                  error of the mixed arithmetic alone.
 * State arrays are always passed as double; in MIXED mode they hold floats.
 */
#ifndef MPCD_ORACLE_H
#define MPCD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_FP64 = 0, ORACLE_MIXED = 1, ORACLE_FP64_FSTREAM = 2 };

/* Random-stream purposes, XORed into the high key word (see oracle_key). */
#define ORACLE_PURPOSE_SHIFT  0x53484654u
#define ORACLE_PURPOSE_ROT    0x524F5441u
#define ORACLE_PURPOSE_THERMO 0x54484D4Fu
#define ORACLE_PURPOSE_VIRT   0x56495254u
#define ORACLE_PURPOSE_AT     0x414E4452u

/* Collision rules. */
enum { ORACLE_SRD = 0, ORACLE_AT = 1 };

typedef struct {
  int32_t n[3];          /* cells per axis; cell edge a = 1, box L_k = n_k   */
  double dt;             /* collision time Delta t                          */
  double alpha;          /* rotation angle (radians)                        */
  double kT;             /* thermal energy                                  */
  double mass;           /* solvent particle mass m                         */
  uint64_t seed;         /* user seed                                       */
  int32_t thermostat;    /* 1 = Maxwell-Boltzmann cell thermostat           */
  int32_t walls_z;       /* 1 = bounce-back walls at z = 0 and z = n_z      */
  double g[3];           /* body-force acceleration (g[2] must be 0 w/ walls)*/
  double virt_density;   /* virtual-particle density in wall-cut cells      */
  int32_t precision;     /* ORACLE_FP64, ORACLE_MIXED or ORACLE_FP64_FSTREAM */
  int32_t chain_len;     /* beads per chain (solute)                        */
  int32_t md_substeps;   /* velocity-Verlet substeps per collision          */
  int32_t collision;     /* ORACLE_SRD (Eq. srd) or ORACLE_AT (Eq. at)      */
  double solute_mass;    /* bead mass M                                     */
  double bond_k;         /* harmonic bond constant                          */
  double bond_r0;        /* harmonic bond rest length                       */
  int32_t angular;       /* 1 = conserve each cell's angular momentum        */
  int32_t pad2_;
  double lj_epsilon;     /* solute non-bonded WCA repulsion: epsilon (0 off) */
  double lj_sigma;       /* and sigma (cutoff 2^(1/6) sigma)                 */
} oracle_params;

/* Philox4x32-10 (Salmon et al., SC11) on one counter block. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The mixed model's own float functions (exposed for their pins):
 * cos and sin of 2 pi w / 2^32, and the natural logarithm. */
void oracle_cos_sin_turn_f(uint32_t w, float* c, float* s);
float oracle_log_f(float x);
/* The mixed model's float -ln(1 - U) for the 53-bit uniform U with high and
 * low words hi, lo (the squared Box-Muller radius over two); lo is used only
 * when 1 - U < 2^-12. */
float oracle_neg_log1m_f(uint32_t hi, uint32_t lo);
/* The mixed model's thermostat factor sqrt(ehat / ek) (ehat, ek > 0): a float
 * estimate refined by one FP64 Newton step, then rounded to float. */
float oracle_xi_mixed(double ehat, double ek);

/* Grid shift of step t: s_k = S_k * 2^-32, S_k in [-2^31, 2^31). */
void oracle_shift(uint64_t seed, uint64_t t, double s[3]);

/* Rotation axis of a cell at step t (cylindrical projection, Sec. 3.6). */
void oracle_axis(uint64_t seed, uint64_t t, uint32_t cell, int32_t precision, double n[3]);

/* Maxwell-Boltzmann kinetic-energy draw for a cell with nc >= 2 members:
 * Gamma(3(nc-1)/2, kT) by Marsaglia-Tsang with its squeeze.  Attempt j reads
 * Philox block A = counter (cell, 1 + 2j): words 0, 2, 1 are the high words
 * of the uniforms U1, U2, U3 (Box-Muller from U1, U2; acceptance from U3);
 * the FP64 model takes their low words from block B = (cell, 2 + 2j), the
 * mixed model only the low word of U1 when 1 - U1 < 2^-12.  In the mixed
 * model the normal, the squeeze and the acceptance are float and
 * E^ = (d v) kT is formed in double from the float d and v.
 * Returns 0, or -4 if 64 attempts were all rejected. */
int32_t oracle_gamma_draw(uint64_t seed, uint64_t t, uint32_t cell, int32_t nc,
                          double kT, int32_t precision, double* ehat);

/* Random velocity dv of one particle for the Andersen-thermostat rule
 * (Sec. 3.7): three Gaussian components of standard deviation sigma
 * (sqrt(kT/m) of that particle) by Box-Muller.  tag: input index of the
 * particle; kind: 0 solvent, 1 solute bead.  MIXED: one Philox block at
 * counter (tag, 2 kind) gives (w0, w1) -> components 0, 1 (cos and sin) and
 * (w2, w3) -> component 2 (cos), all in float; FP64: 53-bit uniforms whose
 * high words come from that block and low words from (tag, 2 kind + 1). */
void oracle_at_draw(uint64_t seed, uint64_t t, uint32_t tag, int32_t kind, double sigma,
                    int32_t precision, double dv[3]);

/* Advance nsteps SRD steps in place.  pos/vel: n*3 (x,y,z per particle);
 * spos/svel: nb*3 bead state (nb a multiple of chain_len).  *step is the
 * step counter t, incremented per step.  If cell_out != NULL it receives the
 * cell id of every particle (solvent then beads) at the last step; if
 * count_out != NULL it receives the member count (solvent + beads) of every
 * cell at the last step (oracle_num_cells entries).
 * The Andersen rule takes no thermostat flag and no walls (-1 otherwise);
 * angular momentum conservation takes no walls and no solute (-1 otherwise).
 * Returns 0, -1 invalid argument, -4 Gamma sampler cap reached. */
int32_t oracle_step(const oracle_params* p, int64_t n, double* pos, double* vel,
                    int64_t nb, double* spos, double* svel, uint64_t* step,
                    int64_t nsteps, int32_t* cell_out, int32_t* count_out);

/* Solute forces (bonds and, with lj_epsilon > 0, the WCA pair repulsion)
 * on nb beads at r (nb x 3; chains of chain_len consecutive beads), and the
 * potential energy they derive from. */
void oracle_solute_forces(const oracle_params* p, int64_t nb, const double* r, double* F);
double oracle_solute_energy(const oracle_params* p, int64_t nb, const double* r);

/* Number of cells of the collision grid (n_z + 2 layers when walls_z). */
int64_t oracle_num_cells(const oracle_params* p);

/* Observables of the current state.  out[0..2] total momentum, out[3] total
 * kinetic energy, out[4] kinetic temperature, out[5] mean cell temperature on
 * the unshifted grid over cells with >= 2 members, out[6] number of occupied
 * cells of that grid, out[7] total mass. */
int32_t oracle_observables(const oracle_params* p, int64_t n, const double* pos,
                           const double* vel, int64_t nb, const double* spos,
                           const double* svel, double* out);

/* Mean solvent v_x in nbins equal slabs of z in [0, n_z). */
int32_t oracle_profile(const oracle_params* p, int64_t n, const double* pos,
                       const double* vel, int32_t nbins, double* out);

#ifdef __cplusplus
}
#endif
#endif
