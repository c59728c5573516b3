// mpcd_internal.cuh -- device-side data layout and small device helpers of
// libmpcd (SRD step of arXiv:1801.10187 on one GB300, sm_103a).
//
// Layout in HBM, per box (Sec. 3.2 particle data and Sec. 3.4 cell list,
// re-laid for GB300): the particles live in their cells.  Cell c owns a row of
// K records; a record is one particle (position, velocity, input index) and
// is 32 bytes in the mixed model -- exactly one DRAM sector -- or 64 bytes in
// FP64.  cnt[c] counts the cell's members; members beyond K sit in an
// overflow list with their cell id.  Rows, counts and overflow lists are
// double buffered: the fused step reads one set (cells of step t) and
// writes the other (cells of step t + 1).  Solute beads (double) have their
// own arrays, grouped per tile of 32 cells.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace mpcd {

// Storage and arithmetic type of the two precision models: FP64, or the mixed
// model's FP32 particles.
template <bool MIXED>
using real_t = typename std::conditional<MIXED, float, double>::type;

// Random-stream purposes XORed into the high key word.
constexpr uint32_t PURPOSE_SHIFT = 0x53484654u;
constexpr uint32_t PURPOSE_ROT = 0x524F5441u;
constexpr uint32_t PURPOSE_THERMO = 0x54484D4Fu;
constexpr uint32_t PURPOSE_VIRT = 0x56495254u;
constexpr uint32_t PURPOSE_AT = 0x414E4452u;

// Collision rules: stochastic rotation (Eq. srd) or Andersen thermostat (Eq. at).
constexpr int RULE_SRD = 0;
constexpr int RULE_AT = 1;

// Error bits raised by kernels (read back by the host at sync points).
constexpr int ERR_GAMMA_CAP = 1;   // thermostat sampler rejected 64 times
constexpr int ERR_CELL_RANGE = 2;  // a cell id left the grid (non-finite position)

constexpr int PTILE = 1024;    // particles per tile of the particle-parallel kernels
constexpr int STILE = 2048;    // entries per scan tile
constexpr int BLOCK = 256;     // threads per block; the fused step has one thread per cell
constexpr int BEAD_TILE = 32;  // cells per bead group
constexpr int ERR_OVERFLOW_CAP = 4;  // overflow list full (cannot happen: it holds N records)
constexpr int ERR_NLIST = 8;   // solute neighbour list: more than NL_MAX pairs for a bead
constexpr int NL_MAX = 64;     // neighbours per bead in the solute pair list
constexpr double NL_SKIN = 0.4;  // neighbour-list buffer (the paper's 0.4 a)

// Passes of the fused step kernel.
enum { MODE_P = 0, MODE_F = 1, MODE_C = 2 };

// One particle (mixed model: 32 bytes, FP64: 64 bytes).  The mixed record
// keeps the velocity in its first 16 bytes, so the cell sums read one
// aligned 16-byte word per particle.
struct __align__(16) RecF {
  float vx, vy, vz;
  uint32_t tag;
  float x, y, z;
  uint32_t pad;
};
struct __align__(16) RecD {
  double x, y, z, vx, vy, vz;
  uint32_t tag, pad;
  uint64_t pad2;
};

struct BoxDev {
  // geometry and sizes
  int32_t n[3];         // cells per axis
  int32_t nzl;          // z layers of the collision grid (n_z, or n_z + 2 with walls)
  int32_t ncells;       // n[0] * n[1] * nzl
  int32_t nsol;         // solvent particles
  int32_t nbead;        // solute beads
  int32_t chain_len;
  int32_t md_substeps;
  int32_t thermostat;
  int32_t walls;
  int32_t K;            // records per cell row
  int32_t ovf_cap;      // capacity of each overflow list
  int32_t tc;           // cells per bead group (BEAD_TILE)
  int32_t nctiles;      // bead groups of this box
  uint32_t seed_lo, seed_hi;
  // parameters, double
  double dt, kT, m, Mb, bond_k, bond_r0, virt_density, sigma_virt;
  double ca, sa, omc;   // cos(alpha), sin(alpha), 1 - cos(alpha)
  double g[3], hg[3], gdt[3], L[3];
  double md_h, md_hh;   // MD substep and half-kick factor (0.5 h) / M
  // mixed model: E_k Mt = hm2 (n S2 - |Q|^2) for a cell of solvent only (hm2 = m^2 2^-65)
  double hm2;
  // parameters, float (mixed model)
  float dt_f, kT_f, m_f, Mb_f, ca_f, sa_f, omc_f, pad_f;
  float g_f[3], hg_f[3], gdt_f[3], L_f[3];
  // particle storage (double buffered; cur selects the current set)
  void* rows[2];        // ncells * K records
  uint32_t* cnt[2];     // members per cell
  void* ovf_rec[2];     // overflow records
  uint32_t* ovf_cell[2];
  uint32_t* ovf_n;      // two counters
  // solute
  double* spos;
  double* svel;
  int32_t* bcell;   // bead cell id of the current step
  uint64_t* bkey;   // bead (group << 32 | slot)
  uint32_t* border; // bead indices grouped by bead group
  int32_t* bgc;     // cell of each grouped bead (same order as border)
  double* bgv;      // velocity of each grouped bead, 3 per bead
  uint32_t* bcount; // per bead group histogram
  uint32_t* bstart; // nctiles + 1
  // updated on the device
  unsigned long long step;
  int32_t cur;
  int32_t collision;    // RULE_SRD or RULE_AT
  // Andersen rule: standard deviation sqrt(kT/m) of a random velocity
  // component, solvent and beads
  double sig, sigb;
  float sig_f, sigb_f;
  int32_t angular;      // 1: angular-momentum correction after the collision rule
  int32_t wca;          // 1: non-bonded WCA repulsion between beads
  // WCA: epsilon, sigma^2, cutoff^2, list radius^2 (cutoff + buffer), (buffer/2)^2
  double lj_eps, lj_sig2, wca_rc2, wca_rl2, wca_half_skin2;
  int32_t nl_hsize;     // hash buckets of the bead grid (2 per bead, tile-rounded)
  int32_t pad_w;
  int32_t* nl_head;     // bucket -> first bead (-1 empty)
  int32_t* nl_next;     // bead -> next bead in its bucket
  int32_t* nl_key;      // bead -> its cell (edge 1, unshifted) at the build
  int32_t* nl_cnt;      // bead -> neighbours listed
  int32_t* nl_nbr;      // bead -> neighbours (NL_MAX each)
  double* nl_rb;        // positions at the build (3 per bead)
  double* bF;           // forces on the beads (3 per bead)
  int32_t* nl_stale;    // 1: a bead moved more than half the buffer since the build
};

// Segments for the segmented exclusive scan (cells of each box, and bead
// counts per collision tile of each box).
struct ScanSeg {
  uint32_t* count;
  uint32_t* start;
  int32_t n;
  int32_t pad;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC11).  The 32x32->64 products
// come from a 32-bit multiply (low half) and __umulhi (high half).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo_a = 0xD2511F53u * c.x;
    const uint32_t hi_a = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo_b = 0xCD9E8D57u * c.z;
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi_b ^ c.y ^ k.x, lo_b, hi_a ^ c.w ^ k.y, lo_a);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint2 box_key(const BoxDev& B, uint32_t purpose) {
  return make_uint2(B.seed_lo, B.seed_hi ^ purpose);
}

__device__ __forceinline__ uint4 draw(const BoxDev& B, uint32_t purpose, uint32_t c0, uint32_t c1,
                                      unsigned long long t) {
  return philox(make_uint4(c0, c1, (uint32_t)t, (uint32_t)(t >> 32)), box_key(B, purpose));
}

// [0,1) from the top 53 bits of the 64-bit word (hi, lo).
// k 2^-53 for the top 53 bits k of (hi, lo), built from k's bits on the
// integer pipe (exact, so the same double as converting k and scaling).
__device__ __forceinline__ double unit53(uint32_t hi, uint32_t lo) {
  const unsigned long long k = (((unsigned long long)hi << 32) | lo) >> 11;
  if (k == 0ull) return 0.0;
  const int lz = __clzll((long long)k);  // 11..63: k's top bit at 63 - lz
  const unsigned long long m = k << (lz - 11);  // top bit at 52: adds one to the exponent
  return __longlong_as_double((long long)(((unsigned long long)(1032 - lz) << 52) + m));
}

// Grid shift of step t, in units of 2^-32 cell edges: S in [-2^31, 2^31).
__device__ __forceinline__ void shift_units(const BoxDev& B, unsigned long long t, long long S[3]) {
  const uint4 w = draw(B, PURPOSE_SHIFT, 0xFFFFFFFFu, 0u, t);
  S[0] = (long long)w.x - 2147483648LL;
  S[1] = (long long)w.y - 2147483648LL;
  S[2] = (long long)w.z - 2147483648LL;
}

constexpr double kTwoPi = 6.283185307179586;

}  // namespace mpcd
