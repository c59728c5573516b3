// k_collide.cu -- cell properties and SRD collision (arXiv:1801.10187,
// Sec. 3.5 cell properties, Sec. 3.6 rotation with the algorithm "SRD
// collision rule", Sec. 2 Eqs. srd and thermo).
//
// Kernels: k_collide<MIXED, THERMO, EXTRA> (fast path; EXTRA = solute beads
// or walls present) and k_collide_overflow (tiles too large for the fast path).
// One block owns a tile of TC consecutive cells of one box.  Because the
// particles are sorted by cell (order[] and start[] from the counting sort),
// the members of the tile are the contiguous range order[start[c0] ..
// start[c0+TC]).  The block
//   A. gathers those velocities into shared memory (coalesced index loads,
//      then the gathers, several in flight per thread),
//   B. gives each cell one thread: sums (int64 fixed point in the mixed model,
//      double in FP64), centre-of-mass velocity, random axis, and with the
//      thermostat a second pass for the kinetic energy about u and the Gamma
//      draw for xi,
//   C. rotates every member about its cell's axis and writes it back.
// Cell sums never leave the SM.  Tiles whose members exceed the shared-memory
// capacity (clustered input) take a block-cooperative path per cell that
// reads global memory directly; it gives the same results.
#include <type_traits>

#include "kernels.h"
#include "mpcd_internal.cuh"

namespace mpcd {

template <bool MIXED>
using real_t = typename std::conditional<MIXED, float, double>::type;

// ---------------------------------------------------------------------------
// Random axis (Sec. 3.6): z = 2u - 1, phi = 2 pi u', with
// sqrt(1 - z^2) = 2 sqrt(u (1 - u)) so that 1 - u is exact.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Exact conversions on the integer pipe.  On GB300 the float<->int64
// conversion instructions share the slow FP64 pipe, so the mixed model does
// them with integer operations; each one is the correctly rounded
// (round-half-even) conversion, identical to the hardware instruction.
// ---------------------------------------------------------------------------
// rne(x * 2^32) for a finite float x (fixed point with 32 fractional bits).
__device__ __forceinline__ long long fix32_rne(float x) {
  const uint32_t b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xFFu);
  if (e == 0) return 0;  // |x| < 2^-126: rounds to 0
  const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = e - 118;  // x 2^32 = m 2^(e - 150 + 32)
  long long q;
  if (sh >= 0) {
    q = m << (sh > 39 ? 39 : sh);  // |x| >= 2^30 is not a velocity; saturate
  } else {
    const int s = -sh;
    if (s >= 25) {
      q = 0;  // m 2^-s < 1/2
    } else {
      const long long rem = m & ((1LL << s) - 1);
      const long long half = 1LL << (s - 1);
      q = m >> s;
      if (rem > half || (rem == half && (q & 1))) q += 1;
    }
  }
  return (b & 0x80000000u) ? -q : q;
}

// rne(q) as a float for any int64 q.
__device__ __forceinline__ float i64_to_float(long long q) {
  if (q == 0) return 0.0f;
  const uint32_t sign = (q < 0) ? 0x80000000u : 0u;
  const unsigned long long a = (q < 0) ? (0ull - (unsigned long long)q) : (unsigned long long)q;
  int e = 63 - __clzll((long long)a);
  unsigned long long m;
  if (e <= 23) {
    m = a << (23 - e);
  } else {
    const int s = e - 23;
    m = a >> s;
    const unsigned long long rem = a & ((1ull << s) - 1ull);
    const unsigned long long half = 1ull << (s - 1);
    if (rem > half || (rem == half && (m & 1ull))) {
      m += 1ull;
      if (m == (1ull << 24)) {
        m >>= 1;
        e += 1;
      }
    }
  }
  return __uint_as_float(sign | ((uint32_t)(e + 127) << 23) | ((uint32_t)m & 0x7FFFFFu));
}

// Exact float of 0 <= n < 2^23 on the FMA pipe (2^23 + n has n as mantissa).
__device__ __forceinline__ float small_to_float(int n) {
  if ((unsigned)n < (1u << 23)) return __int_as_float(0x4B000000 | n) - 8388608.0f;
  return i64_to_float((long long)n);
}

// Float sin / cos / log of the mixed model, from IEEE basic operations only
// (every platform rounds them the same way): Taylor series of sin and cos on
// [0, pi/4] through x^9 / x^10, and log via x = m 2^e, m in [sqrt(1/2),
// sqrt(2)), ln m = 2 atanh((m - 1) / (m + 1)) summed through t^11.
__device__ __forceinline__ void series_sincos(float x, float& s, float& c) {
  const float x2 = x * x;
  const float s3 = (float)(-1.0 / 6.0), s5 = (float)(1.0 / 120.0);
  const float s7 = (float)(-1.0 / 5040.0), s9 = (float)(1.0 / 362880.0);
  const float c2 = -0.5f, c4 = (float)(1.0 / 24.0), c6 = (float)(-1.0 / 720.0);
  const float c8 = (float)(1.0 / 40320.0), c10 = (float)(-1.0 / 3628800.0);
  s = x + x * (x2 * (s3 + x2 * (s5 + x2 * (s7 + x2 * s9))));
  c = 1.0f + x2 * (c2 + x2 * (c4 + x2 * (c6 + x2 * (c8 + x2 * c10))));
}

// cos and sin of 2 pi w / 2^32: octant from the top three bits (an exact swap
// or negation), the other 29 bits place the angle inside it; odd octants are
// measured back from their upper end so the series argument is in [0, pi/4].
__device__ __forceinline__ void turn_cos_sin(uint32_t w, float& c, float& s) {
  const uint32_t o = w >> 29;
  const uint32_t f = w & 0x1FFFFFFFu;
  const uint32_t g = (o & 1u) ? (0x20000000u - f) : f;
  const float quarter_pi = (float)(3.14159265358979323846 / 4.0);
  const float x = (i64_to_float((long long)g) * 0x1p-29f) * quarter_pi;
  float sb, cb;
  series_sincos(x, sb, cb);
  switch (o) {
    case 0: c = cb; s = sb; break;
    case 1: c = sb; s = cb; break;
    case 2: c = -sb; s = cb; break;
    case 3: c = -cb; s = sb; break;
    case 4: c = -cb; s = -sb; break;
    case 5: c = -sb; s = -cb; break;
    case 6: c = sb; s = -cb; break;
    default: c = cb; s = -sb; break;
  }
}

__device__ __forceinline__ float series_log(float x) {
  if (!(x > 0.0f)) return x == 0.0f ? -INFINITY : __int_as_float(0x7FC00000);
  if (isinf(x)) return x;
  int e = 0;
  uint32_t b = __float_as_uint(x);
  if ((b >> 23) == 0) {  // subnormal
    x = x * 0x1p23f;
    b = __float_as_uint(x);
    e = -23;
  }
  e += (int)((b >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
  if (m > 1.41421354f) {
    m = m * 0.5f;
    e += 1;
  }
  const float t = (m - 1.0f) / (m + 1.0f);
  const float t2 = t * t;
  const float l3 = (float)(1.0 / 3.0), l5 = (float)(1.0 / 5.0), l7 = (float)(1.0 / 7.0);
  const float l9 = (float)(1.0 / 9.0), l11 = (float)(1.0 / 11.0);
  const float series = 1.0f + t2 * (l3 + t2 * (l5 + t2 * (l7 + t2 * (l9 + t2 * l11))));
  const float ln2 = (float)0.69314718055994530942;
  return (e >= 0 ? small_to_float(e) : -small_to_float(-e)) * ln2 + (2.0f * t) * series;
}

__device__ __forceinline__ void axis_of(const BoxDev& B, unsigned long long t, uint32_t cell,
                                        float n[3]) {
  const uint4 w = draw(B, PURPOSE_ROT, cell, 0u, t);
  const float a = i64_to_float((long long)w.x) * 0x1p-32f;
  const float b = i64_to_float(4294967296LL - (long long)w.x) * 0x1p-32f;
  const float z = i64_to_float(2LL * (long long)w.x - 4294967296LL) * 0x1p-32f;
  const float r = 2.0f * sqrtf(a * b);
  float c, s;
  turn_cos_sin(w.y, c, s);
  n[0] = r * c;
  n[1] = r * s;
  n[2] = z;
}

__device__ __forceinline__ void axis_of(const BoxDev& B, unsigned long long t, uint32_t cell,
                                        double n[3]) {
  const uint4 w = draw(B, PURPOSE_ROT, cell, 0u, t);
  const double a = (double)w.x * 0x1p-32;
  const double b = (double)(4294967296LL - (long long)w.x) * 0x1p-32;
  const double z = a - b;
  const double r = 2.0 * sqrt(a * b);
  const double phi = kTwoPi * ((double)w.y * 0x1p-32);
  n[0] = r * cos(phi);
  n[1] = r * sin(phi);
  n[2] = z;
}

// ---------------------------------------------------------------------------
// Eq. (thermo) / Sec. 3.6: E^ ~ Gamma(3(Nc-1)/2, kT) by Marsaglia-Tsang with a
// Box-Muller normal; attempt j uses counters (cell, 1+2j) and (cell, 2+2j).
// The float version settles acceptances within 1e-3 (1 + d) of the boundary
// in double from the same uniforms.  Returns false after 64 rejections.
// ---------------------------------------------------------------------------
__device__ bool gamma_draw(const BoxDev& B, unsigned long long t, uint32_t cell, int nc,
                           float& ehat) {
  const float kk = 1.5f * small_to_float(nc - 1);
  const float d = kk - 1.0f / 3.0f;
  const float c = 1.0f / sqrtf(9.0f * d);
  const double dd = (double)d, cd = (double)c;
  for (uint32_t j = 0; j < 64u; ++j) {
    const uint4 wa = draw(B, PURPOSE_THERMO, cell, 1u + 2u * j, t);
    const uint4 wb = draw(B, PURPOSE_THERMO, cell, 2u + 2u * j, t);
    const float e1 = i64_to_float(4294967296LL - (long long)wa.x) * 0x1p-32f;
    const float U3 = i64_to_float((long long)wb.x) * 0x1p-32f;
    float c2, s2;
    turn_cos_sin(wa.z, c2, s2);
    const float x = sqrtf(-2.0f * series_log(e1)) * c2;
    const float t1 = 1.0f + c * x;
    if (!(t1 > 0.0f)) continue;
    const float v = t1 * t1 * t1;
    const float lhs = series_log(U3);
    const float rhs = 0.5f * (x * x) + d - d * v + d * series_log(v);
    const float diff = lhs - rhs;
    bool accept;
    if (fabsf(diff) > 1e-3f * (1.0f + d)) {
      accept = diff < 0.0f;
    } else {
      const double xd = sqrt(-2.0 * log((double)e1)) * cos(kTwoPi * ((double)wa.z * 0x1p-32));
      const double td = 1.0 + cd * xd;
      if (!(td > 0.0)) continue;
      const double vd = td * td * td;
      accept = log((double)U3) < 0.5 * xd * xd + dd - dd * vd + dd * log(vd);
    }
    if (accept) {
      ehat = d * v * B.kT_f;
      return true;
    }
  }
  return false;
}

__device__ bool gamma_draw(const BoxDev& B, unsigned long long t, uint32_t cell, int nc,
                           double& ehat) {
  const double kk = 1.5 * (double)(nc - 1);
  const double d = kk - 1.0 / 3.0;
  const double c = 1.0 / sqrt(9.0 * d);
  for (uint32_t j = 0; j < 64u; ++j) {
    const uint4 wa = draw(B, PURPOSE_THERMO, cell, 1u + 2u * j, t);
    const uint4 wb = draw(B, PURPOSE_THERMO, cell, 2u + 2u * j, t);
    const double U1 = unit53(wa.x, wa.y), U2 = unit53(wa.z, wa.w), U3 = unit53(wb.x, wb.y);
    const double x = sqrt(-2.0 * log(1.0 - U1)) * cos(kTwoPi * U2);
    const double t1 = 1.0 + c * x;
    if (!(t1 > 0.0)) continue;
    const double v = t1 * t1 * t1;
    if (log(U3) < 0.5 * x * x + d - d * v + d * log(v)) {
      ehat = d * v * B.kT;
      return true;
    }
  }
  return false;
}

// ---------------------------------------------------------------------------
// Walls: virtual particles in the part of a wall-cut cell outside the channel
// (count with mean rho_v * f_out, Gaussian velocities of variance kT/m).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int virtual_count(const BoxDev& B, unsigned long long t, uint32_t cell,
                                             double sz) {
  const int cz = (int)(cell / (uint32_t)(B.n[0] * B.n[1]));
  const double H = B.L[2];
  const double lo = (double)(cz - 1) + sz;
  const double hi = lo + 1.0;
  const double a = lo > 0.0 ? lo : 0.0;
  const double b = hi < H ? hi : H;
  double inside = b - a;
  if (inside < 0.0) inside = 0.0;
  if (inside > 1.0) inside = 1.0;
  const double fout = 1.0 - inside;
  if (!(fout > 0.0) || !(fout < 1.0)) return 0;
  const double lam = B.virt_density * fout;
  const double fl = floor(lam);
  int nv = (int)fl;
  const uint4 w = draw(B, PURPOSE_VIRT, cell, 0u, t);
  if (unit53(w.x, w.y) < lam - fl) nv += 1;
  return nv;
}

__device__ __forceinline__ void virtual_velocity(const BoxDev& B, unsigned long long t,
                                                 uint32_t cell, int q, double vv[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint4 w = draw(B, PURPOSE_VIRT, cell, 1u + 3u * (uint32_t)q + (uint32_t)k, t);
    const double U = unit53(w.x, w.y), U2 = unit53(w.z, w.w);
    vv[k] = B.sigma_virt * (sqrt(-2.0 * log(1.0 - U)) * cos(kTwoPi * U2));
  }
}

// ---------------------------------------------------------------------------
// Accumulators of one cell.  Mixed model: solvent momentum as the sum of
// rne(v 2^32) (mass factored out), extra particles (beads, virtual) as the
// sum of rne(m v 2^32), energies the same way; all exact int64 sums, so the
// result does not depend on member order.  FP64: plain double sums.
// ---------------------------------------------------------------------------
template <bool MIXED> struct CellAcc;

template <> struct CellAcc<true> {
  long long q[3] = {0, 0, 0}, x[3] = {0, 0, 0};
  long long es = 0, ex = 0;
  int ns = 0, nb = 0, nv = 0;
  __device__ __forceinline__ void add_solvent(const BoxDev&, const float v[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) q[k] += fix32_rne(v[k]);
    ns += 1;
  }
  __device__ __forceinline__ void add_extra(double mass, const double v[3], bool bead) {
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] += __double2ll_rn((mass * v[k]) * 4294967296.0);
    if (bead) nb += 1;
    else nv += 1;
  }
  __device__ __forceinline__ void merge(const CellAcc& o) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      q[k] += o.q[k];
      x[k] += o.x[k];
    }
    es += o.es;
    ex += o.ex;
    ns += o.ns;
    nb += o.nb;
    nv += o.nv;
  }
  // u = P / M.  Without beads or virtual particles the extra terms are exact
  // zeros and are left out (same result).
  __device__ __forceinline__ void mean_velocity(const BoxDev& B, float u[3], bool extra) const {
    float M = B.m_f * small_to_float(ns);
    if (extra) M = M + (small_to_float(nb) * B.Mb_f + small_to_float(nv) * B.m_f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float P = B.m_f * i64_to_float(q[k]);
      if (extra) P = P + i64_to_float(x[k]);
      u[k] = (P * 0x1p-32f) / M;
    }
  }
  __device__ __forceinline__ void add_solvent_energy(const BoxDev&, const float v[3],
                                                     const float u[3]) {
    const float d0 = v[0] - u[0], d1 = v[1] - u[1], d2 = v[2] - u[2];
    const float e = d0 * d0 + d1 * d1 + d2 * d2;
    es += fix32_rne(e);
  }
  __device__ __forceinline__ void add_extra_energy(double mass, const double v[3], const float u[3]) {
    const double d0 = v[0] - (double)u[0], d1 = v[1] - (double)u[1], d2 = v[2] - (double)u[2];
    const double e = d0 * d0 + d1 * d1 + d2 * d2;
    ex += __double2ll_rn((mass * e) * 4294967296.0);
  }
  __device__ __forceinline__ float energy(const BoxDev& B, bool extra) const {
    float E = B.m_f * i64_to_float(es);
    if (extra) E = E + i64_to_float(ex);
    return (0.5f * E) * 0x1p-32f;
  }
  __device__ __forceinline__ void add_energy_partial(const CellAcc& o) { es += o.es; }
};

template <> struct CellAcc<false> {
  double P[3] = {0, 0, 0};
  double E = 0.0;
  int ns = 0, nb = 0, nv = 0;
  __device__ __forceinline__ void add_solvent(const BoxDev& B, const double v[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) P[k] += B.m * v[k];
    ns += 1;
  }
  __device__ __forceinline__ void add_extra(double mass, const double v[3], bool bead) {
#pragma unroll
    for (int k = 0; k < 3; ++k) P[k] += mass * v[k];
    if (bead) nb += 1;
    else nv += 1;
  }
  __device__ __forceinline__ void merge(const CellAcc& o) {
#pragma unroll
    for (int k = 0; k < 3; ++k) P[k] += o.P[k];
    E += o.E;
    ns += o.ns;
    nb += o.nb;
    nv += o.nv;
  }
  __device__ __forceinline__ void mean_velocity(const BoxDev& B, double u[3], bool) const {
    const double M = (double)ns * B.m + (double)nb * B.Mb + (double)nv * B.m;
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = P[k] / M;
  }
  __device__ __forceinline__ void add_solvent_energy(const BoxDev& B, const double v[3],
                                                     const double u[3]) {
    add_extra_energy(B.m, v, u);
  }
  __device__ __forceinline__ void add_extra_energy(double mass, const double v[3], const double u[3]) {
    const double d0 = v[0] - u[0], d1 = v[1] - u[1], d2 = v[2] - u[2];
    const double e = d0 * d0 + d1 * d1 + d2 * d2;
    E += (0.5 * mass) * e;
  }
  __device__ __forceinline__ double energy(const BoxDev&, bool) const { return E; }
  __device__ __forceinline__ void add_energy_partial(const CellAcc& o) { E += o.E; }
};

// Rodrigues form of R(alpha) about unit axis n applied to d (Eq. srd).
__device__ __forceinline__ void rotate(const float n[3], float ca, float sa, float omc,
                                       const float d[3], float out[3]) {
  const float nd = fmaf(n[2], d[2], fmaf(n[1], d[1], n[0] * d[0]));
  const float cr0 = fmaf(n[1], d[2], -(n[2] * d[1]));
  const float cr1 = fmaf(n[2], d[0], -(n[0] * d[2]));
  const float cr2 = fmaf(n[0], d[1], -(n[1] * d[0]));
  const float ndo = nd * omc;
  out[0] = fmaf(n[0], ndo, fmaf(cr0, sa, d[0] * ca));
  out[1] = fmaf(n[1], ndo, fmaf(cr1, sa, d[1] * ca));
  out[2] = fmaf(n[2], ndo, fmaf(cr2, sa, d[2] * ca));
}
__device__ __forceinline__ void rotate(const double n[3], double ca, double sa, double omc,
                                       const double d[3], double out[3]) {
  const double nd = fma(n[2], d[2], fma(n[1], d[1], n[0] * d[0]));
  const double cr0 = fma(n[1], d[2], -(n[2] * d[1]));
  const double cr1 = fma(n[2], d[0], -(n[0] * d[2]));
  const double cr2 = fma(n[0], d[1], -(n[1] * d[0]));
  const double ndo = nd * omc;
  out[0] = fma(n[0], ndo, fma(cr0, sa, d[0] * ca));
  out[1] = fma(n[1], ndo, fma(cr1, sa, d[1] * ca));
  out[2] = fma(n[2], ndo, fma(cr2, sa, d[2] * ca));
}

// Per-cell collision parameters.
template <typename T> struct CellParams {
  T u[3];
  T n[3];
  T xi;
};

// Finish a cell whose solvent sums are in `a`: add beads and virtual
// particles, compute u, the axis and (thermostat) xi.  `bead_in(j, b)`
// enumerates the tile's beads; `solvent_energy(u, acc)` adds the solvent's
// energy about u (a second pass over the members, done by the caller).
// `thermo` and `extra` are compile-time constants at the fast-path call sites.
template <bool MIXED, class BeadIn, class SolventEnergy>
__device__ __forceinline__ void finish_cell(const BoxDev& B, unsigned long long t, uint32_t cell,
                                            double sz, CellAcc<MIXED>& a, int nbt, BeadIn bead_in,
                                            SolventEnergy solvent_energy, bool thermo, bool extra,
                                            CellParams<real_t<MIXED>>& out, int* err) {
  using T = real_t<MIXED>;
  if (extra) {
    for (int j = 0; j < nbt; ++j) {
      int b;
      if (bead_in(j, b)) {
        const double vb[3] = {B.svel[3 * b], B.svel[3 * b + 1], B.svel[3 * b + 2]};
        a.add_extra(B.Mb, vb, true);
      }
    }
    if (B.walls) {
      const int nv = virtual_count(B, t, cell, sz);
      for (int q = 0; q < nv; ++q) {
        double vv[3];
        virtual_velocity(B, t, cell, q, vv);
        a.add_extra(B.m, vv, false);
      }
    }
  }
  T u[3];
  a.mean_velocity(B, u, extra);
  T n[3];
  axis_of(B, t, cell, n);
  T xi = (T)1;
  if (thermo) {
    solvent_energy(u, a);
    if (extra) {
      for (int j = 0; j < nbt; ++j) {
        int b;
        if (bead_in(j, b)) {
          const double vb[3] = {B.svel[3 * b], B.svel[3 * b + 1], B.svel[3 * b + 2]};
          a.add_extra_energy(B.Mb, vb, u);
        }
      }
      for (int q = 0; q < a.nv; ++q) {
        double vv[3];
        virtual_velocity(B, t, cell, q, vv);
        a.add_extra_energy(B.m, vv, u);
      }
    }
    const int nc = a.ns + a.nb + a.nv;
    const T Ek = a.energy(B, extra);
    if (nc >= 2 && Ek > (T)0) {
      T ehat;
      if (gamma_draw(B, t, cell, nc, ehat)) {
        if constexpr (MIXED) xi = sqrtf(ehat / Ek);
        else xi = sqrt(ehat / Ek);
      } else {
        atomicOr(err, ERR_GAMMA_CAP);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    out.u[k] = u[k];
    out.n[k] = n[k];
  }
  out.xi = xi;
}

template <bool MIXED>
__device__ __forceinline__ void collide_one(const BoxDev& B, const CellParams<real_t<MIXED>>& p,
                                            real_t<MIXED> v[3], bool thermo) {
  using T = real_t<MIXED>;
  T d[3], rr[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = v[k] - p.u[k];
  if constexpr (MIXED) rotate(p.n, B.ca_f, B.sa_f, B.omc_f, d, rr);
  else rotate(p.n, B.ca, B.sa, B.omc, d, rr);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T r = thermo ? p.xi * rr[k] : rr[k];
    v[k] = p.u[k] + r;
  }
}

// Beads are double in both models; in the mixed model they rotate with the
// cell's float parameters widened to double.
template <bool MIXED>
__device__ __forceinline__ void collide_bead(const BoxDev& B, const CellParams<real_t<MIXED>>& p,
                                             double v[3], bool thermo) {
  double n[3], u[3], d[3], rr[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    n[k] = (double)p.n[k];
    u[k] = (double)p.u[k];
    d[k] = v[k] - u[k];
  }
  rotate(n, B.ca, B.sa, B.omc, d, rr);
  const double xi = (double)p.xi;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double r = thermo ? xi * rr[k] : rr[k];
    v[k] = u[k] + r;
  }
}

// ---------------------------------------------------------------------------
// Fast path.  Shared memory (byte offsets from collide_smem_layout):
//   st[BLOCK+1] u32 | sidx[cap] u32 | vx, vy, vz[cap] T | lc[cap] u16 |
//   prm[BLOCK] CellParams | bidx[bcap] u32 | blc[bcap] u16
// ---------------------------------------------------------------------------
template <bool MIXED>
__host__ __device__ inline size_t collide_smem_layout(int cap, int bcap, size_t off[8]) {
  using T = real_t<MIXED>;
  size_t o = 0;
  auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
  off[0] = o; o = al(o + sizeof(uint32_t) * (BLOCK + 1));
  off[1] = o; o = al(o + sizeof(uint32_t) * cap);
  off[2] = o; o = al(o + sizeof(T) * 3 * cap);
  off[3] = o; o = al(o + sizeof(uint16_t) * cap);
  off[4] = o; o = al(o + sizeof(CellParams<T>) * BLOCK);
  off[5] = o; o = al(o + sizeof(uint32_t) * bcap);
  off[6] = o; o = al(o + sizeof(uint16_t) * bcap);
  off[7] = o;
  return o;
}

constexpr int GATHER = 4;  // independent gathers in flight per thread

template <bool MIXED, bool THERMO, bool EXTRA>
__global__ void __launch_bounds__(BLOCK, MIXED ? 4 : 2)
    k_collide(const BoxDev* __restrict__ boxes, const int2* __restrict__ tiles, int ntiles, int cap,
              int bcap, int2* __restrict__ ovf, int* __restrict__ novf, int* err) {
  using T = real_t<MIXED>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  size_t off[8];
  collide_smem_layout<MIXED>(cap, bcap, off);
  uint32_t* st = (uint32_t*)(smem_raw + off[0]);
  uint32_t* sidx = (uint32_t*)(smem_raw + off[1]);
  T* vx = (T*)(smem_raw + off[2]);
  T* vy = vx + cap;
  T* vz = vy + cap;
  uint16_t* lc = (uint16_t*)(smem_raw + off[3]);
  CellParams<T>* prm = (CellParams<T>*)(smem_raw + off[4]);
  uint32_t* bidx = (uint32_t*)(smem_raw + off[5]);
  uint16_t* blc = (uint16_t*)(smem_raw + off[6]);
  __shared__ long long sSz;

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int2 tt = tiles[tile];
    const BoxDev& B = boxes[tt.x];
    const unsigned long long t = B.step;
    const int c0 = tt.y;
    const int ncl = min(B.tc, B.ncells - c0);
    __syncthreads();
    for (int c = threadIdx.x; c <= ncl; c += BLOCK) st[c] = B.start[c0 + c];
    if (EXTRA && threadIdx.x == 0) {
      long long S[3];
      shift_units(B, t, S);
      sSz = S[2];
    }
    __syncthreads();
    const uint32_t p0 = st[0];
    const int np = (int)(st[ncl] - p0);
    int b0 = 0, nbt = 0;
    if (EXTRA && B.nbead > 0) {
      const int tl = c0 / B.tc;
      b0 = (int)B.bstart[tl];
      nbt = (int)B.bstart[tl + 1] - b0;
    }
    if (np > cap || nbt > bcap) {
      if (threadIdx.x == 0) ovf[atomicAdd(novf, 1)] = tt;
      continue;
    }
    const uint32_t* __restrict__ order = B.order;
    T* __restrict__ v = (T*)B.v;

    // ---- A: gather the tile's members, GATHER loads in flight per thread ----
    for (int base = 0; base < np; base += BLOCK * GATHER) {
      uint32_t idx[GATHER];
#pragma unroll
      for (int j = 0; j < GATHER; ++j) {
        const int k = base + j * BLOCK + threadIdx.x;
        idx[j] = (k < np) ? order[p0 + k] : 0u;
      }
      T w[GATHER][3];
#pragma unroll
      for (int j = 0; j < GATHER; ++j) {
        const int k = base + j * BLOCK + threadIdx.x;
        if (k < np) {
          w[j][0] = v[3 * idx[j]];
          w[j][1] = v[3 * idx[j] + 1];
          w[j][2] = v[3 * idx[j] + 2];
        }
      }
#pragma unroll
      for (int j = 0; j < GATHER; ++j) {
        const int k = base + j * BLOCK + threadIdx.x;
        if (k < np) {
          sidx[k] = idx[j];
          vx[k] = w[j][0];
          vy[k] = w[j][1];
          vz[k] = w[j][2];
        }
      }
    }
    for (int c = threadIdx.x; c < ncl; c += BLOCK) {
      const int e = (int)(st[c + 1] - p0);
      for (int k = (int)(st[c] - p0); k < e; ++k) lc[k] = (uint16_t)c;
    }
    if (EXTRA) {
      for (int j = threadIdx.x; j < nbt; j += BLOCK) {
        const uint32_t b = B.border[b0 + j];
        bidx[j] = b;
        blc[j] = (uint16_t)(B.bcell[b] - c0);
      }
    }
    __syncthreads();

    // ---- B: one thread per cell ----
    const double sz = EXTRA ? (double)sSz * 0x1p-32 : 0.0;
    for (int c = threadIdx.x; c < ncl; c += BLOCK) {
      const int kb = (int)(st[c] - p0), ke = (int)(st[c + 1] - p0);
      bool any = ke > kb;
      if (EXTRA)
        for (int j = 0; j < nbt; ++j) any |= (blc[j] == c);
      if (!any) continue;
      CellAcc<MIXED> a;
      for (int k = kb; k < ke; ++k) {
        const T w[3] = {vx[k], vy[k], vz[k]};
        a.add_solvent(B, w);
      }
      auto bead_in = [&](int j, int& b) {
        if (blc[j] != c) return false;
        b = (int)bidx[j];
        return true;
      };
      auto solvent_energy = [&](const T u[3], CellAcc<MIXED>& acc) {
        for (int k = kb; k < ke; ++k) {
          const T w[3] = {vx[k], vy[k], vz[k]};
          acc.add_solvent_energy(B, w, u);
        }
      };
      finish_cell<MIXED>(B, t, (uint32_t)(c0 + c), sz, a, EXTRA ? nbt : 0, bead_in,
                         solvent_energy, THERMO, EXTRA, prm[c], err);
    }
    __syncthreads();

    // ---- C: rotate and write back ----
    for (int k = threadIdx.x; k < np; k += BLOCK) {
      const CellParams<T> p = prm[lc[k]];
      T w[3] = {vx[k], vy[k], vz[k]};
      collide_one<MIXED>(B, p, w, THERMO);
      const uint32_t i = sidx[k];
      v[3 * i] = w[0];
      v[3 * i + 1] = w[1];
      v[3 * i + 2] = w[2];
    }
    if (EXTRA) {
      for (int j = threadIdx.x; j < nbt; j += BLOCK) {
        const int b = (int)bidx[j];
        double w[3] = {B.svel[3 * b], B.svel[3 * b + 1], B.svel[3 * b + 2]};
        collide_bead<MIXED>(B, prm[blc[j]], w, THERMO);
        B.svel[3 * b] = w[0];
        B.svel[3 * b + 1] = w[1];
        B.svel[3 * b + 2] = w[2];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Tiles the fast path queued (members beyond its shared-memory capacity):
// cell by cell, the whole block reduces straight from global memory.  Same
// arithmetic, so the same results.
// ---------------------------------------------------------------------------
template <bool MIXED>
__device__ CellAcc<MIXED> block_merge(CellAcc<MIXED> a, CellAcc<MIXED>* red) {
  __syncthreads();
  red[threadIdx.x] = a;
  __syncthreads();
  for (int s = BLOCK / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      CellAcc<MIXED> o = red[threadIdx.x];
      o.merge(red[threadIdx.x + s]);
      red[threadIdx.x] = o;
    }
    __syncthreads();
  }
  CellAcc<MIXED> r = red[0];
  __syncthreads();
  return r;
}

template <bool MIXED>
__global__ void __launch_bounds__(BLOCK) k_collide_overflow(const BoxDev* __restrict__ boxes,
                                                            const int2* __restrict__ ovf,
                                                            const int* __restrict__ novf, int* err) {
  using T = real_t<MIXED>;
  __shared__ CellAcc<MIXED> red[BLOCK];
  __shared__ CellParams<T> pc;
  __shared__ T su[3];
  __shared__ int sflag;
  const int n = *novf;
  for (int q = blockIdx.x; q < n; q += gridDim.x) {
    const int2 tt = ovf[q];
    const BoxDev& B = boxes[tt.x];
    const unsigned long long t = B.step;
    const int c0 = tt.y;
    const int ncl = min(B.tc, B.ncells - c0);
    const bool thermo = B.thermostat != 0;
    const bool extra = B.walls != 0 || B.nbead > 0;
    long long S[3];
    shift_units(B, t, S);
    const double sz = (double)S[2] * 0x1p-32;
    int b0 = 0, nbt = 0;
    if (B.nbead > 0) {
      const int tl = c0 / B.tc;
      b0 = (int)B.bstart[tl];
      nbt = (int)B.bstart[tl + 1] - b0;
    }
    const uint32_t* __restrict__ order = B.order;
    T* __restrict__ v = (T*)B.v;
    for (int c = 0; c < ncl; ++c) {
      const uint32_t kb = B.start[c0 + c], ke = B.start[c0 + c + 1];
      const uint32_t cell = (uint32_t)(c0 + c);
      __syncthreads();
      if (threadIdx.x == 0) {
        int any = (ke > kb) ? 1 : 0;
        for (int j = 0; j < nbt && !any; ++j) any = (B.bcell[B.border[b0 + j]] == (int)cell) ? 1 : 0;
        sflag = any;
      }
      __syncthreads();
      if (!sflag) continue;
      CellAcc<MIXED> a;
      for (uint32_t k = kb + threadIdx.x; k < ke; k += BLOCK) {
        const uint32_t i = order[k];
        const T w[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
        a.add_solvent(B, w);
      }
      CellAcc<MIXED> tot = block_merge<MIXED>(a, red);
      auto bead_in = [&](int j, int& bb) {
        bb = (int)B.border[b0 + j];
        return B.bcell[bb] == (int)cell;
      };
      if (threadIdx.x == 0) {
        CellAcc<MIXED> b = tot;
        if (extra) {
          for (int j = 0; j < nbt; ++j) {
            int bb;
            if (!bead_in(j, bb)) continue;
            const double vb[3] = {B.svel[3 * bb], B.svel[3 * bb + 1], B.svel[3 * bb + 2]};
            b.add_extra(B.Mb, vb, true);
          }
          if (B.walls) {
            const int nv = virtual_count(B, t, cell, sz);
            for (int qq = 0; qq < nv; ++qq) {
              double vv[3];
              virtual_velocity(B, t, cell, qq, vv);
              b.add_extra(B.m, vv, false);
            }
          }
        }
        T u[3];
        b.mean_velocity(B, u, extra);
        su[0] = u[0];
        su[1] = u[1];
        su[2] = u[2];
      }
      __syncthreads();
      CellAcc<MIXED> ea;
      if (thermo) {
        const T u[3] = {su[0], su[1], su[2]};
        for (uint32_t k = kb + threadIdx.x; k < ke; k += BLOCK) {
          const uint32_t i = order[k];
          const T w[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
          ea.add_solvent_energy(B, w, u);
        }
      }
      const CellAcc<MIXED> etot = block_merge<MIXED>(ea, red);
      if (threadIdx.x == 0) {
        auto solvent_energy = [&](const T[3], CellAcc<MIXED>& acc) { acc.add_energy_partial(etot); };
        finish_cell<MIXED>(B, t, cell, sz, tot, nbt, bead_in, solvent_energy, thermo, extra, pc, err);
      }
      __syncthreads();
      const CellParams<T> p = pc;
      for (uint32_t k = kb + threadIdx.x; k < ke; k += BLOCK) {
        const uint32_t i = order[k];
        T w[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
        collide_one<MIXED>(B, p, w, thermo);
        v[3 * i] = w[0];
        v[3 * i + 1] = w[1];
        v[3 * i + 2] = w[2];
      }
      for (int j = threadIdx.x; j < nbt; j += BLOCK) {
        int bb;
        if (!bead_in(j, bb)) continue;
        double w[3] = {B.svel[3 * bb], B.svel[3 * bb + 1], B.svel[3 * bb + 2]};
        collide_bead<MIXED>(B, p, w, thermo);
        B.svel[3 * bb] = w[0];
        B.svel[3 * bb + 1] = w[1];
        B.svel[3 * bb + 2] = w[2];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <bool M, bool TH, bool EX>
static void* collide_fn() {
  return (void*)k_collide<M, TH, EX>;
}

static void* collide_variant(bool mixed, int variant) {
  const bool th = (variant & 1) != 0, ex = (variant & 2) != 0;
  if (mixed) {
    if (th) return ex ? collide_fn<true, true, true>() : collide_fn<true, true, false>();
    return ex ? collide_fn<true, false, true>() : collide_fn<true, false, false>();
  }
  if (th) return ex ? collide_fn<false, true, true>() : collide_fn<false, true, false>();
  return ex ? collide_fn<false, false, true>() : collide_fn<false, false, false>();
}

size_t collide_smem_bytes(bool mixed, int cap, int bcap) {
  size_t off[8];
  return mixed ? collide_smem_layout<true>(cap, bcap, off) : collide_smem_layout<false>(cap, bcap, off);
}

cudaError_t prepare_collide(bool mixed, size_t smem) {
  for (int v = 0; v < 4; ++v) {
    cudaError_t e = cudaFuncSetAttribute(collide_variant(mixed, v),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int collide_blocks_per_sm(bool mixed, int variant, size_t smem) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, collide_variant(mixed, variant), BLOCK, smem);
  return nb;
}

void launch_collide(bool mixed, int variant, const BoxDev* boxes, const int2* tiles, int ntiles,
                    int grid, int cap, int bcap, size_t smem, int2* ovf, int* novf, int* err,
                    cudaStream_t s) {
  if (ntiles <= 0) return;
  void* args[] = {(void*)&boxes, (void*)&tiles, (void*)&ntiles, (void*)&cap, (void*)&bcap,
                  (void*)&ovf, (void*)&novf, (void*)&err};
  cudaLaunchKernel(collide_variant(mixed, variant), dim3(grid), dim3(BLOCK), args, smem, s);
}

void launch_collide_overflow(bool mixed, const BoxDev* boxes, const int2* ovf, const int* novf,
                             int grid, int* err, cudaStream_t s) {
  if (mixed) k_collide_overflow<true><<<grid, BLOCK, 0, s>>>(boxes, ovf, novf, err);
  else k_collide_overflow<false><<<grid, BLOCK, 0, s>>>(boxes, ovf, novf, err);
}

}  // namespace mpcd
