// dev_collide.cuh -- device helpers of the cell properties and the SRD
// collision (arXiv:1801.10187, Sec. 3.5 cell properties; Sec. 3.6 random
// axis, Maxwell-Boltzmann thermostat and the algorithm "SRD collision rule";
// Sec. 2 Eqs. srd and thermo).
#pragma once
#include <type_traits>

#include "mpcd_internal.cuh"

namespace mpcd {

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

// rne(x * 2^32) = H * 2^20 + L for |x| < 2^10, with H = rne(x 2^12) and
// L = rne((x 2^12 - H) 2^20), both obtained by adding 1.5 * 2^23 (which rounds
// to an integer in place) and reading the bits: eight FP32/INT32 operations,
// exact, and summable in int32 over a cell.  Returns false outside the range.
__device__ __forceinline__ bool split32(float x, int& H, int& L) {
  const float a = x * 4096.0f;
  if (!(fabsf(a) < 4194304.0f)) return false;
  const float t = __fadd_rn(a, 12582912.0f);
  H = __float_as_int(t) - 0x4B400000;
  const float hf = __fsub_rn(t, 12582912.0f);
  const float l = __fmul_rn(__fsub_rn(a, hf), 1048576.0f);
  const float t2 = __fadd_rn(l, 12582912.0f);
  L = __float_as_int(t2) - 0x4B400000;
  return true;
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

// Correctly rounded floats of 32-bit words: the word itself, 2^32 minus the
// word, and twice the word minus 2^32 (the last two as an exact power-of-two
// scaling of a 32-bit value); they equal i64_to_float of the same integers.
__device__ __forceinline__ float word_to_float(uint32_t w) { return __uint2float_rn(w); }
__device__ __forceinline__ float comp_word_to_float(uint32_t w) {
  return w == 0u ? 4294967296.0f : __uint2float_rn(0u - w);
}
__device__ __forceinline__ float centred_word_half_to_float(uint32_t w) {
  return __int2float_rn((int)(w ^ 0x80000000u));  // w - 2^31
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
  const float x = (word_to_float(g) * 0x1p-29f) * quarter_pi;
  float sb, cb;
  series_sincos(x, sb, cb);
  // octants 1, 2, 5, 6 swap the two; cos is negative in octants 2..5, sin in 4..7
  const bool swap = ((o + 1u) >> 1) & 1u;
  const uint32_t cneg = (((o + 2u) >> 2) & 1u) << 31, sneg = ((o >> 2) & 1u) << 31;
  c = __uint_as_float(__float_as_uint(swap ? sb : cb) ^ cneg);
  s = __uint_as_float(__float_as_uint(swap ? cb : sb) ^ sneg);
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

// rne(q) as a float for 0 <= q < 2^63, on the integer pipe.
__device__ __forceinline__ float u63_to_float(unsigned long long q) { return i64_to_float((long long)q); }

// -ln(1 - U) in float (the squared Box-Muller radius over two) for the 53-bit
// uniform U with high word hi; lo_of() supplies its low word and is called
// only when 1 - U < 2^-12.  U < 1/2: 2 atanh(U / (2 - U)) with U = hi 2^-32
// (series through t^15, t <= 1/3), free of the cancellation of 1 - U near 1;
// otherwise -ln(e), e = 1 - U = (2^32 - hi) 2^-32, or, in the far tail, e
// from all 53 bits, (2^32 - hi) 2^21 - lo / 2^11 in units of 2^-53, so that
// the radius follows the FP64 model's uniform there; ln(e) by the operations
// of series_log (e is a normal float <= 1).  Both ranges share one division
// and one Horner chain: the second range takes its two highest coefficients
// as zero, which leaves every rounding of its shorter series unchanged, and
// its exponent term is zero in the first range (adding +0 changes nothing),
// so a warp whose lanes fall in both ranges runs the series once.
template <class LoOf>
__device__ __forceinline__ float neg_log1m(uint32_t hi, LoOf lo_of) {
  const bool low = hi < 0x80000000u;
  float num, den;
  int ex = 0;
  if (low) {
    const float U = word_to_float(hi) * 0x1p-32f;
    num = U;
    den = 2.0f - U;
  } else {
    float e;
    if (hi < 0xFFF00000u) {
      e = comp_word_to_float(hi) * 0x1p-32f;
    } else {
      const uint32_t lo = lo_of();
      const unsigned long long q =
          ((unsigned long long)(0u - hi) << 21) - (unsigned long long)(lo >> 11);
      e = u63_to_float(q) * 0x1p-53f;
    }
    const uint32_t b = __float_as_uint(e);
    ex = (int)((b >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
    if (m > 1.41421354f) {
      m = m * 0.5f;
      ex += 1;
    }
    num = m - 1.0f;
    den = m + 1.0f;
  }
  const float t = num / den;
  const float t2 = t * t;
  const float l3 = (float)(1.0 / 3.0), l5 = (float)(1.0 / 5.0), l7 = (float)(1.0 / 7.0);
  const float l9 = (float)(1.0 / 9.0), l11 = (float)(1.0 / 11.0);
  const float l13 = low ? (float)(1.0 / 13.0) : 0.0f, l15 = low ? (float)(1.0 / 15.0) : 0.0f;
  const float series =
      1.0f + t2 * (l3 + t2 * (l5 + t2 * (l7 + t2 * (l9 + t2 * (l11 + t2 * (l13 + t2 * l15))))));
  const float ln2 = (float)0.69314718055994530942;
  const float r = (ex >= 0 ? small_to_float(ex) : -small_to_float(-ex)) * ln2 + (2.0f * t) * series;
  return low ? r : -r;
}

__device__ __forceinline__ void axis_of(const BoxDev& B, unsigned long long t, uint32_t cell,
                                        float n[3]) {
  const uint4 w = draw(B, PURPOSE_ROT, cell, 0u, t);
  const float z = centred_word_half_to_float(w.x) * 0x1p-31f;
  // sqrt(1 - z^2) = 2 sqrt(u (1 - u)), u (1 - u) 2^64 = w (2^32 - w) exact in 64 bits
  const unsigned long long q = (unsigned long long)w.x * (unsigned long long)(0u - w.x);
  const float r = 2.0f * sqrtf(u63_to_float(q) * 0x1p-64f);
  float c, s;
  turn_cos_sin(w.y, c, s);
  n[0] = r * c;
  n[1] = r * s;
  n[2] = z;
}

// Exact conversions to double on the integer pipe (the FP64 pipe of GB300
// runs at about 1/64 of the FP32 rate and also executes the conversion
// instructions): a float, and an integer 0 <= q < 2^53.  Other inputs (zero,
// subnormal or non-finite floats; other integers) take the hardware
// conversion, which gives the same value.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)f;
  const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ double ll2d_exact(long long q) {
  if (q <= 0 || q >= (1LL << 53)) return __ll2double_rn(q);
  const int lz = __clzll(q);  // the top bit of q at 63 - lz <= 52
  const unsigned long long m = (unsigned long long)q << (lz - 11);
  return __longlong_as_double((long long)(((unsigned long long)(1022 + 63 - lz) << 52) + m));
}

// FP64 model: u = w.x 2^-32, z = 2u - 1, sqrt(1 - z^2) = 2 sqrt(u (1 - u)) and
// phi = 2 pi w.y 2^-32, with the words converted on the integer pipe and
// (sin phi, cos phi) from one sincospi of phi / pi = w.y 2^-31 (exact).
__device__ __forceinline__ void axis_of(const BoxDev& B, unsigned long long t, uint32_t cell,
                                        double n[3]) {
  const uint4 w = draw(B, PURPOSE_ROT, cell, 0u, t);
  const double a = ll2d_exact((long long)w.x) * 0x1p-32;
  const double b = ll2d_exact(4294967296LL - (long long)w.x) * 0x1p-32;
  const double z = a - b;
  const double r = 2.0 * sqrt(a * b);
  double sp, cp;
  sincospi(ll2d_exact((long long)w.y) * 0x1p-31, &sp, &cp);
  n[0] = r * cp;
  n[1] = r * sp;
  n[2] = z;
}

// Mixed model, Eq. (thermo): xi = sqrt(E^/E_k) to double accuracy, rounded to
// float.  H, E: E^ and E_k in double; Hf, Ef: float estimates of them formed
// by float operations from the same exact factors.  y0 = sqrt(Hf / Ef) is
// refined by one Newton step in double, y1 = y0 + (E^ - y0^2 E_k) /
// (2 y0 E_k): the residual by one fused multiply-add (y0^2 is exact in
// double), the step's 1/(2 y0 E_k) in float (its rounding scales a
// correction of relative size 1e-7).  With the factors converted on the
// integer pipe, about eight FP64-pipe instructions per cell in all instead of
// the two dozen of a double division and square root.  E^ = 0 gives xi = 0.
__device__ __forceinline__ float xi_mixed(double H, float Hf, double E, float Ef) {
  const float y0 = sqrtf(__fdiv_rn(Hf, Ef));
  if (!(y0 > 0.0f)) return y0;
  const double yd = f2d_exact(y0);
  const double r = __fma_rn(-__dmul_rn(yd, yd), E, H);
  const float inv = __fdiv_rn(0.5f, __fmul_rn(y0, Ef));
  return __double2float_rn(__fma_rn(r, f2d_exact(inv), yd));
}

// The nearest double (ties to even) of an unsigned 128-bit integer, on the
// integer pipe.
__device__ __forceinline__ double u128_to_double(unsigned __int128 x) {
  const unsigned long long hi = (unsigned long long)(x >> 64), lo = (unsigned long long)x;
  if (hi == 0ull && lo < (1ull << 53)) return ll2d_exact((long long)lo);
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  const int p = 127 - lz;  // the top bit, >= 53 here
  const int sh = p - 52;
  unsigned __int128 m = x >> sh;
  const unsigned __int128 rem = x & (((unsigned __int128)1 << sh) - 1);
  const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
  if (rem > half || (rem == half && (m & 1))) m += 1;
  int e = p;
  if (m >> 53) {
    m >>= 1;
    e += 1;
  }
  return __longlong_as_double((long long)(((unsigned long long)(e + 1023) << 52) |
                                          ((unsigned long long)m & ((1ull << 52) - 1ull))));
}

// Mixed model, Eq. (thermo) with the one pass of Sec. 3.5 (momentum, mass and
// kinetic energy together): E_k = K - |P|^2 / (2 Mt) from the cell's exact
// sums, returned times the cell mass Mt (also returned).  Solvent only (ns
// members, momentum sums Q of V = rne(v 2^32), second moment S2 = sum V^2):
// E_k Mt = (m^2 / 2) 2^-64 (ns S2 - |Q|^2), the integer exact (>= 0 by
// Cauchy-Schwarz) and rounded once.  With beads or virtual particles
// (momentum sums X of rne(m v 2^32), kinetic sums Kx of rne(m |v|^2 2^32)):
// K = m S2 2^-64 + Kx 2^-32, P = (m Q + X) 2^-32, E_k Mt = (Mt K - |P|^2) / 2
// in double.
__device__ __forceinline__ double mixed_ek_mt(const BoxDev& B, int ns, int nbd, int nv,
                                              const long long Q[3], __int128 S2,
                                              const long long X[3], long long Kx, double& Mt) {
  const double m = B.m;
  if (nbd == 0 && nv == 0) {
    const __int128 D = (__int128)ns * S2 - ((__int128)Q[0] * Q[0] + (__int128)Q[1] * Q[1] +
                                            (__int128)Q[2] * Q[2]);
    Mt = m * ll2d_exact(ns);
    return B.hm2 * u128_to_double((unsigned __int128)D);
  }
  Mt = (m * ll2d_exact(ns) + B.Mb * ll2d_exact(nbd)) + m * ll2d_exact(nv);
  const double K = ((m * u128_to_double((unsigned __int128)S2)) * 0x1p-64) + ll2d_exact(Kx) * 0x1p-32;
  double P2 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double P = (m * ll2d_exact(Q[k]) + ll2d_exact(X[k])) * 0x1p-32;
    P2 = P2 + P * P;
  }
  return 0.5 * (Mt * K - P2);
}

// ---------------------------------------------------------------------------
// Eq. (thermo) / Sec. 3.6: E^ ~ Gamma(3(Nc-1)/2, kT) by Marsaglia-Tsang with a
// Box-Muller normal and the squeeze U3 < 1 - 0.0331 x^4 (inside the acceptance
// region, so it accepts without logarithms).  Attempt j reads Philox block
// A = counter (cell, 1 + 2j): words 0, 2, 1 are the high words of U1, U2, U3;
// their low words are in block B = (cell, 2 + 2j).  gamma_draw_mixed, the
// mixed model's sampler, decides every acceptance in float with the series
// above (block B only for the far tail of the radius, see neg_log1m) and
// returns the accepted d and v (E^ = d v kT); gamma_draw is the FP64 sampler.
// Both return false after 64 rejections.
// ---------------------------------------------------------------------------
__device__ inline bool gamma_draw_mixed(const BoxDev& B, unsigned long long t, uint32_t cell,
                                        int nc, float& dout, float& vout) {
  const float kk = 1.5f * small_to_float(nc - 1);
  const float d = kk - 1.0f / 3.0f;
  const float c = 1.0f / sqrtf(9.0f * d);
  for (uint32_t j = 0; j < 64u; ++j) {
    const uint4 wa = draw(B, PURPOSE_THERMO, cell, 1u + 2u * j, t);
    const float U3 = word_to_float(wa.y) * 0x1p-32f;
    float c2, s2;
    turn_cos_sin(wa.z, c2, s2);
    const float L = neg_log1m(wa.x, [&] { return draw(B, PURPOSE_THERMO, cell, 2u + 2u * j, t).x; });
    const float x = sqrtf(2.0f * L) * c2;
    const float t1 = 1.0f + c * x;
    if (!(t1 > 0.0f)) continue;
    const float v = t1 * t1 * t1;
    const float x2 = x * x;
    bool accept = U3 < 1.0f - 0.0331f * (x2 * x2);
    if (!accept) accept = series_log(U3) < 0.5f * x2 + d - d * v + d * series_log(v);
    if (accept) {
      dout = d;
      vout = v;
      return true;
    }
  }
  return false;
}

// Mixed model: the thermostat factor of a cell with E_k Mt = Ep and mass Mt
// (mixed_ek_mt), Eq. thermo, from the sampler's accepted pair (d, v),
// E^ = d v kT; d < 0 marks a sampler that gave up.  xi is left at 1 when
// E_k = 0; false if E_k > 0 and there is no draw.
__device__ __forceinline__ bool thermo_xi_from_draw(const BoxDev& B, float d, float v, double Ep,
                                                    double Mt, float& xi) {
  if (!(Ep > 0.0)) return true;
  if (d < 0.0f) return false;
  const double H = ((f2d_exact(d) * f2d_exact(v)) * B.kT) * Mt;
  xi = xi_mixed(H, __double2float_rn(H), Ep, __double2float_rn(Ep));
  return true;
}

__device__ inline bool gamma_draw(const BoxDev& B, unsigned long long t, uint32_t cell, int nc,
                                  double& ehat) {
  const double kk = 1.5 * (double)(nc - 1);
  const double d = kk - 1.0 / 3.0;
  const double c = 1.0 / sqrt(9.0 * d);
  for (uint32_t j = 0; j < 64u; ++j) {
    const uint4 wa = draw(B, PURPOSE_THERMO, cell, 1u + 2u * j, t);
    const uint4 wb = draw(B, PURPOSE_THERMO, cell, 2u + 2u * j, t);
    const double U1 = unit53(wa.x, wb.x), U2 = unit53(wa.z, wb.z), U3 = unit53(wa.y, wb.y);
    const double x = sqrt(-2.0 * log(1.0 - U1)) * cospi(2.0 * U2);  // cos(2 pi U2)
    const double t1 = 1.0 + c * x;
    if (!(t1 > 0.0)) continue;
    const double v = t1 * t1 * t1;
    const double x2 = x * x;
    if (U3 < 1.0 - 0.0331 * (x2 * x2) || log(U3) < 0.5 * x2 + d - d * v + d * log(v)) {
      ehat = d * v * B.kT;
      return true;
    }
  }
  return false;
}

// ---------------------------------------------------------------------------
// Eq. (at) / Sec. 3.7: Gaussian random velocity of one particle for the
// Andersen-thermostat rule, keyed by (seed, step, tag, kind); kind 0 is the
// solvent, 1 the solute beads.  Box-Muller on Philox block A = counter
// (tag, 2 kind): words (0, 1) give components 0 and 1 (cos and sin
// branches), words (2, 3) component 2 (cos).  The float version stays in
// float with the mixed model's series (block B = (tag, 2 kind + 1) only for
// the far tail of a radius, see neg_log1m); the FP64 version takes the low
// words of its 53-bit uniforms from block B.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void at_draw(const BoxDev& B, unsigned long long t, uint32_t tag,
                                        uint32_t kind, float sigma, float dv[3]) {
  const uint4 w = draw(B, PURPOSE_AT, tag, 2u * kind, t);
  const float r1 =
      sqrtf(2.0f * neg_log1m(w.x, [&] { return draw(B, PURPOSE_AT, tag, 2u * kind + 1u, t).x; }));
  const float r2 =
      sqrtf(2.0f * neg_log1m(w.z, [&] { return draw(B, PURPOSE_AT, tag, 2u * kind + 1u, t).z; }));
  float c1, s1, c2, s2;
  turn_cos_sin(w.y, c1, s1);
  turn_cos_sin(w.w, c2, s2);
  dv[0] = sigma * (r1 * c1);
  dv[1] = sigma * (r1 * s1);
  dv[2] = sigma * (r2 * c2);
}

__device__ __forceinline__ void at_draw(const BoxDev& B, unsigned long long t, uint32_t tag,
                                        uint32_t kind, double sigma, double dv[3]) {
  const uint4 wa = draw(B, PURPOSE_AT, tag, 2u * kind, t);
  const uint4 wb = draw(B, PURPOSE_AT, tag, 2u * kind + 1u, t);
  const double U1 = unit53(wa.x, wb.x), U2 = unit53(wa.y, wb.y);
  const double U3 = unit53(wa.z, wb.z), U4 = unit53(wa.w, wb.w);
  const double r1 = sqrt(-2.0 * log(1.0 - U1)), r2 = sqrt(-2.0 * log(1.0 - U3));
  double s1, c1;
  sincospi(2.0 * U2, &s1, &c1);  // angle 2 pi U2 (2 U2 exact): no argument reduction
  dv[0] = sigma * (r1 * c1);
  dv[1] = sigma * (r1 * s1);
  dv[2] = sigma * (r2 * cospi(2.0 * U4));
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
    vv[k] = B.sigma_virt * (sqrt(-2.0 * log(1.0 - U)) * cospi(2.0 * U2));
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
  __int128 s2 = 0;  // sum of V^2, V = rne(v 2^32), over members and components
  long long kx = 0;  // extras: sum of rne(m |v|^2 2^32)
  int ns = 0, nb = 0, nv = 0;
  __device__ __forceinline__ void add_solvent(const BoxDev&, const float v[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const long long V = fix32_rne(v[k]);
      q[k] += V;
      s2 += (__int128)V * V;
    }
    ns += 1;
  }
  __device__ __forceinline__ void add_extra(double mass, const double v[3], bool bead) {
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] += __double2ll_rn((mass * v[k]) * 4294967296.0);
    kx += __double2ll_rn((mass * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])) * 4294967296.0);
    if (bead) nb += 1;
    else nv += 1;
  }
  __device__ __forceinline__ void merge(const CellAcc& o) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      q[k] += o.q[k];
      x[k] += o.x[k];
    }
    s2 += o.s2;
    kx += o.kx;
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
  // E_k times the cell mass, and the mass (the thermostat factor is FP64)
  __device__ __forceinline__ double ek_mt(const BoxDev& B, double& Mt) const {
    return mixed_ek_mt(B, ns, nb, nv, q, s2, x, kx, Mt);
  }
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

// Two halves of the per-cell work once the solvent sums are in `a`.
// cell_mean: add the beads of the cell (`bead_in(j, b)` enumerates the bead
// group) and, with walls, the virtual particles; return u.  cell_finish:
// with the thermostat add the beads' and virtual particles' energies about u
// (the solvent's energy is already in `a`), draw xi; draw the axis.  `thermo`
// and `extra` are compile-time constants at the call sites.
template <bool MIXED, class BeadIn>
__device__ __forceinline__ void cell_mean(const BoxDev& B, unsigned long long t, uint32_t cell,
                                          double sz, CellAcc<MIXED>& a, int nbt, BeadIn bead_in,
                                          bool extra, real_t<MIXED> u[3]) {
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
  a.mean_velocity(B, u, extra);
}

template <bool MIXED, class BeadIn>
__device__ __forceinline__ void cell_finish(const BoxDev& B, unsigned long long t, uint32_t cell,
                                            CellAcc<MIXED>& a, const real_t<MIXED> u[3], int nbt,
                                            BeadIn bead_in, bool thermo, bool extra,
                                            CellParams<real_t<MIXED>>& out, int* err) {
  using T = real_t<MIXED>;
  T n[3];
  axis_of(B, t, cell, n);
  T xi = (T)1;
  if (thermo) {
    if constexpr (!MIXED) {  // the FP64 model's energy about u of the extras
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
    }
    // Eq. thermo: xi = sqrt(E^ / E_k), in FP64 in both models (the mixed
    // model rounds it to the float that scales its relative velocities)
    const int nc = a.ns + a.nb + a.nv;
    if (nc >= 2) {
      if constexpr (MIXED) {
        double Mt;
        const double Ep = a.ek_mt(B, Mt);
        float d = -1.0f, v = 0.0f;
        if (Ep > 0.0 && !gamma_draw_mixed(B, t, cell, nc, d, v)) d = -1.0f;
        if (!thermo_xi_from_draw(B, d, v, Ep, Mt, xi)) atomicOr(err, ERR_GAMMA_CAP);
      } else {
        const double Ek = a.energy(B, extra);
        double ehat;
        if (Ek > 0.0) {
          if (gamma_draw(B, t, cell, nc, ehat)) xi = sqrt(ehat / Ek);
          else atomicOr(err, ERR_GAMMA_CAP);
        }
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


}  // namespace mpcd
