/*
 * mpcd_oracle.c -- plain CPU oracle for the SRD step (test infrastructure).
 *
 * Written for a reader holding the paper (arXiv:1801.10187) beside it: every
 * stage is a straight loop over particles or cells, in the paper's order
 * (Sec. 3, step flow: stream, bin, cell properties, collide).  No sorting, no
 * blocking, no fusion.  Compiled with -O2 -ffp-contract=off so that no
 * multiply-add is fused except where fma()/fmaf() is written out.
 *
 * Only the test suite, the smoke check and the benchmark's CPU baseline use
 * this file; the GPU path shares no code with it.
 */
#include "mpcd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC11:  */
/* "Parallel random numbers: as easy as 1, 2, 3").  Ten rounds; each round   */
/* multiplies counter words 0 and 2 by two fixed odd constants, mixes the    */
/* high halves with the other words and the key; the key advances by two     */
/* Weyl constants between rounds.  The paper (Sec. 3.6) uses a hash-based    */
/* generator seeded by (cell, timestep, seed); Philox plays that role here.  */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u; /* golden-ratio Weyl increment */
      k1 += 0xBB67AE85u; /* sqrt(3)-1 Weyl increment    */
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One draw: counter (c0, c1, t_lo, t_hi), key (seed_lo, seed_hi ^ purpose). */
static void draw4(uint64_t seed, uint32_t purpose, uint32_t c0, uint32_t c1, uint64_t t,
                  uint32_t w[4]) {
  uint32_t ctr[4] = {c0, c1, (uint32_t)t, (uint32_t)(t >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ purpose};
  oracle_philox4x32_10(ctr, key, w);
}

/* Uniform double in [0,1): top 53 bits of the 64-bit word (hi, lo). */
static double u01_53(uint32_t hi, uint32_t lo) {
  uint64_t x = ((uint64_t)hi << 32) | (uint64_t)lo;
  return (double)(x >> 11) * 0x1p-53;
}

static const double TWO_PI = 6.283185307179586;

/* ------------------------------------------------------------------------ */
/* Float sin, cos and log used by the mixed model, built from IEEE basic     */
/* operations only so that every platform rounds them identically:           */
/*   sin, cos on [0, pi/4]: Taylor series through x^9 / x^10 (truncation      */
/*   below 2e-9);  log: x = m 2^e with m in [sqrt(1/2), sqrt(2)), then        */
/*   ln m = 2 atanh(t), t = (m-1)/(m+1), series through t^11 (below 1e-9).    */
/* ------------------------------------------------------------------------ */
static void sincos_series_f(float x, float* s, float* c) {
  const float x2 = x * x;
  const float s3 = (float)(-1.0 / 6.0), s5 = (float)(1.0 / 120.0);
  const float s7 = (float)(-1.0 / 5040.0), s9 = (float)(1.0 / 362880.0);
  const float c2 = -0.5f, c4 = (float)(1.0 / 24.0), c6 = (float)(-1.0 / 720.0);
  const float c8 = (float)(1.0 / 40320.0), c10 = (float)(-1.0 / 3628800.0);
  *s = x + x * (x2 * (s3 + x2 * (s5 + x2 * (s7 + x2 * s9))));
  *c = 1.0f + x2 * (c2 + x2 * (c4 + x2 * (c6 + x2 * (c8 + x2 * c10))));
}

/* cos and sin of 2 pi w / 2^32: the top three bits of w give the octant, the
 * other 29 the position inside it; odd octants are measured back from their
 * upper end, so the series argument stays in [0, pi/4] and the octant map is
 * an exact swap / negation. */
static void cos_sin_turn_f(uint32_t w, float* c, float* s) {
  const uint32_t o = w >> 29;
  const uint32_t f = w & 0x1FFFFFFFu;
  const uint32_t g = (o & 1u) ? (0x20000000u - f) : f;
  const float quarter_pi = (float)(3.14159265358979323846 / 4.0);
  const float x = ((float)g * 0x1p-29f) * quarter_pi;
  float sb, cb;
  sincos_series_f(x, &sb, &cb);
  switch (o) {
    case 0: *c = cb; *s = sb; break;
    case 1: *c = sb; *s = cb; break;
    case 2: *c = -sb; *s = cb; break;
    case 3: *c = -cb; *s = sb; break;
    case 4: *c = -cb; *s = -sb; break;
    case 5: *c = -sb; *s = -cb; break;
    case 6: *c = sb; *s = -cb; break;
    default: *c = cb; *s = -sb; break;
  }
}

static float log_series_f(float x) {
  if (!(x > 0.0f)) return x == 0.0f ? -INFINITY : NAN;
  if (isinf(x)) return x;
  int e = 0;
  uint32_t b;
  memcpy(&b, &x, 4);
  if ((b >> 23) == 0) { /* subnormal: scale into the normal range */
    x = x * 0x1p23f;
    memcpy(&b, &x, 4);
    e = -23;
  }
  e += (int)((b >> 23) & 0xFFu) - 127;
  uint32_t mb = (b & 0x7FFFFFu) | 0x3F800000u;
  float m;
  memcpy(&m, &mb, 4);
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
  return (float)e * ln2 + (2.0f * t) * series;
}

/* -ln(1 - U) in float, the squared Box-Muller radius over two, for the 53-bit
 * uniform U whose high and low words are hi and lo.  Three ranges, each free
 * of cancellation:
 *   U < 1/2              : 2 atanh(U / (2 - U)) = -ln(1 - U), U = hi 2^-32,
 *                          the atanh series through t^15 (t <= 1/3);
 *   1 - U >= 2^-12       : -ln(e), e = 1 - U = (2^32 - hi) 2^-32;
 *   1 - U < 2^-12        : -ln(e) with e from all 53 bits,
 *                          e = (2^53 - (hi 2^21 + lo / 2^11)) 2^-53,
 *                          so that the radius's far tail is that of the FP64
 *                          model's uniform (32 bits resolve e only to 2^-32). */
static float neg_log1m_f(uint32_t hi, uint32_t lo) {
  if (hi < 0x80000000u) {
    const float U = (float)hi * 0x1p-32f;
    const float t = U / (2.0f - U);
    const float t2 = t * t;
    const float l3 = (float)(1.0 / 3.0), l5 = (float)(1.0 / 5.0), l7 = (float)(1.0 / 7.0);
    const float l9 = (float)(1.0 / 9.0), l11 = (float)(1.0 / 11.0), l13 = (float)(1.0 / 13.0);
    const float l15 = (float)(1.0 / 15.0);
    const float series =
        1.0f + t2 * (l3 + t2 * (l5 + t2 * (l7 + t2 * (l9 + t2 * (l11 + t2 * (l13 + t2 * l15))))));
    return (2.0f * t) * series;
  }
  float e;
  if (hi < 0xFFF00000u) {
    e = (float)(4294967296LL - (int64_t)hi) * 0x1p-32f;
  } else {
    const int64_t q = ((4294967296LL - (int64_t)hi) << 21) - (int64_t)(lo >> 11);
    e = (float)q * 0x1p-53f;
  }
  return -log_series_f(e);
}

static float xi_mixed(double H, float Hf, double E, float Ef);
float oracle_xi_mixed(double ehat, double ek) {
  return xi_mixed(ehat, (float)ehat, ek, (float)ek);
}
void oracle_cos_sin_turn_f(uint32_t w, float* c, float* s) { cos_sin_turn_f(w, c, s); }
float oracle_log_f(float x) { return log_series_f(x); }
float oracle_neg_log1m_f(uint32_t hi, uint32_t lo) { return neg_log1m_f(hi, lo); }

/* ------------------------------------------------------------------------ */
/* Sec. 2 / Sec. 3.4: random grid shift, one vector per step.  Quantised to  */
/* 2^-32 (cell edge a = 1) so that floor(x - s) is exact in double.          */
/* ------------------------------------------------------------------------ */
void oracle_shift(uint64_t seed, uint64_t t, double s[3]) {
  uint32_t w[4];
  draw4(seed, ORACLE_PURPOSE_SHIFT, 0xFFFFFFFFu, 0u, t, w);
  for (int k = 0; k < 3; ++k) {
    int64_t S = (int64_t)w[k] - (int64_t)2147483648LL;
    s[k] = (double)S * 0x1p-32;
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.6: rotation axis uniform on the unit sphere by cylindrical          */
/* projection: z uniform in [-1,1), phi uniform in [0, 2 pi).                 */
/* ------------------------------------------------------------------------ */
void oracle_axis(uint64_t seed, uint64_t t, uint32_t cell, int32_t precision, double n[3]) {
  uint32_t w[4];
  draw4(seed, ORACLE_PURPOSE_ROT, cell, 0u, t, w);
  /* z = 2u - 1 and sqrt(1 - z^2) = 2 sqrt(u (1 - u)) with u = w0 / 2^32, so
   * that 1 - u is exact and the pole region keeps full relative precision.
   * The mixed model takes u (1 - u) 2^64 = w0 (2^32 - w0) as an exact 64-bit
   * integer product, rounded once to float. */
  if (precision == ORACLE_MIXED) {
    float z = (float)(2LL * (int64_t)w[0] - 4294967296LL) * 0x1p-32f;
    uint64_t q = (uint64_t)w[0] * (uint64_t)(4294967296ULL - (uint64_t)w[0]);
    float r = 2.0f * sqrtf((float)q * 0x1p-64f);
    float cphi, sphi;
    cos_sin_turn_f(w[1], &cphi, &sphi);
    n[0] = (double)(r * cphi);
    n[1] = (double)(r * sphi);
    n[2] = (double)z;
  } else {
    double a = (double)w[0] * 0x1p-32;
    double b = (double)(4294967296LL - (int64_t)w[0]) * 0x1p-32;
    double z = a - b;
    double r = 2.0 * sqrt(a * b);
    double phi = TWO_PI * ((double)w[1] * 0x1p-32);
    n[0] = r * cos(phi);
    n[1] = r * sin(phi);
    n[2] = z;
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2 Eq. (thermo) and Sec. 3.6: kinetic energy of a cell relative to    */
/* its centre of mass drawn from the Maxwell-Boltzmann distribution for      */
/* 3(Nc-1) degrees of freedom, i.e. Gamma(shape 3(Nc-1)/2, scale kT), by     */
/* Marsaglia & Tsang (2000) with a Box-Muller normal (cosine branch).        */
/* Attempt j uses counters (cell, 1+2j) and (cell, 2+2j).                     */
/* ------------------------------------------------------------------------ */
/* The mixed model's attempt loop: the accepted Marsaglia-Tsang pair (d, v),
 * E^ = d v kT.  Returns 0, or -4 after 64 rejections. */
static int32_t gamma_mixed_dv(uint64_t seed, uint64_t t, uint32_t cell, int32_t nc, float* dout,
                              float* vout) {
  {
    float kk = 1.5f * (float)(nc - 1);
    float d = kk - 1.0f / 3.0f;
    float c = 1.0f / sqrtf(9.0f * d);
    for (uint32_t j = 0; j < 64; ++j) {
      /* Attempt j: block A = counter (cell, 1 + 2j).  Its words 0, 2 and 1 are
       * the high words of U1, U2 and U3; block B = (cell, 2 + 2j) holds their
       * low words.  The mixed model reads a low word only for the radius's
       * far tail (neg_log1m_f), else block A alone. */
      uint32_t wa[4], wb[4];
      draw4(seed, ORACLE_PURPOSE_THERMO, cell, 1u + 2u * j, t, wa);
      draw4(seed, ORACLE_PURPOSE_THERMO, cell, 2u + 2u * j, t, wb);
      float U3 = (float)wa[1] * 0x1p-32f;
      float c2, s2;
      cos_sin_turn_f(wa[2], &c2, &s2);
      float x = sqrtf(2.0f * neg_log1m_f(wa[0], wb[0])) * c2;
      float t1 = 1.0f + c * x;
      if (!(t1 > 0.0f)) continue;
      float v = t1 * t1 * t1;
      /* Squeeze of Marsaglia and Tsang (2000): U3 < 1 - 0.0331 x^4 lies inside
       * the acceptance region, so it accepts without the logarithms. */
      float x2 = x * x;
      if (U3 < 1.0f - 0.0331f * (x2 * x2)) {
        *dout = d;
        *vout = v;
        return 0;
      }
      float lhs = log_series_f(U3);
      float rhs = 0.5f * x2 + d - d * v + d * log_series_f(v);
      int accept = lhs < rhs;
      if (accept) {
        *dout = d;
        *vout = v;
        return 0;
      }
    }
    return -4;
  }
}

int32_t oracle_gamma_draw(uint64_t seed, uint64_t t, uint32_t cell, int32_t nc, double kT,
                          int32_t precision, double* ehat) {
  if (nc < 2) return -1;
  if (precision == ORACLE_MIXED) {
    float d, v;
    int32_t st = gamma_mixed_dv(seed, t, cell, nc, &d, &v);
    if (st == 0) *ehat = ((double)d * (double)v) * kT;
    return st;
  }
  double kk = 1.5 * (double)(nc - 1);
  double d = kk - 1.0 / 3.0;
  double c = 1.0 / sqrt(9.0 * d);
  for (uint32_t j = 0; j < 64; ++j) {
    uint32_t wa[4], wb[4];
    draw4(seed, ORACLE_PURPOSE_THERMO, cell, 1u + 2u * j, t, wa);
    draw4(seed, ORACLE_PURPOSE_THERMO, cell, 2u + 2u * j, t, wb);
    /* 53-bit uniforms: high words from block A (as in the mixed model), low
     * words from block B. */
    double U1 = u01_53(wa[0], wb[0]), U2 = u01_53(wa[2], wb[2]), U3 = u01_53(wa[1], wb[1]);
    double x = sqrt(-2.0 * log(1.0 - U1)) * cos(TWO_PI * U2);
    double t1 = 1.0 + c * x;
    if (!(t1 > 0.0)) continue;
    double v = t1 * t1 * t1;
    double x2 = x * x;
    if (U3 < 1.0 - 0.0331 * (x2 * x2) || log(U3) < 0.5 * x2 + d - d * v + d * log(v)) {
      *ehat = d * v * kT;
      return 0;
    }
  }
  return -4;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2, Eq. (at) and Sec. 3.7: the Andersen-thermostat rule draws a       */
/* Gaussian random velocity for every particle by Box-Muller, keyed by the   */
/* step, the particle's tag and the seed.  One Box-Muller pair gives         */
/* components 0 and 1 (cos and sin branches), a second pair's cos branch    */
/* component 2.                                                             */
/* ------------------------------------------------------------------------ */
void oracle_at_draw(uint64_t seed, uint64_t t, uint32_t tag, int32_t kind, double sigma,
                    int32_t precision, double dv[3]) {
  uint32_t wa[4];
  draw4(seed, ORACLE_PURPOSE_AT, tag, 2u * (uint32_t)kind, t, wa);
  uint32_t wb[4];
  draw4(seed, ORACLE_PURPOSE_AT, tag, 2u * (uint32_t)kind + 1u, t, wb);
  if (precision == ORACLE_MIXED) {
    /* radii from the high words (block B's low words only in the far tail) */
    float r1 = sqrtf(2.0f * neg_log1m_f(wa[0], wb[0]));
    float r2 = sqrtf(2.0f * neg_log1m_f(wa[2], wb[2]));
    float c1, s1, c2, s2;
    cos_sin_turn_f(wa[1], &c1, &s1);
    cos_sin_turn_f(wa[3], &c2, &s2);
    float sg = (float)sigma;
    dv[0] = (double)(sg * (r1 * c1));
    dv[1] = (double)(sg * (r1 * s1));
    dv[2] = (double)(sg * (r2 * c2));
    return;
  }
  double U1 = u01_53(wa[0], wb[0]), U2 = u01_53(wa[1], wb[1]);
  double U3 = u01_53(wa[2], wb[2]), U4 = u01_53(wa[3], wb[3]);
  double r1 = sqrt(-2.0 * log(1.0 - U1)), r2 = sqrt(-2.0 * log(1.0 - U3));
  dv[0] = sigma * (r1 * cos(TWO_PI * U2));
  dv[1] = sigma * (r1 * sin(TWO_PI * U2));
  dv[2] = sigma * (r2 * cos(TWO_PI * U4));
}

/* ------------------------------------------------------------------------ */
/* Geometry helpers                                                          */
/* ------------------------------------------------------------------------ */
int64_t oracle_num_cells(const oracle_params* p) {
  int64_t nz = p->n[2] + (p->walls_z ? 2 : 0);
  return (int64_t)p->n[0] * (int64_t)p->n[1] * nz;
}

/* Periodic wrap into [0, L). */
static double wrap_d(double x, double L) {
  if (x >= L) x -= L;
  else if (x < 0.0) x += L;
  if (!(x >= 0.0 && x < L)) {
    x = x - L * floor(x / L);
    if (!(x >= 0.0 && x < L)) x = 0.0;
  }
  return x;
}
static float wrap_f(float x, float L) {
  if (x >= L) x -= L;
  else if (x < 0.0f) x += L;
  if (!(x >= 0.0f && x < L)) {
    x = x - L * floorf(x / L);
    if (!(x >= 0.0f && x < L)) x = 0.0f;
  }
  return x;
}

/* Sec. 3.4: cell of a position under grid shift s.  floor(x - s) is exact
 * here (s is a multiple of 2^-32, |s| < 1/2), then periodic wrap of the cell
 * coordinate; with walls the z layer index is floor(z - s_z) + 1 in
 * [0, n_z + 1].  Cells are numbered x fastest. */
static int32_t cell_of(const oracle_params* p, const double s[3], double x, double y, double z) {
  int64_t c[3];
  double r[3] = {x, y, z};
  for (int k = 0; k < 3; ++k) {
    int64_t i = (int64_t)floor(r[k] - s[k]);
    if (k == 2 && p->walls_z) {
      i += 1;
      if (i < 0) i = 0;
      if (i > p->n[2] + 1) i = p->n[2] + 1;
    } else {
      int64_t n = p->n[k];
      i = ((i % n) + n) % n;
    }
    c[k] = i;
  }
  return (int32_t)(c[0] + (int64_t)p->n[0] * (c[1] + (int64_t)p->n[1] * c[2]));
}

/* ------------------------------------------------------------------------ */
/* Sec. 2 Eq. (stream): ballistic streaming over dt.  With a body force g   */
/* the motion is the constant-acceleration parabola.  With walls at z = 0    */
/* and z = H the particle is moved to the wall at the hit time, its whole    */
/* velocity reversed (no-slip bounce-back), and the remaining time streamed. */
/* ------------------------------------------------------------------------ */
static void stream_d(const oracle_params* p, double* r, double* v) {
  const double dt = p->dt;
  double L[3] = {(double)p->n[0], (double)p->n[1], (double)p->n[2]};
  if (p->walls_z) {
    double H = L[2];
    double zn = fma(v[2], dt, r[2]);
    if (!(zn >= 0.0 && zn < H)) {
      double wall = (zn < 0.0) ? 0.0 : H;
      double tau = (wall - r[2]) / v[2];
      if (!(tau >= 0.0)) tau = 0.0;
      if (tau > dt) tau = dt;
      for (int k = 0; k < 2; ++k) {
        r[k] = fma(v[k], tau, r[k]) + ((0.5 * p->g[k]) * tau) * tau;
        v[k] = v[k] + p->g[k] * tau;
      }
      for (int k = 0; k < 3; ++k) v[k] = -v[k];
      double rem = dt - tau;
      for (int k = 0; k < 2; ++k) {
        r[k] = fma(v[k], rem, r[k]) + ((0.5 * p->g[k]) * rem) * rem;
        v[k] = v[k] + p->g[k] * rem;
      }
      double z = fma(v[2], rem, wall);
      if (z < 0.0) z = 0.0;
      if (z >= H) z = nextafter(H, 0.0);
      r[2] = z;
      for (int k = 0; k < 2; ++k) r[k] = wrap_d(r[k], L[k]);
      return;
    }
  }
  for (int k = 0; k < 3; ++k) {
    double hg = ((0.5 * p->g[k]) * dt) * dt;
    r[k] = fma(v[k], dt, r[k]) + hg;
    v[k] = v[k] + p->g[k] * dt;
    if (!(k == 2 && p->walls_z)) r[k] = wrap_d(r[k], L[k]);
  }
}

/* The same streaming rule with every operation rounded to float. */
static void stream_f(const oracle_params* p, float* r, float* v) {
  const float dt = (float)p->dt;
  float L[3] = {(float)p->n[0], (float)p->n[1], (float)p->n[2]};
  float g[3] = {(float)p->g[0], (float)p->g[1], (float)p->g[2]};
  if (p->walls_z) {
    float H = L[2];
    float zn = fmaf(v[2], dt, r[2]);
    if (!(zn >= 0.0f && zn < H)) {
      float wall = (zn < 0.0f) ? 0.0f : H;
      float tau = (wall - r[2]) / v[2];
      if (!(tau >= 0.0f)) tau = 0.0f;
      if (tau > dt) tau = dt;
      for (int k = 0; k < 2; ++k) {
        r[k] = fmaf(v[k], tau, r[k]) + ((0.5f * g[k]) * tau) * tau;
        v[k] = v[k] + g[k] * tau;
      }
      for (int k = 0; k < 3; ++k) v[k] = -v[k];
      float rem = dt - tau;
      for (int k = 0; k < 2; ++k) {
        r[k] = fmaf(v[k], rem, r[k]) + ((0.5f * g[k]) * rem) * rem;
        v[k] = v[k] + g[k] * rem;
      }
      float z = fmaf(v[2], rem, wall);
      if (z < 0.0f) z = 0.0f;
      if (z >= H) z = nextafterf(H, 0.0f);
      r[2] = z;
      for (int k = 0; k < 2; ++k) r[k] = wrap_f(r[k], L[k]);
      return;
    }
  }
  for (int k = 0; k < 3; ++k) {
    float hg = (float)(((0.5 * p->g[k]) * p->dt) * p->dt);
    float gdt = (float)(p->g[k] * p->dt);
    r[k] = fmaf(v[k], dt, r[k]) + hg;
    v[k] = v[k] + gdt;
    if (!(k == 2 && p->walls_z)) r[k] = wrap_f(r[k], L[k]);
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2 (solute) / Sec. 3.6: beads between collisions follow velocity      */
/* Verlet with harmonic bonds U = k/2 (r - r0)^2 along each linear chain.    */
/* ------------------------------------------------------------------------ */
static void bond_forces(const oracle_params* p, int64_t nb, const double* r, double* F) {
  double L[3] = {(double)p->n[0], (double)p->n[1], (double)p->n[2]};
  int64_t cl = p->chain_len;
  for (int64_t i = 0; i < nb; ++i) {
    double f3[3] = {0.0, 0.0, 0.0};
    int64_t b = i % cl;
    for (int side = 0; side < 2; ++side) {
      int64_t j;
      if (side == 0) { if (b == 0) continue; j = i - 1; }
      else { if (b == cl - 1) continue; j = i + 1; }
      double d[3];
      for (int k = 0; k < 3; ++k) {
        d[k] = r[3 * j + k] - r[3 * i + k];
        d[k] = d[k] - L[k] * nearbyint(d[k] / L[k]); /* minimum image */
      }
      double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (!(dist > 0.0)) continue;
      double f = (p->bond_k * (dist - p->bond_r0)) / dist;
      for (int k = 0; k < 3; ++k) f3[k] += f * d[k];
    }
    for (int k = 0; k < 3; ++k) F[3 * i + k] = f3[k];
  }
}

/* Non-bonded solute forces (Sec. 4.3 uses a bead-spring model with
 * non-bonded pair forces from a neighbour list; the potential is only cited).
 * Reading: the Weeks-Chandler-Andersen repulsion between every pair of beads,
 * U(r) = 4 eps ((sigma/r)^12 - (sigma/r)^6) + eps for r < 2^(1/6) sigma,
 * 0 beyond, minimum-image distances; the force on bead i from j is
 * (24 eps / r^2) (2 (sigma/r)^12 - (sigma/r)^6) (r_i - r_j).  Every pair is
 * visited (no neighbour list here). */
static void pair_forces(const oracle_params* p, int64_t nb, const double* r, double* F) {
  double L[3] = {(double)p->n[0], (double)p->n[1], (double)p->n[2]};
  double eps = p->lj_epsilon, s2 = p->lj_sigma * p->lj_sigma;
  double rc2 = pow(2.0, 1.0 / 3.0) * s2;
  for (int64_t i = 0; i < nb; ++i) {
    for (int64_t j = 0; j < nb; ++j) {
      if (j == i) continue;
      double d[3];
      for (int k = 0; k < 3; ++k) {
        d[k] = r[3 * j + k] - r[3 * i + k];
        d[k] = d[k] - L[k] * nearbyint(d[k] / L[k]);
      }
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (!(r2 < rc2)) continue;
      double q = s2 / r2;
      double q6 = q * q * q;
      double g = 24.0 * eps * q6 * (2.0 * q6 - 1.0) / r2;
      for (int k = 0; k < 3; ++k) F[3 * i + k] -= g * d[k];
    }
  }
}

static void solute_forces(const oracle_params* p, int64_t nb, const double* r, double* F) {
  bond_forces(p, nb, r, F);
  if (p->lj_epsilon > 0.0) pair_forces(p, nb, r, F);
}

/* Potential energy of the solute: harmonic bonds k/2 (r - r0)^2 and, when
 * on, the WCA repulsion of every pair (each pair once). */
double oracle_solute_energy(const oracle_params* p, int64_t nb, const double* r) {
  double L[3] = {(double)p->n[0], (double)p->n[1], (double)p->n[2]};
  int64_t cl = p->chain_len > 0 ? p->chain_len : 1;
  double U = 0.0;
  for (int64_t i = 0; i < nb; ++i) {
    for (int64_t j = i + 1; j < nb; ++j) {
      double d[3];
      for (int k = 0; k < 3; ++k) {
        d[k] = r[3 * j + k] - r[3 * i + k];
        d[k] = d[k] - L[k] * nearbyint(d[k] / L[k]);
      }
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (j == i + 1 && (i % cl) != cl - 1) {
        double x = sqrt(r2) - p->bond_r0;
        U += 0.5 * p->bond_k * x * x;
      }
      if (p->lj_epsilon > 0.0) {
        double s2 = p->lj_sigma * p->lj_sigma;
        if (r2 < pow(2.0, 1.0 / 3.0) * s2) {
          double q6 = pow(s2 / r2, 3.0);
          U += 4.0 * p->lj_epsilon * (q6 * q6 - q6) + p->lj_epsilon;
        }
      }
    }
  }
  return U;
}

void oracle_solute_forces(const oracle_params* p, int64_t nb, const double* r, double* F) {
  solute_forces(p, nb, r, F);
}

static void md_substeps(const oracle_params* p, int64_t nb, double* r, double* v) {
  double L[3] = {(double)p->n[0], (double)p->n[1], (double)p->n[2]};
  double h = p->dt / (double)p->md_substeps;
  double hh = (0.5 * h) / p->solute_mass;
  double* F = (double*)malloc(sizeof(double) * 3 * (size_t)nb);
  solute_forces(p, nb, r, F);
  for (int s = 0; s < p->md_substeps; ++s) {
    for (int64_t i = 0; i < 3 * nb; ++i) v[i] = v[i] + hh * F[i];
    for (int64_t i = 0; i < nb; ++i)
      for (int k = 0; k < 3; ++k) r[3 * i + k] = wrap_d(r[3 * i + k] + h * v[3 * i + k], L[k]);
    solute_forces(p, nb, r, F);
    for (int64_t i = 0; i < 3 * nb; ++i) v[i] = v[i] + hh * F[i];
  }
  free(F);
}

/* ------------------------------------------------------------------------ */
/* Walls: virtual particles fill the part of a wall-cut cell that lies       */
/* outside the channel (Lamura et al. 2001): count with mean rho_v * f_out,  */
/* Gaussian velocities of variance kT/m and zero mean.                       */
/* ------------------------------------------------------------------------ */
static double outside_fraction(const oracle_params* p, const double s[3], int64_t cz) {
  double H = (double)p->n[2];
  double lo = (double)(cz - 1) + s[2];
  double hi = lo + 1.0;
  double a = lo > 0.0 ? lo : 0.0;
  double b = hi < H ? hi : H;
  double inside = b - a;
  if (inside < 0.0) inside = 0.0;
  if (inside > 1.0) inside = 1.0;
  return 1.0 - inside;
}

static int32_t virtual_count(const oracle_params* p, uint64_t t, uint32_t cell, double fout) {
  if (!(fout > 0.0) || !(fout < 1.0)) return 0;
  double lam = p->virt_density * fout;
  double fl = floor(lam);
  int32_t nv = (int32_t)fl;
  uint32_t w[4];
  draw4(p->seed, ORACLE_PURPOSE_VIRT, cell, 0u, t, w);
  if (u01_53(w[0], w[1]) < lam - fl) nv += 1;
  return nv;
}

static void virtual_velocity(const oracle_params* p, uint64_t t, uint32_t cell, int32_t q,
                             double vv[3]) {
  double sigma = sqrt(p->kT / p->mass);
  for (int k = 0; k < 3; ++k) {
    uint32_t w[4];
    draw4(p->seed, ORACLE_PURPOSE_VIRT, cell, 1u + 3u * (uint32_t)q + (uint32_t)k, t, w);
    double U = u01_53(w[0], w[1]), U2 = u01_53(w[2], w[3]);
    vv[k] = sigma * (sqrt(-2.0 * log(1.0 - U)) * cos(TWO_PI * U2));
  }
}

/* ------------------------------------------------------------------------ */
/* Angular-momentum conservation (Sec. 2: the rules conserve linear momentum */
/* only; the paper cites Noguchi & Gompper for the constraint that restores  */
/* angular momentum).  After the collision rule, every member of a cell      */
/* receives omega x r_c, where r_c is its position relative to the cell's    */
/* centre of mass and omega solves Pi omega = dL with                        */
/* dL = sum m r_c x (v - v') (v before, v' after the rule) and the inertia    */
/* tensor Pi = sum m (|r_c|^2 I - r_c r_c^T): the cell's angular momentum    */
/* about its centre of mass is then what it was before the collision, and    */
/* its linear momentum is unchanged (sum m r_c = 0).  Positions are taken    */
/* in the frame of the shifted cell (rel_pos, in [0, 1) per axis).  A cell   */
/* of two members (or with all members on a line) has an inertia tensor of  */
/* rank two; there omega = 2 dL / tr(Pi), which solves the system on the    */
/* plane normal to the line (dL has no component along it).  The mixed       */
/* model sums in int64 fixed point (scale 2^32) and solves in float.         */
/* ------------------------------------------------------------------------ */
static double rel_pos(const oracle_params* p, double x, double s, int64_t i, int k) {
  double d = (x - s) - (double)i;
  double L = (double)p->n[k];
  if (d < 0.0) d += L;
  else if (d >= 1.0) d -= L;
  return d;
}

/* The mixed model's relative position, in float: x = fl + f with fl = floor(x)
 * and f exact, i0 = floor(x - s) the unwrapped cell coordinate of the
 * binning (exact), and x - s - i0 = (f - s) + (fl - i0), with s rounded to
 * float and fl - i0 in {-1, 0, 1}. */
static float rel_pos_f(double x, double s) {
  float xf = (float)x;
  float fl = floorf(xf);
  float f = xf - fl;
  double i0 = floor((double)xf - s);
  float adj = (float)((double)fl - i0);
  return (f - (float)s) + adj;
}

static void cell_coords(const oracle_params* p, int32_t c, int64_t ic[3]) {
  int64_t nx = p->n[0], ny = p->n[1];
  ic[0] = c % nx;
  ic[1] = (c / nx) % ny;
  ic[2] = c / (nx * ny);
}

/* omega from Pi omega = dL, Pi = [[a, b, c], [b, d, e], [c, e, f]] (float). */
static void solve_omega_f(int32_t nc, const float P[6], const float dL[3], float w[3]) {
  float a = P[0], b = P[1], c = P[2], d = P[3], e = P[4], f = P[5];
  float A = d * f - e * e, B = c * e - b * f, C = b * e - c * d;
  float D = a * f - c * c, E = b * c - a * e, F = a * d - b * b;
  float det = a * A + b * B + c * C;
  float tr = a + d + f;
  float t3 = tr / 3.0f;
  if (nc >= 3 && det > 1e-6f * (t3 * t3 * t3)) {
    w[0] = (A * dL[0] + B * dL[1] + C * dL[2]) / det;
    w[1] = (B * dL[0] + D * dL[1] + E * dL[2]) / det;
    w[2] = (C * dL[0] + E * dL[1] + F * dL[2]) / det;
  } else if (tr > 0.0f) {
    float g = 2.0f / tr;
    for (int k = 0; k < 3; ++k) w[k] = dL[k] * g;
  } else {
    w[0] = w[1] = w[2] = 0.0f;
  }
}

static void solve_omega_d(int32_t nc, const double P[6], const double dL[3], double w[3]) {
  double a = P[0], b = P[1], c = P[2], d = P[3], e = P[4], f = P[5];
  double A = d * f - e * e, B = c * e - b * f, C = b * e - c * d;
  double D = a * f - c * c, E = b * c - a * e, F = a * d - b * b;
  double det = a * A + b * B + c * C;
  double tr = a + d + f;
  double t3 = tr / 3.0;
  if (nc >= 3 && det > 1e-6 * (t3 * t3 * t3)) {
    w[0] = (A * dL[0] + B * dL[1] + C * dL[2]) / det;
    w[1] = (B * dL[0] + D * dL[1] + E * dL[2]) / det;
    w[2] = (C * dL[0] + E * dL[1] + F * dL[2]) / det;
  } else if (tr > 0.0) {
    double g = 2.0 / tr;
    for (int k = 0; k < 3; ++k) w[k] = dL[k] * g;
  } else {
    w[0] = w[1] = w[2] = 0.0;
  }
}

/* v0: velocities before the collision, vel: after it (corrected in place). */
static void angular_correction(const oracle_params* p, int64_t n, const double* pos,
                               const double* v0, double* vel, const int32_t* cellid,
                               const double s[3], int64_t ncells, const int32_t* cnt) {
  const int mixed = (p->precision == ORACLE_MIXED);
  const double m = p->mass;
  const float mf = (float)m;
  int64_t* Q = (int64_t*)calloc((size_t)ncells * 3, sizeof(int64_t));
  int64_t* Lq = (int64_t*)calloc((size_t)ncells * 3, sizeof(int64_t));
  int64_t* Pq = (int64_t*)calloc((size_t)ncells * 6, sizeof(int64_t));
  double* Qd = (double*)calloc((size_t)ncells * 3, sizeof(double));
  double* Ldd = (double*)calloc((size_t)ncells * 3, sizeof(double));
  double* Pdd = (double*)calloc((size_t)ncells * 6, sizeof(double));
  double* rcm = (double*)calloc((size_t)ncells * 3, sizeof(double));
  double* om = (double*)calloc((size_t)ncells * 3, sizeof(double));
  /* positions relative to the shifted cell, one member at a time */
  #define REL(i, r)                                                       \
    do {                                                                  \
      int64_t ic_[3];                                                     \
      cell_coords(p, cellid[i], ic_);                                     \
      for (int k_ = 0; k_ < 3; ++k_)                                      \
        r[k_] = mixed ? (double)rel_pos_f(pos[3 * (i) + k_], s[k_])       \
                      : rel_pos(p, pos[3 * (i) + k_], s[k_], ic_[k_], k_); \
    } while (0)
  /* centre of mass of each cell */
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = cellid[i];
    double r[3];
    REL(i, r);
    for (int k = 0; k < 3; ++k) {
      if (mixed) Q[3 * c + k] += llrint((double)(float)r[k] * 0x1p32);
      else Qd[3 * c + k] += r[k];
    }
  }
  for (int64_t c = 0; c < ncells; ++c) {
    if (cnt[c] == 0) continue;
    for (int k = 0; k < 3; ++k) {
      if (mixed) rcm[3 * c + k] = (double)(((float)Q[3 * c + k] * 0x1p-32f) / (float)cnt[c]);
      else rcm[3 * c + k] = Qd[3 * c + k] / (double)cnt[c];
    }
  }
  /* dL = sum m r_c x (v - v') and the inertia tensor */
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = cellid[i];
    double r[3];
    REL(i, r);
    if (mixed) {
      float rc[3], dv[3], x[3], t[6];
      for (int k = 0; k < 3; ++k) {
        rc[k] = (float)r[k] - (float)rcm[3 * c + k];
        dv[k] = (float)v0[3 * i + k] - (float)vel[3 * i + k];
      }
      x[0] = rc[1] * dv[2] - rc[2] * dv[1];
      x[1] = rc[2] * dv[0] - rc[0] * dv[2];
      x[2] = rc[0] * dv[1] - rc[1] * dv[0];
      t[0] = rc[1] * rc[1] + rc[2] * rc[2];
      t[1] = rc[0] * rc[1];
      t[2] = rc[0] * rc[2];
      t[3] = rc[0] * rc[0] + rc[2] * rc[2];
      t[4] = rc[1] * rc[2];
      t[5] = rc[0] * rc[0] + rc[1] * rc[1];
      for (int k = 0; k < 3; ++k) Lq[3 * c + k] += llrint((double)x[k] * 0x1p32);
      for (int k = 0; k < 6; ++k) Pq[6 * c + k] += llrint((double)t[k] * 0x1p32);
    } else {
      double rc[3], dv[3];
      for (int k = 0; k < 3; ++k) {
        rc[k] = r[k] - rcm[3 * c + k];
        dv[k] = v0[3 * i + k] - vel[3 * i + k];
      }
      Ldd[3 * c + 0] += m * (rc[1] * dv[2] - rc[2] * dv[1]);
      Ldd[3 * c + 1] += m * (rc[2] * dv[0] - rc[0] * dv[2]);
      Ldd[3 * c + 2] += m * (rc[0] * dv[1] - rc[1] * dv[0]);
      Pdd[6 * c + 0] += m * (rc[1] * rc[1] + rc[2] * rc[2]);
      Pdd[6 * c + 1] -= m * (rc[0] * rc[1]);
      Pdd[6 * c + 2] -= m * (rc[0] * rc[2]);
      Pdd[6 * c + 3] += m * (rc[0] * rc[0] + rc[2] * rc[2]);
      Pdd[6 * c + 4] -= m * (rc[1] * rc[2]);
      Pdd[6 * c + 5] += m * (rc[0] * rc[0] + rc[1] * rc[1]);
    }
  }
  /* omega of each cell */
  for (int64_t c = 0; c < ncells; ++c) {
    if (cnt[c] == 0) continue;
    if (mixed) {
      float P[6], dL[3], w[3];
      for (int k = 0; k < 3; ++k) dL[k] = mf * ((float)Lq[3 * c + k] * 0x1p-32f);
      for (int k = 0; k < 6; ++k) {
        float e = mf * ((float)Pq[6 * c + k] * 0x1p-32f);
        P[k] = (k == 1 || k == 2 || k == 4) ? -e : e;
      }
      solve_omega_f(cnt[c], P, dL, w);
      for (int k = 0; k < 3; ++k) om[3 * c + k] = (double)w[k];
    } else {
      solve_omega_d(cnt[c], &Pdd[6 * c], &Ldd[3 * c], &om[3 * c]);
    }
  }
  /* v'' = v' + omega x r_c */
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = cellid[i];
    double r[3];
    REL(i, r);
    if (mixed) {
      float rc[3], w[3];
      for (int k = 0; k < 3; ++k) {
        rc[k] = (float)r[k] - (float)rcm[3 * c + k];
        w[k] = (float)om[3 * c + k];
      }
      float a0 = w[1] * rc[2] - w[2] * rc[1];
      float a1 = w[2] * rc[0] - w[0] * rc[2];
      float a2 = w[0] * rc[1] - w[1] * rc[0];
      vel[3 * i + 0] = (double)((float)vel[3 * i + 0] + a0);
      vel[3 * i + 1] = (double)((float)vel[3 * i + 1] + a1);
      vel[3 * i + 2] = (double)((float)vel[3 * i + 2] + a2);
    } else {
      double rc[3];
      const double* w = &om[3 * c];
      for (int k = 0; k < 3; ++k) rc[k] = r[k] - rcm[3 * c + k];
      vel[3 * i + 0] += w[1] * rc[2] - w[2] * rc[1];
      vel[3 * i + 1] += w[2] * rc[0] - w[0] * rc[2];
      vel[3 * i + 2] += w[0] * rc[1] - w[1] * rc[0];
    }
  }
  #undef REL
  free(Q); free(Lq); free(Pq); free(Qd); free(Ldd); free(Pdd); free(rcm); free(om);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2 Eq. (srd) written as a Rodrigues rotation of dv about the unit     */
/* axis n by angle alpha:  dv' = dv cos a + (n x dv) sin a + n (n.dv)(1-cos a)*/
/* ------------------------------------------------------------------------ */
static void rotate_d(const double n[3], double ca, double sa, double omc, const double d[3],
                     double out[3]) {
  double nd = fma(n[2], d[2], fma(n[1], d[1], n[0] * d[0]));
  double cr[3] = {fma(n[1], d[2], -(n[2] * d[1])), fma(n[2], d[0], -(n[0] * d[2])),
                  fma(n[0], d[1], -(n[1] * d[0]))};
  double ndo = nd * omc;
  for (int k = 0; k < 3; ++k) out[k] = fma(n[k], ndo, fma(cr[k], sa, d[k] * ca));
}
static void rotate_f(const float n[3], float ca, float sa, float omc, const float d[3],
                     float out[3]) {
  float nd = fmaf(n[2], d[2], fmaf(n[1], d[1], n[0] * d[0]));
  float cr[3] = {fmaf(n[1], d[2], -(n[2] * d[1])), fmaf(n[2], d[0], -(n[0] * d[2])),
                 fmaf(n[0], d[1], -(n[1] * d[0]))};
  float ndo = nd * omc;
  for (int k = 0; k < 3; ++k) out[k] = fmaf(n[k], ndo, fmaf(cr[k], sa, d[k] * ca));
}

/* Mixed model, Eq. (thermo): xi = sqrt(E^/E_k) to double accuracy, rounded
 * to float.  H, E: E^ and E_k in double; Hf, Ef: their float estimates
 * (formed from the same exact quantities by float operations, see one_step).
 * The float estimate y0 = sqrt(Hf / Ef) (about 1e-7 relative) is refined by
 * one Newton step in double,
 *   y1 = y0 + (E^ - y0^2 E_k) / (2 y0 E_k),
 * the residual by one fused multiply-add (y0^2 is exact in double) and the
 * step's 1/(2 y0 E_k) in float: its rounding scales a correction of relative
 * size 1e-7, so y1 is within a few 1e-14 of the square root.  E^ = 0 (kT = 0)
 * gives xi = 0. */
static float xi_mixed(double H, float Hf, double E, float Ef) {
  const float y0 = sqrtf(Hf / Ef);
  if (!(y0 > 0.0f)) return y0;
  const double r = fma(-((double)y0 * (double)y0), E, H);
  const float inv = 0.5f / (y0 * Ef);
  return (float)fma(r, (double)inv, (double)y0);
}

/* ------------------------------------------------------------------------ */
/* One SRD step (Sec. 3 step flow)                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t* cnt;   /* real members (solvent + beads) */
  int32_t* nsol;  /* solvent members                */
  int32_t* nbead; /* bead members                   */
  int32_t* nvirt; /* virtual particles (walls)      */
  double* M;      /* FP64 mode: mass                */
  double* P;      /* FP64 mode: momentum (3 per cell) */
  double* E;      /* FP64 mode: kinetic energy about u */
  int64_t* Qs;    /* MIXED: solvent sum of rne(v 2^32) (3 per cell) */
  int64_t* Qx;    /* MIXED: beads/virtual sum of rne(m v 2^32) (3 per cell) */
  __int128* S2;   /* MIXED: solvent sum of V^2 over members and components, V = rne(v 2^32) */
  int64_t* Kx;    /* MIXED: beads/virtual sum of rne(m |v|^2 2^32) */
  double* u;      /* centre-of-mass velocity (3 per cell) */
  double* axis;   /* rotation axis (3 per cell) */
  double* xi;     /* thermostat scale factor */
  double* D;      /* FP64, Andersen rule: sum m dv (3 per cell) */
  int64_t* Qd;    /* MIXED, Andersen rule: solvent sum of rne(dv 2^32) */
  int64_t* Qdx;   /* MIXED, Andersen rule: beads sum of rne(M dv 2^32) */
  double* dbar;   /* Andersen rule: mass-weighted mean random velocity (3 per cell) */
} cellbuf;

/* Mixed model, Eq. (thermo) with Sec. 3.5's one pass: E_k = K - |P|^2 / (2 Mt)
 * from the cell's exact sums, returned multiplied by the cell mass Mt (set in
 * *Mt).  A cell of solvent only (n members, momentum sums Q of V = rne(v 2^32),
 * second moment S2 = sum V^2): E_k Mt = (m^2 / 2) 2^-64 (n S2 - |Q|^2), the
 * integer exact (Cauchy-Schwarz keeps it >= 0) and rounded once.  With beads
 * or virtual particles (momentum sums X of rne(m v 2^32), kinetic sums Kx of
 * rne(m |v|^2 2^32)): K = m S2 2^-64 + Kx 2^-32, P = (m Q + X) 2^-32 and
 * E_k Mt = (Mt K - |P|^2) / 2 in double. */
static double mixed_ek_mt(const oracle_params* p, const cellbuf* cb, int64_t c, double hm2,
                          double* Mt) {
  const double m = p->mass;
  const int32_t ns = cb->nsol[c], nbd = cb->nbead[c], nv = cb->nvirt[c];
  const int64_t* Q = &cb->Qs[3 * c];
  if (nbd == 0 && nv == 0) {
    const __int128 D = (__int128)ns * cb->S2[c] -
                       ((__int128)Q[0] * Q[0] + (__int128)Q[1] * Q[1] + (__int128)Q[2] * Q[2]);
    *Mt = m * (double)ns;
    return hm2 * (double)D;
  }
  const int64_t* X = &cb->Qx[3 * c];
  *Mt = (m * (double)ns + p->solute_mass * (double)nbd) + m * (double)nv;
  const double K = ((m * (double)cb->S2[c]) * 0x1p-64) + (double)cb->Kx[c] * 0x1p-32;
  double P2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double P = (m * (double)Q[k] + (double)X[k]) * 0x1p-32;
    P2 = P2 + P * P;
  }
  return 0.5 * (*Mt * K - P2);
}

static int32_t one_step(const oracle_params* p, int64_t n, double* pos, double* vel, int64_t nb,
                        double* spos, double* svel, uint64_t t, int32_t* cellid, cellbuf* cb,
                        int64_t ncells) {
  const int mixed = (p->precision == ORACLE_MIXED);
  /* Float streaming: the mixed model, and the FP64 model of one mixed step
   * (ORACLE_FP64_FSTREAM), which streams the float state as the mixed model
   * does and takes every later stage in double. */
  const int fstream = mixed || (p->precision == ORACLE_FP64_FSTREAM);
  const int32_t arith = mixed ? ORACLE_MIXED : ORACLE_FP64;
  const double m = p->mass, Mb = p->solute_mass;
  const double ca = cos(p->alpha), sa = sin(p->alpha), omc = 1.0 - ca;
  /* mixed model: E_k Mt = hm2 (n S2 - |Q|^2) for a cell of solvent only */
  const double hm2 = ((0.5 * m) * m) * 0x1p-64;
  int32_t status = 0;

  /* Solute: MD substeps between collisions (Sec. 3.6, last paragraph). */
  if (nb > 0) md_substeps(p, nb, spos, svel);

  /* Grid shift for this step. */
  double s[3];
  oracle_shift(p->seed, t, s);

  /* Stream the solvent. */
  for (int64_t i = 0; i < n; ++i) {
    if (fstream) {
      float r[3] = {(float)pos[3 * i], (float)pos[3 * i + 1], (float)pos[3 * i + 2]};
      float v[3] = {(float)vel[3 * i], (float)vel[3 * i + 1], (float)vel[3 * i + 2]};
      stream_f(p, r, v);
      for (int k = 0; k < 3; ++k) { pos[3 * i + k] = r[k]; vel[3 * i + k] = v[k]; }
    } else {
      stream_d(p, &pos[3 * i], &vel[3 * i]);
    }
  }

  /* Velocities before the collision (angular-momentum correction). */
  double* v0 = NULL;
  if (p->angular) {
    v0 = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    memcpy(v0, vel, sizeof(double) * 3 * (size_t)n);
  }

  /* Bin solvent then beads. */
  for (int64_t i = 0; i < n; ++i)
    cellid[i] = cell_of(p, s, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]);
  for (int64_t b = 0; b < nb; ++b)
    cellid[n + b] = cell_of(p, s, spos[3 * b], spos[3 * b + 1], spos[3 * b + 2]);

  /* Cell properties (Sec. 3.5): count, mass, momentum. */
  memset(cb->cnt, 0, sizeof(int32_t) * ncells);
  memset(cb->nsol, 0, sizeof(int32_t) * ncells);
  memset(cb->nbead, 0, sizeof(int32_t) * ncells);
  memset(cb->nvirt, 0, sizeof(int32_t) * ncells);
  if (mixed) {
    memset(cb->Qs, 0, sizeof(int64_t) * 3 * ncells);
    memset(cb->Qx, 0, sizeof(int64_t) * 3 * ncells);
    memset(cb->S2, 0, sizeof(__int128) * ncells);
    memset(cb->Kx, 0, sizeof(int64_t) * ncells);
  } else {
    memset(cb->M, 0, sizeof(double) * ncells);
    memset(cb->P, 0, sizeof(double) * 3 * ncells);
    memset(cb->E, 0, sizeof(double) * ncells);
  }
  /* Mixed model: the same pass accumulates the kinetic energy as the exact
   * integer sum of V^2 (Sec. 3.5: momentum, mass and kinetic energy in one
   * pass), so E_k = K - |P|^2 / 2M carries no rounding before the final
   * conversion. */
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = cellid[i];
    cb->cnt[c] += 1;
    cb->nsol[c] += 1;
    for (int k = 0; k < 3; ++k) {
      if (mixed) {
        const int64_t V = llrint(vel[3 * i + k] * 0x1p32);
        cb->Qs[3 * c + k] += V;
        cb->S2[c] += (__int128)V * V;
      } else {
        cb->P[3 * c + k] += m * vel[3 * i + k];
      }
    }
    if (!mixed) cb->M[c] += m;
  }
  for (int64_t b = 0; b < nb; ++b) {
    int32_t c = cellid[n + b];
    cb->cnt[c] += 1;
    cb->nbead[c] += 1;
    for (int k = 0; k < 3; ++k) {
      if (mixed) cb->Qx[3 * c + k] += llrint((Mb * svel[3 * b + k]) * 0x1p32);
      else cb->P[3 * c + k] += Mb * svel[3 * b + k];
    }
    if (mixed) {
      const double* w = &svel[3 * b];
      cb->Kx[c] += llrint((Mb * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2])) * 0x1p32);
    }
    if (!mixed) cb->M[c] += Mb;
  }
  /* Walls: virtual particles in occupied cells cut by a wall. */
  if (p->walls_z) {
    int64_t nxy = (int64_t)p->n[0] * p->n[1];
    for (int64_t c = 0; c < ncells; ++c) {
      if (cb->cnt[c] == 0) continue;
      double fout = outside_fraction(p, s, c / nxy);
      int32_t nv = virtual_count(p, t, (uint32_t)c, fout);
      cb->nvirt[c] = nv;
      for (int32_t q = 0; q < nv; ++q) {
        double vv[3];
        virtual_velocity(p, t, (uint32_t)c, q, vv);
        for (int k = 0; k < 3; ++k) {
          if (mixed) cb->Qx[3 * c + k] += llrint((m * vv[k]) * 0x1p32);
          else cb->P[3 * c + k] += m * vv[k];
        }
        if (mixed) cb->Kx[c] += llrint((m * (vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2])) * 0x1p32);
        if (!mixed) cb->M[c] += m;
      }
    }
  }

  /* Centre-of-mass velocity u = P / M. */
  const float mf = (float)m, Mbf = (float)Mb;
  for (int64_t c = 0; c < ncells; ++c) {
    if (cb->cnt[c] == 0) continue;
    if (mixed) {
      float Mx = (float)cb->nbead[c] * Mbf + (float)cb->nvirt[c] * mf;
      float Mt = mf * (float)cb->nsol[c] + Mx;
      for (int k = 0; k < 3; ++k) {
        float P = mf * (float)cb->Qs[3 * c + k] + (float)cb->Qx[3 * c + k];
        cb->u[3 * c + k] = (double)((P * 0x1p-32f) / Mt);
      }
    } else {
      for (int k = 0; k < 3; ++k) cb->u[3 * c + k] = cb->P[3 * c + k] / cb->M[c];
    }
  }

  /* Andersen-thermostat rule, Eq. (at) and Sec. 3.7: a Gaussian random
   * velocity dv_i for every member, its mass-weighted mean over the cell,
   * dbar = sum m_i dv_i / sum m_i (the paper's (1/Nc) sum dv_j when all masses
   * are equal), and v_i <- u + dv_i - dbar. */
  if (p->collision == ORACLE_AT) {
    const double sig = sqrt(p->kT / m), sigb = sqrt(p->kT / Mb);
    double dv[3];
    if (mixed) {
      memset(cb->Qd, 0, sizeof(int64_t) * 3 * ncells);
      memset(cb->Qdx, 0, sizeof(int64_t) * 3 * ncells);
    } else {
      memset(cb->D, 0, sizeof(double) * 3 * ncells);
    }
    for (int64_t i = 0; i < n; ++i) {
      int32_t c = cellid[i];
      oracle_at_draw(p->seed, t, (uint32_t)i, 0, sig, arith, dv);
      for (int k = 0; k < 3; ++k) {
        if (mixed) cb->Qd[3 * c + k] += llrint(dv[k] * 0x1p32);
        else cb->D[3 * c + k] += m * dv[k];
      }
    }
    for (int64_t b = 0; b < nb; ++b) {
      int32_t c = cellid[n + b];
      oracle_at_draw(p->seed, t, (uint32_t)b, 1, sigb, arith, dv);
      for (int k = 0; k < 3; ++k) {
        if (mixed) cb->Qdx[3 * c + k] += llrint((Mb * dv[k]) * 0x1p32);
        else cb->D[3 * c + k] += Mb * dv[k];
      }
    }
    for (int64_t c = 0; c < ncells; ++c) {
      if (cb->cnt[c] == 0) continue;
      if (mixed) {
        float Mt = mf * (float)cb->nsol[c] + (float)cb->nbead[c] * Mbf;
        for (int k = 0; k < 3; ++k) {
          float Pd = mf * (float)cb->Qd[3 * c + k] + (float)cb->Qdx[3 * c + k];
          cb->dbar[3 * c + k] = (double)((Pd * 0x1p-32f) / Mt);
        }
      } else {
        for (int k = 0; k < 3; ++k) cb->dbar[3 * c + k] = cb->D[3 * c + k] / cb->M[c];
      }
    }
    for (int64_t i = 0; i < n; ++i) {
      int32_t c = cellid[i];
      oracle_at_draw(p->seed, t, (uint32_t)i, 0, sig, arith, dv);
      for (int k = 0; k < 3; ++k) {
        if (mixed) {
          float w = (float)cb->u[3 * c + k] + (float)dv[k];
          vel[3 * i + k] = (double)(w - (float)cb->dbar[3 * c + k]);
        } else {
          vel[3 * i + k] = (cb->u[3 * c + k] + dv[k]) - cb->dbar[3 * c + k];
        }
      }
    }
    for (int64_t b = 0; b < nb; ++b) {
      int32_t c = cellid[n + b];
      oracle_at_draw(p->seed, t, (uint32_t)b, 1, sigb, arith, dv);
      for (int k = 0; k < 3; ++k)
        svel[3 * b + k] = (cb->u[3 * c + k] + dv[k]) - cb->dbar[3 * c + k];
    }
    if (p->angular) {
      angular_correction(p, n, pos, v0, vel, cellid, s, ncells, cb->nsol);
      free(v0);
    }
    return status;
  }

  /* Thermostat, FP64 model: kinetic energy about u, Eq. (thermo), in a second
   * pass (the mixed model has it from the exact sums above). */
  if (p->thermostat && !mixed) {
    for (int64_t i = 0; i < n; ++i) {
      int32_t c = cellid[i];
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = vel[3 * i + k] - cb->u[3 * c + k];
      double e = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      cb->E[c] += (0.5 * m) * e;
    }
    for (int64_t b = 0; b < nb; ++b) {
      int32_t c = cellid[n + b];
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = svel[3 * b + k] - cb->u[3 * c + k];
      double e = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      cb->E[c] += (0.5 * Mb) * e;
    }
    if (p->walls_z) {
      for (int64_t c = 0; c < ncells; ++c) {
        for (int32_t q = 0; q < cb->nvirt[c]; ++q) {
          double vv[3], d[3];
          virtual_velocity(p, t, (uint32_t)c, q, vv);
          for (int k = 0; k < 3; ++k) d[k] = vv[k] - cb->u[3 * c + k];
          double e = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          cb->E[c] += (0.5 * m) * e;
        }
      }
    }
  }

  /* Per-cell axis and scale factor xi (Sec. 3.6). */
  for (int64_t c = 0; c < ncells; ++c) {
    cb->xi[c] = 1.0;
    if (cb->cnt[c] == 0) continue;
    oracle_axis(p->seed, t, (uint32_t)c, arith, &cb->axis[3 * c]);
    int32_t nc = cb->cnt[c] + cb->nvirt[c];
    if (p->thermostat && nc >= 2) {
      /* Mixed model: E_k Mt (E_k times the cell's mass) from the exact sums,
       * and xi = sqrt(E^ Mt / (E_k Mt)) to double accuracy (xi_mixed),
       * rounded to the float that scales the float relative velocities. */
      double Ek, Mt = 1.0;
      if (mixed) Ek = mixed_ek_mt(p, cb, c, hm2, &Mt);
      else Ek = cb->E[c];
      if (Ek > 0.0) {
        if (mixed) {
          float d, v;
          int32_t st = gamma_mixed_dv(p->seed, t, (uint32_t)c, nc, &d, &v);
          if (st != 0) { status = st; continue; }
          const double H = (((double)d * (double)v) * p->kT) * Mt;
          cb->xi[c] = (double)xi_mixed(H, (float)H, Ek, (float)Ek);
        } else {
          double ehat;
          int32_t st = oracle_gamma_draw(p->seed, t, (uint32_t)c, nc, p->kT, arith, &ehat);
          if (st != 0) { status = st; continue; }
          cb->xi[c] = sqrt(ehat / Ek);
        }
      }
    }
  }

  /* Collide, Eq. (srd) / Algorithm (SRD collision rule). */
  const float caf = (float)ca, saf = (float)sa, omcf = (float)omc;
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = cellid[i];
    if (mixed) {
      float nf[3], uf[3], d[3], rr[3];
      for (int k = 0; k < 3; ++k) {
        nf[k] = (float)cb->axis[3 * c + k];
        uf[k] = (float)cb->u[3 * c + k];
        d[k] = (float)vel[3 * i + k] - uf[k];
      }
      rotate_f(nf, caf, saf, omcf, d, rr);
      float xif = (float)cb->xi[c];
      for (int k = 0; k < 3; ++k) {
        float r = p->thermostat ? xif * rr[k] : rr[k];
        vel[3 * i + k] = (double)(uf[k] + r);
      }
    } else {
      double d[3], rr[3];
      for (int k = 0; k < 3; ++k) d[k] = vel[3 * i + k] - cb->u[3 * c + k];
      rotate_d(&cb->axis[3 * c], ca, sa, omc, d, rr);
      for (int k = 0; k < 3; ++k) {
        double r = p->thermostat ? cb->xi[c] * rr[k] : rr[k];
        vel[3 * i + k] = cb->u[3 * c + k] + r;
      }
    }
  }
  for (int64_t b = 0; b < nb; ++b) {
    int32_t c = cellid[n + b];
    double d[3], rr[3];
    for (int k = 0; k < 3; ++k) d[k] = svel[3 * b + k] - cb->u[3 * c + k];
    rotate_d(&cb->axis[3 * c], ca, sa, omc, d, rr);
    for (int k = 0; k < 3; ++k) {
      double r = p->thermostat ? cb->xi[c] * rr[k] : rr[k];
      svel[3 * b + k] = cb->u[3 * c + k] + r;
    }
  }
  if (p->angular) {
    angular_correction(p, n, pos, v0, vel, cellid, s, ncells, cb->nsol);
    free(v0);
  }
  return status;
}

static int32_t check_params(const oracle_params* p, int64_t n, int64_t nb) {
  for (int k = 0; k < 3; ++k)
    if (p->n[k] < 1) return -1;
  if (n < 0 || nb < 0) return -1;
  if (p->precision != ORACLE_FP64 && p->precision != ORACLE_MIXED &&
      p->precision != ORACLE_FP64_FSTREAM)
    return -1;
  if (!(p->dt > 0.0) || !(p->mass > 0.0) || !(p->kT >= 0.0)) return -1;
  if (p->walls_z && (p->g[2] != 0.0 || nb > 0)) return -1;
  if (p->collision != ORACLE_SRD && p->collision != ORACLE_AT) return -1;
  if (p->collision == ORACLE_AT && (p->thermostat || p->walls_z)) return -1;
  if (p->angular && (p->walls_z || nb > 0)) return -1;
  if (p->lj_epsilon < 0.0 || (p->lj_epsilon > 0.0 && !(p->lj_sigma > 0.0))) return -1;
  if (nb > 0 && (p->chain_len < 1 || nb % p->chain_len != 0 || p->md_substeps < 1 ||
                 !(p->solute_mass > 0.0)))
    return -1;
  if (oracle_num_cells(p) > 2147483647LL) return -1;
  return 0;
}

int32_t oracle_step(const oracle_params* p, int64_t n, double* pos, double* vel, int64_t nb,
                    double* spos, double* svel, uint64_t* step, int64_t nsteps,
                    int32_t* cell_out, int32_t* count_out) {
  int32_t st = check_params(p, n, nb);
  if (st) return st;
  int64_t ncells = oracle_num_cells(p);
  cellbuf cb;
  cb.cnt = (int32_t*)calloc((size_t)ncells, sizeof(int32_t));
  cb.nsol = (int32_t*)calloc((size_t)ncells, sizeof(int32_t));
  cb.nbead = (int32_t*)calloc((size_t)ncells, sizeof(int32_t));
  cb.nvirt = (int32_t*)calloc((size_t)ncells, sizeof(int32_t));
  cb.M = (double*)calloc((size_t)ncells, sizeof(double));
  cb.P = (double*)calloc((size_t)ncells * 3, sizeof(double));
  cb.E = (double*)calloc((size_t)ncells, sizeof(double));
  cb.Qs = (int64_t*)calloc((size_t)ncells * 3, sizeof(int64_t));
  cb.Qx = (int64_t*)calloc((size_t)ncells * 3, sizeof(int64_t));
  cb.S2 = (__int128*)calloc((size_t)ncells, sizeof(__int128));
  cb.Kx = (int64_t*)calloc((size_t)ncells, sizeof(int64_t));
  cb.u = (double*)calloc((size_t)ncells * 3, sizeof(double));
  cb.axis = (double*)calloc((size_t)ncells * 3, sizeof(double));
  cb.xi = (double*)calloc((size_t)ncells, sizeof(double));
  cb.D = (double*)calloc((size_t)ncells * 3, sizeof(double));
  cb.Qd = (int64_t*)calloc((size_t)ncells * 3, sizeof(int64_t));
  cb.Qdx = (int64_t*)calloc((size_t)ncells * 3, sizeof(int64_t));
  cb.dbar = (double*)calloc((size_t)ncells * 3, sizeof(double));
  int32_t* cellid = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + nb + 1));
  for (int64_t it = 0; it < nsteps && st == 0; ++it) {
    st = one_step(p, n, pos, vel, nb, spos, svel, *step, cellid, &cb, ncells);
    *step += 1;
  }
  if (nsteps > 0 && cell_out) memcpy(cell_out, cellid, sizeof(int32_t) * (size_t)(n + nb));
  if (nsteps > 0 && count_out) memcpy(count_out, cb.cnt, sizeof(int32_t) * (size_t)ncells);
  free(cellid);
  free(cb.cnt); free(cb.nsol); free(cb.nbead); free(cb.nvirt);
  free(cb.M); free(cb.P); free(cb.E);
  free(cb.Qs); free(cb.Qx); free(cb.S2); free(cb.Kx);
  free(cb.u); free(cb.axis); free(cb.xi);
  free(cb.D); free(cb.Qd); free(cb.Qdx); free(cb.dbar);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.5 (last paragraph): net momentum, energy and temperature.          */
/* ------------------------------------------------------------------------ */
int32_t oracle_observables(const oracle_params* p, int64_t n, const double* pos,
                           const double* vel, int64_t nb, const double* spos, const double* svel,
                           double* out) {
  int32_t st = check_params(p, n, nb);
  if (st) return st;
  const double m = p->mass, Mb = p->solute_mass;
  double P[3] = {0, 0, 0}, KE = 0.0, Mtot = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double* v = &vel[3 * i];
    for (int k = 0; k < 3; ++k) P[k] += m * v[k];
    KE += (0.5 * m) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    Mtot += m;
  }
  for (int64_t b = 0; b < nb; ++b) {
    const double* v = &svel[3 * b];
    for (int k = 0; k < 3; ++k) P[k] += Mb * v[k];
    KE += (0.5 * Mb) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    Mtot += Mb;
  }
  int64_t ntot = n + nb;
  double Tkin = 0.0;
  if (ntot > 1 && Mtot > 0.0) {
    double pp = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
    Tkin = 2.0 * (KE - pp / (2.0 * Mtot)) / (3.0 * (double)(ntot - 1));
  }
  /* Mean cell temperature on the unshifted grid. */
  oracle_params q = *p;
  q.walls_z = 0; /* unshifted cells of the channel: no extra layers needed */
  int64_t nc = (int64_t)p->n[0] * p->n[1] * p->n[2];
  int32_t* cnt = (int32_t*)calloc((size_t)nc, sizeof(int32_t));
  double* M = (double*)calloc((size_t)nc, sizeof(double));
  double* Pc = (double*)calloc((size_t)nc * 3, sizeof(double));
  double* K = (double*)calloc((size_t)nc, sizeof(double));
  double s0[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < ntot; ++i) {
    const double* r = i < n ? &pos[3 * i] : &spos[3 * (i - n)];
    const double* v = i < n ? &vel[3 * i] : &svel[3 * (i - n)];
    double mi = i < n ? m : Mb;
    int32_t c = cell_of(&q, s0, r[0], r[1], r[2]);
    cnt[c] += 1;
    M[c] += mi;
    for (int k = 0; k < 3; ++k) Pc[3 * c + k] += mi * v[k];
    K[c] += (0.5 * mi) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  }
  double Tsum = 0.0;
  int64_t nT = 0, occ = 0;
  for (int64_t c = 0; c < nc; ++c) {
    if (cnt[c] >= 1) occ += 1;
    if (cnt[c] >= 2) {
      double pp = Pc[3 * c] * Pc[3 * c] + Pc[3 * c + 1] * Pc[3 * c + 1] + Pc[3 * c + 2] * Pc[3 * c + 2];
      double Ek = K[c] - pp / (2.0 * M[c]);
      Tsum += 2.0 * Ek / (3.0 * (double)(cnt[c] - 1));
      nT += 1;
    }
  }
  free(cnt); free(M); free(Pc); free(K);
  out[0] = P[0]; out[1] = P[1]; out[2] = P[2];
  out[3] = KE;
  out[4] = Tkin;
  out[5] = nT > 0 ? Tsum / (double)nT : 0.0;
  out[6] = (double)occ;
  out[7] = Mtot;
  return 0;
}

int32_t oracle_profile(const oracle_params* p, int64_t n, const double* pos, const double* vel,
                       int32_t nbins, double* out) {
  if (nbins < 1 || n < 0) return -1;
  double H = (double)p->n[2];
  double* sum = (double*)calloc((size_t)nbins, sizeof(double));
  int64_t* cnt = (int64_t*)calloc((size_t)nbins, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    int64_t b = (int64_t)floor(pos[3 * i + 2] / H * (double)nbins);
    if (b < 0) b = 0;
    if (b >= nbins) b = nbins - 1;
    sum[b] += vel[3 * i];
    cnt[b] += 1;
  }
  for (int32_t b = 0; b < nbins; ++b) out[b] = cnt[b] ? sum[b] / (double)cnt[b] : 0.0;
  free(sum);
  free(cnt);
  return 0;
}
