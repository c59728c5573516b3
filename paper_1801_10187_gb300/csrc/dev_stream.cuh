// dev_stream.cuh -- device helpers of the streaming and binning steps
// (arXiv:1801.10187, Sec. 2 Eq. stream; Sec. 3.4 binning with a grid shift).
#pragma once
#include "mpcd_internal.cuh"

namespace mpcd {

// ---------------------------------------------------------------------------
// Periodic wrap into [0, L).  The second branch only runs for positions more
// than one box length out (or at the rounding edge x + L == L).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float wrap(float x, float L) {
  if (x >= L) x -= L;
  else if (x < 0.0f) x += L;
  if (!(x >= 0.0f && x < L)) {
    x = x - L * floorf(x / L);
    if (!(x >= 0.0f && x < L)) x = 0.0f;
  }
  return x;
}
__device__ __forceinline__ double wrap(double x, double L) {
  if (x >= L) x -= L;
  else if (x < 0.0) x += L;
  if (!(x >= 0.0 && x < L)) {
    x = x - L * floor(x / L);
    if (!(x >= 0.0 && x < L)) x = 0.0;
  }
  return x;
}

// The same wrap with its common case settled on the bit pattern: for L > 0 a
// double with +0 <= x < L is exactly one whose bits, read as an unsigned
// integer, are below L's (negatives and -0 carry the sign bit, NaN and x >= L
// sit above), and wrap() returns such an x unchanged.  Everything else takes
// wrap() itself, so the result is wrap()'s for every x; only the compare
// leaves the FP64 pipe.
__device__ __forceinline__ double wrap_bits(double x, double L) {
  if ((unsigned long long)__double_as_longlong(x) < (unsigned long long)__double_as_longlong(L))
    return x;
  return wrap(x, L);
}

// floor(RN(x - s)), the double expression of Sec. 3.4's cell index, for x = +-0
// or 0 <= x < 2^21 and s = S 2^-32 in [-1/2, 1/2), in integer arithmetic.  S
// is an integer, so floor(x - s) = floor((floor(x 2^32) - S) 2^-32), and
// floor(x 2^32) is x's significand shifted by its exponent.  The rounded
// difference has the same floor except at one point: a difference that
// rounds must leave x's binade upwards (s < 0), so for x >= 1/2 it lies in
// [2^j, 2^j + 1/2] above the integer 2^j, and for x < 1/2 it is at most
// 1 - 2^-54, which rounds (to even) up to 1 only for x = 1/2 - 2^-54 and
// s = -1/2.  Above 2^21 (boxes with more cells per axis) the double
// expression itself is used.
__device__ __forceinline__ int floor_minus_shift(double x, long long S, double s) {
  const long long b = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL;
  const int e = (int)(b >> 52);  // biased exponent; x 2^32 = m 2^(e - 1043)
  if (e >= 1044) return (int)floor(x - s);
  if (b == 0x3FDFFFFFFFFFFFFFLL && S == -2147483648LL) return 1;
  const long long m = (b & 0x000FFFFFFFFFFFFFLL) | 0x0010000000000000LL;
  const long long X = m >> min(1043 - e, 63);  // 0 for zeros and subnormals
  return (int)((X - S) >> 32);
}

// ---------------------------------------------------------------------------
// Eq. (stream): r <- r + v dt (+ g dt^2 / 2, v <- v + g dt).  With walls in z
// the particle reaches the wall at tau, its velocity is reversed (no-slip
// bounce-back) and it streams for the remaining dt - tau.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void stream_one(const BoxDev& B, float r[3], float v[3]) {
  const float dt = B.dt_f;
  if (B.walls) {
    const float H = B.L_f[2];
    const float zn = fmaf(v[2], dt, r[2]);
    if (!(zn >= 0.0f && zn < H)) {
      const float wall = (zn < 0.0f) ? 0.0f : H;
      float tau = (wall - r[2]) / v[2];
      if (!(tau >= 0.0f)) tau = 0.0f;
      if (tau > dt) tau = dt;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        r[k] = fmaf(v[k], tau, r[k]) + ((0.5f * B.g_f[k]) * tau) * tau;
        v[k] = v[k] + B.g_f[k] * tau;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = -v[k];
      const float rem = dt - tau;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        r[k] = fmaf(v[k], rem, r[k]) + ((0.5f * B.g_f[k]) * rem) * rem;
        v[k] = v[k] + B.g_f[k] * rem;
      }
      float z = fmaf(v[2], rem, wall);
      if (z < 0.0f) z = 0.0f;
      if (z >= H) z = nextafterf(H, 0.0f);
      r[2] = z;
      r[0] = wrap(r[0], B.L_f[0]);
      r[1] = wrap(r[1], B.L_f[1]);
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r[k] = fmaf(v[k], dt, r[k]) + B.hg_f[k];
    v[k] = v[k] + B.gdt_f[k];
    if (!(k == 2 && B.walls)) r[k] = wrap(r[k], B.L_f[k]);
  }
}

__device__ __forceinline__ void stream_one(const BoxDev& B, double r[3], double v[3]) {
  const double dt = B.dt;
  if (B.walls) {
    const double H = B.L[2];
    const double zn = fma(v[2], dt, r[2]);
    if (!(zn >= 0.0 && zn < H)) {
      const double wall = (zn < 0.0) ? 0.0 : H;
      double tau = (wall - r[2]) / v[2];
      if (!(tau >= 0.0)) tau = 0.0;
      if (tau > dt) tau = dt;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        r[k] = fma(v[k], tau, r[k]) + ((0.5 * B.g[k]) * tau) * tau;
        v[k] = v[k] + B.g[k] * tau;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = -v[k];
      const double rem = dt - tau;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        r[k] = fma(v[k], rem, r[k]) + ((0.5 * B.g[k]) * rem) * rem;
        v[k] = v[k] + B.g[k] * rem;
      }
      double z = fma(v[2], rem, wall);
      if (z < 0.0) z = 0.0;
      if (z >= H) z = nextafter(H, 0.0);
      r[2] = z;
      r[0] = wrap(r[0], B.L[0]);
      r[1] = wrap(r[1], B.L[1]);
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r[k] = fma(v[k], dt, r[k]) + B.hg[k];
    v[k] = v[k] + B.gdt[k];
    if (!(k == 2 && B.walls)) r[k] = wrap(r[k], B.L[k]);
  }
}

// ---------------------------------------------------------------------------
// Sec. 3.4 binning under the grid shift s = S 2^-32.  floor(x - s) computed
// exactly: for a float x >= 0, X = floor(x 2^32) comes from the exponent and
// mantissa bits, and floor(x - s) = (X - S) >> 32 because S is an integer.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long floor_fix32(float x) {
  const uint32_t bits = __float_as_uint(x) & 0x7FFFFFFFu;
  const int e = (int)(bits >> 23);
  if (e == 0) return 0;  // zero or below 2^-126
  const long long m = (long long)((bits & 0x7FFFFFu) | 0x800000u);
  const int sh = e - 118;  // x 2^32 = m 2^(e - 150 + 32)
  if (sh >= 0) return sh > 38 ? (1LL << 62) : (m << sh);
  return (-sh) >= 24 ? 0 : (m >> (-sh));
}

__device__ __forceinline__ int axis_cell(float x, long long S) {
  return (int)((floor_fix32(x) - S) >> 32);
}
__device__ __forceinline__ int axis_cell(double x, long long S) {
  const double f = floor(x - (double)S * 0x1p-32);
  return (f >= -2147483648.0 && f < 2147483647.0) ? (int)f : 0x40000000;
}

// Cell id (x fastest); out-of-grid coordinates (non-finite input) are
// clamped and flagged.
template <typename T>
__device__ __forceinline__ uint32_t cell_of(const BoxDev& B, const long long S[3], const T x[3],
                                            int* err) {
  int c[3];
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int i = axis_cell(x[k], S[k]);
    if (k == 2 && B.walls) {
      i += 1;
      if (i < 0) i = 0;
      if (i > B.n[2] + 1) i = B.n[2] + 1;
    } else {
      const int n = B.n[k];
      if (i < 0) i += n;
      if (i >= n) i -= n;
      if (i < 0 || i >= n) {
        bad = true;
        i = 0;
      }
    }
    c[k] = i;
  }
  if (bad) atomicOr(err, ERR_CELL_RANGE);
  return (uint32_t)(c[0] + B.n[0] * (c[1] + B.n[1] * c[2]));
}


}  // namespace mpcd
