// dev_angular.cuh -- helpers of the angular-momentum correction shared by
// the per-cell and warp-spread step kernels (the constraint the paper cites
// after Eqs. srd and at, Sec. 2: each cell's relative velocities receive a
// rigid rotation omega x r_c with Pi omega = sum m r_c x (v - v')).
#pragma once
#include <cuda_runtime.h>

namespace mpcd {

// The mixed model's coordinate relative to the shifted cell, in float: with
// x = fl + f (fl = floor(x) by a round-down add of 2^23, f exact) and the
// unwrapped cell coordinate i0 = fl - [f < lo] + [f >= hi] of the exact
// binning (lo, hi: the float thresholds of the shift s), x - s - i0 =
// (f - sf) + ([f < lo] - [f >= hi]) with sf = RN(s).  Needs 0 <= x < 2^23.
__device__ __forceinline__ float rel_pos_f(float x, float sf, float lo, float hi) {
  const float fl = __fsub_rn(__fadd_rd(x, 8388608.0f), 8388608.0f);
  const float f = __fsub_rn(x, fl);
  const float adj = (f < lo ? 1.0f : 0.0f) - (f >= hi ? 1.0f : 0.0f);
  return (f - sf) + adj;
}

// Float thresholds of the shift s = S 2^-32: f < s iff f < lo, f >= 1 + s
// iff f >= hi, for every float f in [0, 1).
__device__ __forceinline__ void shift_thresholds(long long S, float& sf, float& lo, float& hi) {
  const double s = (double)S * 0x1p-32;
  sf = (float)s;
  lo = ((double)sf < s) ? nextafterf(sf, INFINITY) : sf;
  const double t = 1.0 + s;
  const float th = (float)t;
  hi = ((double)th < t) ? nextafterf(th, INFINITY) : th;
}

// omega from Pi omega = dL, Pi = [[a, b, c], [b, d, e], [c, e, f]]: by the
// adjugate when Pi is well conditioned (nc >= 3), else 2 dL / tr(Pi), the
// solution on the plane normal to a two-member (or collinear) cell.
template <typename T>
__device__ __forceinline__ void solve_omega(int nc, const T P[6], const T dL[3], T w[3]) {
  const T a = P[0], b = P[1], c = P[2], d = P[3], e = P[4], f = P[5];
  const T A = d * f - e * e, Bc = c * e - b * f, C = b * e - c * d;
  const T D = a * f - c * c, E = b * c - a * e, F = a * d - b * b;
  const T det = a * A + b * Bc + c * C;
  const T tr = a + d + f;
  const T t3 = tr / (T)3;
  if (nc >= 3 && det > (T)1e-6 * (t3 * t3 * t3)) {
    w[0] = (A * dL[0] + Bc * dL[1] + C * dL[2]) / det;
    w[1] = (Bc * dL[0] + D * dL[1] + E * dL[2]) / det;
    w[2] = (C * dL[0] + E * dL[1] + F * dL[2]) / det;
  } else if (tr > (T)0) {
    const T g = (T)2 / tr;
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = dL[k] * g;
  } else {
    w[0] = w[1] = w[2] = (T)0;
  }
}

}  // namespace mpcd
