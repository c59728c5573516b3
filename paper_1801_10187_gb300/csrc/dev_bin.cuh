// dev_bin.cuh -- helpers of the mixed model's fused step kernels: exact float
// binning under the grid shift (Sec. 3.4), the periodic wrap, streamed record
// stores with an L2 policy, and the conversion of split fixed-point sums.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dev_collide.cuh"
#include "mpcd_internal.cuh"

namespace mpcd {

// L2 policy "evict first": pass 2 reads each record for the last time in the
// step and the records it writes are read again only next step, so neither
// should push out records that pass 1 has read and pass 2 has yet to re-read.
// (At 10^7 particles: DRAM traffic 761 -> 678 MB per step.)
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async16_last_use(void* smem, const void* gmem,
                                                    unsigned long long pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem),
               "l"(pol)
               : "memory");
}
// 16-byte global -> shared asynchronous copy (L2 only, default eviction).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void store_rec_streaming(RecF* p, const float r[3], const float v[3],
                                                    uint32_t tag, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8}, %9;" ::"l"(p),
               "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(__uint_as_float(tag)), "f"(r[0]), "f"(r[1]),
               "f"(r[2]), "f"(0.0f), "l"(pol)
               : "memory");
}

// rne(Q) as a float for Q = sh 2^20 + sl + x: one rounding of an exact sum of
// two exact floats when the parts are small (always, for real velocities).
__device__ __forceinline__ float split_sum_to_float(int sh, int sl, long long x) {
  if (x == 0 && sh > -16777216 && sh < 16777216 && sl > -16777216 && sl < 16777216)
    return __fadd_rn(__int2float_rn(sh) * 1048576.0f, __int2float_rn(sl));
  return i64_to_float((long long)sh * 1048576LL + (long long)sl + x);
}

// floor(x - s) for 0 <= x < 2^22 and s = S 2^-32 in [-1/2, 1/2), exactly:
// x = i0 + f with i0 = floor(x) (round-down add of 2^23) and f exact; then
// floor(x - s) = i0 - [f < s] + [f >= 1 + s].  f is a float, so f < s is
// f < lo with lo = RN(s), or its successor when RN(s) < s; f >= 1 + s is
// f >= hi with hi = RN(1 + s), or its successor when RN(1 + s) < 1 + s.
__device__ __forceinline__ void bin_thresholds(long long S, float& lo, float& hi) {
  const double s = (double)S * 0x1p-32;
  const float sh = (float)s;
  lo = ((double)sh < s) ? nextafterf(sh, INFINITY) : sh;
  const double t = 1.0 + s;
  const float th = (float)t;
  hi = ((double)th < t) ? nextafterf(th, INFINITY) : th;
}

__device__ __forceinline__ int bin_axis(float x, float lo, float hi, int n) {
  const float t = __fadd_rd(x, 8388608.0f);
  const int i0 = __float_as_int(t) - 0x4B000000;
  const float f = __fsub_rn(x, __fsub_rn(t, 8388608.0f));
  int i = i0 - (f < lo ? 1 : 0) + (f >= hi ? 1 : 0);
  if (i < 0) i += n;
  if (i >= n) i -= n;
  return i;
}

__device__ __forceinline__ float wrap_fast(float x, float L) {
  if (x >= L) x -= L;
  else if (x < 0.0f) x += L;
  return x;
}

}  // namespace mpcd
