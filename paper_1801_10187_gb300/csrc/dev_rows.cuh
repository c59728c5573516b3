// dev_rows.cuh -- records of the cell rows and their insertion (the cell
// list of arXiv:1801.10187 Sec. 3.4, kept as fixed-capacity rows per cell).
#pragma once
#include <type_traits>

#include "mpcd_internal.cuh"

namespace mpcd {

template <bool MIXED>
using rec_t = typename std::conditional<MIXED, RecF, RecD>::type;

// A mixed-model record is one 32-byte sector, moved by one 256-bit access
// (records are 32-byte aligned: row bases are allocation-aligned and every
// row and slot is a multiple of 32 bytes).
__device__ __forceinline__ void load_rec(const RecF* p, float r[3], float v[3], uint32_t& tag) {
  float t;
  [[maybe_unused]] float pad;
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(t), "=f"(r[0]), "=f"(r[1]),
                 "=f"(r[2]), "=f"(pad)
               : "l"(p));
  tag = __float_as_uint(t);
}
__device__ __forceinline__ void store_rec(RecF* p, const float r[3], const float v[3], uint32_t tag) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]),
               "f"(v[1]), "f"(v[2]), "f"(__uint_as_float(tag)), "f"(r[0]), "f"(r[1]), "f"(r[2]),
               "f"(0.0f)
               : "memory");
}
__device__ __forceinline__ void load_rec(const RecD* p, double r[3], double v[3], uint32_t& tag) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  const double2 c = reinterpret_cast<const double2*>(p)[2];
  const uint4 d = reinterpret_cast<const uint4*>(p)[3];
  r[0] = a.x; r[1] = a.y; r[2] = b.x;
  v[0] = b.y; v[1] = c.x; v[2] = c.y;
  tag = d.x;
}
__device__ __forceinline__ void store_rec(RecD* p, const double r[3], const double v[3], uint32_t tag) {
  reinterpret_cast<double2*>(p)[0] = make_double2(r[0], r[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(r[2], v[0]);
  reinterpret_cast<double2*>(p)[2] = make_double2(v[1], v[2]);
  reinterpret_cast<uint4*>(p)[3] = make_uint4(tag, 0u, 0u, 0u);
}
__device__ __forceinline__ void load_v(const RecF* p, float v[3]) {
  const float4 a = reinterpret_cast<const float4*>(p)[0];
  v[0] = a.x; v[1] = a.y; v[2] = a.z;
}
__device__ __forceinline__ void load_v(const RecD* p, double v[3]) {
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  const double2 c = reinterpret_cast<const double2*>(p)[2];
  v[0] = b.y; v[1] = c.x; v[2] = c.y;
}

// Append a record to the row of cell c in the output set (or to the output
// overflow list when the row is full).
template <bool MIXED>
__device__ __forceinline__ void insert(const BoxDev& B, int out, uint32_t c,
                                       const real_t<MIXED> r[3], const real_t<MIXED> v[3],
                                       uint32_t tag, int* err) {
  using R = rec_t<MIXED>;
  const uint32_t slot = atomicAdd(&B.cnt[out][c], 1u);
  if (slot < (uint32_t)B.K) {
    store_rec(((R*)B.rows[out]) + (size_t)c * B.K + slot, r, v, tag);
  } else {
    const uint32_t j = atomicAdd(&B.ovf_n[out], 1u);
    if (j < (uint32_t)B.ovf_cap) {
      store_rec(((R*)B.ovf_rec[out]) + j, r, v, tag);
      B.ovf_cell[out][j] = c;
    } else {
      atomicOr(err, ERR_OVERFLOW_CAP);
    }
  }
}

}  // namespace mpcd
