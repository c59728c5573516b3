// k_step.cu -- streaming, binning, solute MD, counting sort by cell and the
// periodic reorder of the SRD step (arXiv:1801.10187, Sec. 2 Eq. stream;
// Sec. 3.4 cell list; Sec. 3.6 solute; Sec. 3.8 sorting).
//
// All kernels are tile loops: a fixed grid walks a host-built table of
// (box, first index) tiles, so one launch serves every box of a batch.
#include <type_traits>

#include "kernels.h"
#include "mpcd_internal.cuh"

namespace mpcd {

template <bool MIXED>
using real_t = typename std::conditional<MIXED, float, double>::type;

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

// ---------------------------------------------------------------------------
// Stream + bin + histogram of the solvent.
// ---------------------------------------------------------------------------
template <bool MIXED>
__global__ void __launch_bounds__(BLOCK) k_stream_bin(const BoxDev* __restrict__ boxes,
                                                      const int2* __restrict__ tiles, int ntiles,
                                                      int* err) {
  using T = real_t<MIXED>;
  __shared__ long long sS[3];
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int2 tt = tiles[tile];
    const BoxDev& B = boxes[tt.x];
    __syncthreads();
    if (threadIdx.x == 0) shift_units(B, B.step, sS);
    __syncthreads();
    const long long S[3] = {sS[0], sS[1], sS[2]};
    const int p1 = min(tt.y + PTILE, B.nsol);
    T* __restrict__ r = (T*)B.r;
    T* __restrict__ v = (T*)B.v;
    uint32_t* __restrict__ count = B.count;
    uint64_t* __restrict__ key = B.key;
    const bool vel_changes = B.walls || B.gdt[0] != 0.0 || B.gdt[1] != 0.0 || B.gdt[2] != 0.0;
    for (int i = tt.y + threadIdx.x; i < p1; i += BLOCK) {
      T x[3] = {r[3 * i], r[3 * i + 1], r[3 * i + 2]};
      T w[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
      stream_one(B, x, w);
      r[3 * i] = x[0];
      r[3 * i + 1] = x[1];
      r[3 * i + 2] = x[2];
      if (vel_changes) {
        v[3 * i] = w[0];
        v[3 * i + 1] = w[1];
        v[3 * i + 2] = w[2];
      }
      const uint32_t cell = cell_of(B, S, x, err);
      const uint32_t slot = atomicAdd(&count[cell], 1u);
      key[i] = ((uint64_t)cell << 32) | slot;
    }
  }
}

// ---------------------------------------------------------------------------
// Solute: velocity-Verlet substeps with harmonic bonds along each chain, then
// binning of the beads with the step's shift.  One block holds whole chains
// in shared memory; bead j of the block is thread j.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bond_force(const BoxDev& B, const double* __restrict__ sr, int j,
                                           int pos_in_chain, double F[3]) {
  F[0] = F[1] = F[2] = 0.0;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    int o;
    if (side == 0) {
      if (pos_in_chain == 0) continue;
      o = j - 1;
    } else {
      if (pos_in_chain == B.chain_len - 1) continue;
      o = j + 1;
    }
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      d[k] = sr[3 * o + k] - sr[3 * j + k];
      d[k] = d[k] - B.L[k] * rint(d[k] / B.L[k]);  // minimum image
    }
    const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(dist > 0.0)) continue;
    const double f = (B.bond_k * (dist - B.bond_r0)) / dist;
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k] += f * d[k];
  }
}

__global__ void k_md_bin(const BoxDev* __restrict__ boxes, const int2* __restrict__ tiles,
                         int chains_per_block, int* err) {
  extern __shared__ double sr[];  // 3 * beads of this block
  const int2 tt = tiles[blockIdx.x];
  const BoxDev& B = boxes[tt.x];
  const int cl = B.chain_len;
  const int nchains = min(chains_per_block, B.nbead / cl - tt.y);
  const int nbb = nchains * cl;
  const int j = threadIdx.x;
  const bool active = j < nbb;
  const int b = tt.y * cl + j;
  double r[3] = {0, 0, 0}, v[3] = {0, 0, 0}, F[3];
  if (active) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      r[k] = B.spos[3 * b + k];
      v[k] = B.svel[3 * b + k];
      sr[3 * j + k] = r[k];
    }
  }
  __syncthreads();
  if (active) bond_force(B, sr, j, j % cl, F);
  for (int s = 0; s < B.md_substeps; ++s) {
    __syncthreads();  // everyone has read sr for the forces
    if (active) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        v[k] = v[k] + B.md_hh * F[k];
        r[k] = wrap(r[k] + B.md_h * v[k], B.L[k]);
        sr[3 * j + k] = r[k];
      }
    }
    __syncthreads();
    if (active) {
      bond_force(B, sr, j, j % cl, F);
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = v[k] + B.md_hh * F[k];
    }
  }
  if (!active) return;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    B.spos[3 * b + k] = r[k];
    B.svel[3 * b + k] = v[k];
  }
  long long S[3];
  shift_units(B, B.step, S);
  const uint32_t cell = cell_of(B, S, r, err);
  B.bcell[b] = (int32_t)cell;
  const uint32_t tl = cell / (uint32_t)B.tc;
  const uint32_t slot = atomicAdd(&B.bcount[tl], 1u);
  B.bkey[b] = ((uint64_t)tl << 32) | slot;
}

// ---------------------------------------------------------------------------
// Segmented exclusive scan (counting sort by cell, Sec. 3.4/3.8).
// Phase 1: per-tile sums.  Phase 2: one block scans the tile sums and
// restarts at each segment.  Phase 3: per-tile scan plus offset; the counts
// are zeroed for the next step and the segment total closes start[n].
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_sum_u32(uint32_t x, uint32_t* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = x;
  __syncthreads();
  uint32_t t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;  // valid in thread 0
}

__global__ void __launch_bounds__(BLOCK) k_scan_reduce(const ScanSeg* __restrict__ segs,
                                                       const int2* __restrict__ tiles, int ntiles,
                                                       uint32_t* __restrict__ tsum) {
  __shared__ uint32_t red[BLOCK / 32];
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int2 tt = tiles[tile];
    const ScanSeg sg = segs[tt.x];
    const int i1 = min(tt.y + STILE, sg.n);
    uint32_t s = 0;
    for (int i = tt.y + threadIdx.x; i < i1; i += BLOCK) s += sg.count[i];
    const uint32_t t = block_sum_u32(s, red);
    if (threadIdx.x == 0) tsum[tile] = t;
  }
}

// One block of 1024 threads: exclusive scan of tsum (as 64-bit) restarted at
// every tile whose first index is 0 (the first tile of a segment).
__global__ void __launch_bounds__(1024) k_scan_tiles(const int2* __restrict__ tiles, int ntiles,
                                                     const uint32_t* __restrict__ tsum,
                                                     unsigned long long* __restrict__ gscan,
                                                     uint32_t* __restrict__ toff) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += 1024) {
    const int t = base + threadIdx.x;
    unsigned long long x = (t < ntiles) ? tsum[t] : 0ull;
    // inclusive warp scan
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if ((threadIdx.x & 31) >= o) inc += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = inc;
    __syncthreads();
    if (threadIdx.x < 32) {
      unsigned long long w = wsum[threadIdx.x];
      unsigned long long wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
        if (threadIdx.x >= o) wi += y;
      }
      wsum[threadIdx.x] = wi - w;  // exclusive warp offsets
    }
    __syncthreads();
    const unsigned long long excl = carry + wsum[threadIdx.x >> 5] + inc - x;
    if (t < ntiles) gscan[t] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + x;
    __syncthreads();
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntiles; t += 1024) {
    const int first = t - tiles[t].y / STILE;
    toff[t] = (uint32_t)(gscan[t] - gscan[first]);
  }
}

__global__ void __launch_bounds__(BLOCK) k_scan_down(const ScanSeg* __restrict__ segs,
                                                     const int2* __restrict__ tiles, int ntiles,
                                                     const uint32_t* __restrict__ toff) {
  constexpr int PER = STILE / BLOCK;  // 8 entries per thread
  __shared__ uint32_t wsum[BLOCK / 32];
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int2 tt = tiles[tile];
    const ScanSeg sg = segs[tt.x];
    const int i0 = tt.y + threadIdx.x * PER;
    uint32_t c[PER];
    uint32_t tot = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = i0 + q;
      c[q] = (i < sg.n) ? sg.count[i] : 0u;
      tot += c[q];
    }
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if ((threadIdx.x & 31) >= o) inc += y;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = inc;
    __syncthreads();
    uint32_t woff = 0;
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) woff += wsum[w];
    uint32_t run = toff[tile] + woff + inc - tot;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = i0 + q;
      if (i < sg.n) {
        sg.start[i] = run;
        sg.count[i] = 0u;
      }
      run += c[q];
    }
    // the thread holding the segment's last entry closes it
    if (i0 <= sg.n - 1 && sg.n - 1 < i0 + PER) sg.start[sg.n] = run;
  }
}

// ---------------------------------------------------------------------------
// Scatter: order[start[cell] + slot] = particle.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BLOCK) k_scatter(const BoxDev* __restrict__ boxes,
                                                   const int2* __restrict__ tiles, int ntiles) {
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int2 tt = tiles[tile];
    const BoxDev& B = boxes[tt.x];
    const int p1 = min(tt.y + PTILE, B.nsol);
    const uint64_t* __restrict__ key = B.key;
    const uint32_t* __restrict__ start = B.start;
    uint32_t* __restrict__ order = B.order;
    for (int i = tt.y + threadIdx.x; i < p1; i += BLOCK) {
      const uint64_t k = key[i];
      order[start[(uint32_t)(k >> 32)] + (uint32_t)k] = (uint32_t)i;
    }
  }
}

__global__ void k_bead_scatter(const BoxDev* __restrict__ boxes, const int2* __restrict__ tiles,
                               int ntiles) {
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int2 tt = tiles[tile];
    const BoxDev& B = boxes[tt.x];
    const int b1 = min(tt.y + PTILE, B.nbead);
    for (int b = tt.y + threadIdx.x; b < b1; b += blockDim.x) {
      const uint64_t k = B.bkey[b];
      B.border[B.bstart[(uint32_t)(k >> 32)] + (uint32_t)k] = (uint32_t)b;
    }
  }
}

// ---------------------------------------------------------------------------
// Sec. 3.8: every sort_period steps the particle data is rewritten in cell
// order (into the second buffers; the end-of-step kernel swaps them) and the
// order becomes the identity, so the collision reads it contiguously.
// ---------------------------------------------------------------------------
template <bool MIXED>
__global__ void __launch_bounds__(BLOCK) k_permute(const BoxDev* __restrict__ boxes,
                                                   const int2* __restrict__ tiles, int ntiles) {
  using T = real_t<MIXED>;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int2 tt = tiles[tile];
    const BoxDev& B = boxes[tt.x];
    if (!(B.sort_period > 0 && (B.step % (unsigned long long)B.sort_period) == 0)) continue;
    const int p1 = min(tt.y + PTILE, B.nsol);
    const T* __restrict__ r = (const T*)B.r;
    const T* __restrict__ v = (const T*)B.v;
    T* __restrict__ r2 = (T*)B.r2;
    T* __restrict__ v2 = (T*)B.v2;
    uint32_t* __restrict__ order = B.order;
    for (int k = tt.y + threadIdx.x; k < p1; k += BLOCK) {
      const uint32_t i = order[k];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        r2[3 * k + q] = r[3 * i + q];
        v2[3 * k + q] = v[3 * i + q];
      }
      B.tag2[k] = B.tag[i];
      order[k] = (uint32_t)k;
    }
  }
}

// After a reorder the second buffers hold the particles in cell order: swap
// them in before the collision reads them.
__global__ void k_swap(BoxDev* boxes, int nboxes) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nboxes) return;
  BoxDev& B = boxes[b];
  const bool due = B.sort_period > 0 && (B.step % (unsigned long long)B.sort_period) == 0;
  if (due) {
    void* t = B.r; B.r = B.r2; B.r2 = t;
    t = B.v; B.v = B.v2; B.v2 = t;
    uint32_t* u = B.tag; B.tag = B.tag2; B.tag2 = u;
  }
  B.permuted = due ? 1 : 0;
}

__global__ void k_end_step(BoxDev* boxes, int nboxes, int* novf) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) *novf = 0;
  if (b >= nboxes) return;
  boxes[b].step += 1ull;
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
void launch_stream_bin(bool mixed, const BoxDev* boxes, const int2* tiles, int ntiles, int grid,
                       int* err, cudaStream_t s) {
  if (ntiles <= 0) return;
  if (mixed) k_stream_bin<true><<<grid, BLOCK, 0, s>>>(boxes, tiles, ntiles, err);
  else k_stream_bin<false><<<grid, BLOCK, 0, s>>>(boxes, tiles, ntiles, err);
}

void launch_md_bin(const BoxDev* boxes, const int2* tiles, int ntiles, int chains_per_block,
                   int threads, int* err, cudaStream_t s) {
  if (ntiles <= 0) return;
  const size_t sm = sizeof(double) * 3 * (size_t)threads;
  k_md_bin<<<ntiles, threads, sm, s>>>(boxes, tiles, chains_per_block, err);
}

void launch_scan(const ScanSeg* segs, const int2* tiles, int ntiles, uint32_t* tsum,
                 unsigned long long* gscan, uint32_t* toff, int grid, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_scan_reduce<<<grid, BLOCK, 0, s>>>(segs, tiles, ntiles, tsum);
  k_scan_tiles<<<1, 1024, 0, s>>>(tiles, ntiles, tsum, gscan, toff);
  k_scan_down<<<grid, BLOCK, 0, s>>>(segs, tiles, ntiles, toff);
}

void launch_scatter(const BoxDev* boxes, const int2* tiles, int ntiles, int grid, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_scatter<<<grid, BLOCK, 0, s>>>(boxes, tiles, ntiles);
}

void launch_bead_scatter(const BoxDev* boxes, const int2* tiles, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_bead_scatter<<<ntiles, BLOCK, 0, s>>>(boxes, tiles, ntiles);
}

void launch_permute(bool mixed, BoxDev* boxes, int nboxes, const int2* tiles, int ntiles,
                    int grid, cudaStream_t s) {
  if (ntiles > 0) {
    if (mixed) k_permute<true><<<grid, BLOCK, 0, s>>>(boxes, tiles, ntiles);
    else k_permute<false><<<grid, BLOCK, 0, s>>>(boxes, tiles, ntiles);
  }
  if (nboxes > 0) k_swap<<<(nboxes + 127) / 128, 128, 0, s>>>(boxes, nboxes);
}

void launch_end_step(BoxDev* boxes, int nboxes, int* novf, cudaStream_t s) {
  if (nboxes <= 0) return;
  k_end_step<<<(nboxes + 127) / 128, 128, 0, s>>>(boxes, nboxes, novf);
}

}  // namespace mpcd
