// k_step.cu -- solute MD and bead grouping, the segmented scan used to group
// the beads, and the small per-step record updates (arXiv:1801.10187, Sec. 2
// and Sec. 3.6 solute coupling; Sec. 3.4 cell lists).
//
// All kernels are tile loops: a fixed grid walks a host-built table of
// (box, first index) tiles, so one launch serves every box of a batch.
#include <type_traits>

#include "dev_stream.cuh"
#include "kernels.h"
#include "mpcd_internal.cuh"

namespace mpcd {

// ---------------------------------------------------------------------------
// Solute: velocity-Verlet substeps with harmonic bonds along each chain, then
// binning of the beads with the step's shift.  One block holds whole chains
// in shared memory; bead j of the block is thread j.
//
// Each bond's force is computed once, by the bead at its left end, as
// g = f d with d = r_{j+1} - r_j; the bead at its right end adds -g.  That is
// the same value, bit for bit, as computing the bond from its own side:
// the difference, the minimum image (rint is odd), the norm and f * d are all
// odd or even in d exactly, so each bead's force is 0 + (left) + (right) as
// before, with one square root and one division per bond instead of two.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bond_right(const BoxDev& B, const double* __restrict__ sr, int j,
                                           int pos_in_chain, double* __restrict__ sg,
                                           int* __restrict__ sok) {
  if (pos_in_chain == B.chain_len - 1) return;  // the chain's last bead: no bond on its right
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d[k] = sr[3 * (j + 1) + k] - sr[3 * j + k];
    // minimum image; a bond shorter than L/4 needs no image (rint gives 0),
    // which saves the FP64 division on nearly every bond
    if (!(fabs(d[k]) < 0.25 * B.L[k])) d[k] = d[k] - B.L[k] * rint(d[k] / B.L[k]);
  }
  const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const bool ok = dist > 0.0;  // coincident beads: no force
  sok[j] = ok ? 1 : 0;
  if (!ok) return;
  const double f = (B.bond_k * (dist - B.bond_r0)) / dist;
#pragma unroll
  for (int k = 0; k < 3; ++k) sg[3 * j + k] = f * d[k];
}

__device__ __forceinline__ void bond_force(const BoxDev& B, const double* __restrict__ sg,
                                           const int* __restrict__ sok, int j, int pos_in_chain,
                                           double F[3]) {
  F[0] = F[1] = F[2] = 0.0;
  if (pos_in_chain > 0 && sok[j - 1]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k] += -sg[3 * (j - 1) + k];
  }
  if (pos_in_chain < B.chain_len - 1 && sok[j]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k] += sg[3 * j + k];
  }
}

__global__ void k_md_bin(const BoxDev* __restrict__ boxes, const int2* __restrict__ tiles,
                         int chains_per_block, int* err) {
  extern __shared__ double sr[];  // 3 * beads of this block, then the bond forces, then flags
  double* sg = sr + 3 * blockDim.x;
  int* sok = reinterpret_cast<int*>(sg + 3 * blockDim.x);
  const int2 tt = tiles[blockIdx.x];
  const BoxDev& B = boxes[tt.x];
  const int cl = B.chain_len;
  const int nchains = min(chains_per_block, B.nbead / cl - tt.y);
  const int nbb = nchains * cl;
  const int j = threadIdx.x;
  const bool active = j < nbb;
  const int pos = j % cl;
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
  // boxes with the non-bonded repulsion ran their MD in k_wca.cu; bin only
  const int nsub = B.wca ? 0 : B.md_substeps;
  if (nsub > 0) {
    __syncthreads();
    if (active) bond_right(B, sr, j, pos, sg, sok);
    __syncthreads();
    if (active) bond_force(B, sg, sok, j, pos, F);
  }
  for (int s = 0; s < nsub; ++s) {
    // every read of sr (the bonds) and of sg (the forces) of the last phase
    // came before a barrier that this thread has passed
    if (active) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        v[k] = v[k] + B.md_hh * F[k];
        r[k] = wrap(r[k] + B.md_h * v[k], B.L[k]);
        sr[3 * j + k] = r[k];
      }
    }
    __syncthreads();
    if (active) bond_right(B, sr, j, pos, sg, sok);
    __syncthreads();
    if (active) {
      bond_force(B, sg, sok, j, pos, F);
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
// Beads: border[bstart[group] + slot] = bead.
// ---------------------------------------------------------------------------
__global__ void k_bead_scatter(const BoxDev* __restrict__ boxes, const int2* __restrict__ tiles,
                               int ntiles) {
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int2 tt = tiles[tile];
    const BoxDev& B = boxes[tt.x];
    const int b1 = min(tt.y + PTILE, B.nbead);
    for (int b = tt.y + threadIdx.x; b < b1; b += blockDim.x) {
      const uint64_t k = B.bkey[b];
      const uint32_t slot = B.bstart[(uint32_t)(k >> 32)] + (uint32_t)k;
      B.border[slot] = (uint32_t)b;
      B.bgc[slot] = B.bcell[b];
      B.bgv[3 * slot] = B.svel[3 * b];
      B.bgv[3 * slot + 1] = B.svel[3 * b + 1];
      B.bgv[3 * slot + 2] = B.svel[3 * b + 2];
    }
  }
}

// ---------------------------------------------------------------------------
// Record updates between the passes: after a streaming pass (modes P and F)
// the output set becomes current and the consumed overflow list is emptied;
// a collision (modes F and C) completes step t.
// ---------------------------------------------------------------------------
__global__ void k_after_pass(BoxDev* boxes, int nboxes, int flip, int advance) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nboxes) return;
  BoxDev& B = boxes[b];
  if (flip) {
    B.ovf_n[B.cur] = 0u;
    B.cur ^= 1;
  }
  if (advance) B.step += 1ull;
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
// Shared memory of k_md_bin: positions and bond forces (3 doubles each) and
// one flag per thread; 1024 threads (one chain of the longest length) need
// 53,248 bytes, beyond the 48 KB granted without asking.
static size_t md_bin_smem(int threads) { return (sizeof(double) * 6 + sizeof(int)) * (size_t)threads; }

int md_bin_prepare() {
  return (int)cudaFuncSetAttribute(k_md_bin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)md_bin_smem(1024));
}

void launch_md_bin(const BoxDev* boxes, const int2* tiles, int ntiles, int chains_per_block,
                   int threads, int* err, cudaStream_t s) {
  if (ntiles <= 0) return;
  const size_t sm = md_bin_smem(threads);
  k_md_bin<<<ntiles, threads, sm, s>>>(boxes, tiles, chains_per_block, err);
}

void launch_scan(const ScanSeg* segs, const int2* tiles, int ntiles, uint32_t* tsum,
                 unsigned long long* gscan, uint32_t* toff, int grid, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_scan_reduce<<<grid, BLOCK, 0, s>>>(segs, tiles, ntiles, tsum);
  k_scan_tiles<<<1, 1024, 0, s>>>(tiles, ntiles, tsum, gscan, toff);
  k_scan_down<<<grid, BLOCK, 0, s>>>(segs, tiles, ntiles, toff);
}

void launch_bead_scatter(const BoxDev* boxes, const int2* tiles, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_bead_scatter<<<ntiles, BLOCK, 0, s>>>(boxes, tiles, ntiles);
}

void launch_after_pass(BoxDev* boxes, int nboxes, bool flip, bool advance, cudaStream_t s) {
  if (nboxes <= 0) return;
  k_after_pass<<<(nboxes + 127) / 128, 128, 0, s>>>(boxes, nboxes, flip ? 1 : 0, advance ? 1 : 0);
}

}  // namespace mpcd
