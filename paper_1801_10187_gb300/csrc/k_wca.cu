// k_wca.cu -- non-bonded solute forces (arXiv:1801.10187, Sec. 4.3: the
// polymer benchmark integrates a bead-spring model by velocity Verlet with
// non-bonded pair forces from a neighbour list of buffer 0.4 a; the pair
// potential is only cited, and the Weeks-Chandler-Andersen repulsion is the
// reading taken here).
//
// Per collision step, for the boxes with the repulsion on:
//   clear, insert   a hash grid of the beads: cells of edge 1 (unshifted),
//                   two buckets per bead, each bucket a linked list built by
//                   atomic exchange of its head
//   list            each bead lists the beads of the 27 surrounding cells
//                   that lie within cutoff + buffer (minimum image)
//   force           bonds (its chain neighbours) plus WCA over the list
//   kick-drift, [clear, insert, list,] force, kick    one velocity-Verlet
//                   substep, md_substeps times
// The list holds every pair within the cutoff while no bead has moved more
// than half the buffer from where it was at the build.  The drift marks the
// box stale when one has, and the list kernels of that substep then rebuild
// it (they return at once for a box that is not stale), so every force uses
// a complete list.  More than NL_MAX listed neighbours raises ERR_NLIST.  The
// later binning of the beads for the collision (k_md_bin) skips its own MD
// for these boxes.
#include "dev_stream.cuh"
#include "kernels.h"
#include "mpcd_internal.cuh"

namespace mpcd {

namespace {

__device__ __forceinline__ uint32_t bucket_of(int key, int hsize) {
  return ((uint32_t)key * 2654435761u) % (uint32_t)hsize;
}

__device__ __forceinline__ int grid_coord(double x, int n) {
  int c = (int)floor(x);
  if (c < 0) c = 0;
  if (c >= n) c = n - 1;
  return c;
}

// minimum-image difference along one axis for |d| < L (both points in the
// box): the same result as d - L rint(d / L), without the division
__device__ __forceinline__ double min_image(double d, double L) {
  if (fabs(d) > 0.5 * L) d -= copysign(L, d);
  return d;
}

// Harmonic bond forces on global bead b from its chain neighbours.
__device__ __forceinline__ void bonds_on(const BoxDev& B, int b, double F[3]) {
  F[0] = F[1] = F[2] = 0.0;
  const int pos = b % B.chain_len;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    int o;
    if (side == 0) {
      if (pos == 0) continue;
      o = b - 1;
    } else {
      if (pos == B.chain_len - 1) continue;
      o = b + 1;
    }
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = min_image(B.spos[3 * o + k] - B.spos[3 * b + k], B.L[k]);
    const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(dist > 0.0)) continue;
    const double f = (B.bond_k * (dist - B.bond_r0)) / dist;
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k] += f * d[k];
  }
}

// A tile of PTILE beads is split over WCA_SPLIT blocks of WCA_THREADS
// threads, one bead per thread, so that even 5 * 10^4 beads fill every SM.
constexpr int WCA_SPLIT = 8;
constexpr int WCA_THREADS = PTILE / WCA_SPLIT;

// f(B, b) for the bead of this thread, in a box with the repulsion on.
template <class F>
__device__ __forceinline__ void for_tile_beads(const BoxDev* boxes, const int2* tiles, F&& f) {
  const int2 tt = tiles[blockIdx.x / WCA_SPLIT];
  const BoxDev& B = boxes[tt.x];
  if (!B.wca) return;
  const int b = tt.y + (int)(blockIdx.x % WCA_SPLIT) * WCA_THREADS + (int)threadIdx.x;
  if (b < B.nbead) f(B, b);
}

}  // namespace

__global__ void __launch_bounds__(WCA_THREADS) k_wca_clear(const BoxDev* __restrict__ boxes, const int2* __restrict__ tiles,
                            int always) {
  const int2 tt = tiles[blockIdx.x / WCA_SPLIT];
  const BoxDev& B = boxes[tt.x];
  if (!B.wca || !(always || *B.nl_stale)) return;
  const int h0 = 2 * tt.y + (int)(blockIdx.x % WCA_SPLIT) * 2 * WCA_THREADS;
  const int h1 = min(h0 + 2 * WCA_THREADS, B.nl_hsize);
  for (int h = h0 + (int)threadIdx.x; h < h1; h += blockDim.x) B.nl_head[h] = -1;
}

__global__ void __launch_bounds__(WCA_THREADS) k_wca_insert(const BoxDev* __restrict__ boxes, const int2* __restrict__ tiles,
                             int always) {
  for_tile_beads(boxes, tiles, [&](const BoxDev& B, int b) {
    if (!(always || *B.nl_stale)) return;
    int c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double x = B.spos[3 * b + k];
      B.nl_rb[3 * b + k] = x;
      c[k] = grid_coord(x, B.n[k]);
    }
    const int key = c[0] + B.n[0] * (c[1] + B.n[1] * c[2]);
    B.nl_key[b] = key;
    B.nl_next[b] = atomicExch(&B.nl_head[bucket_of(key, B.nl_hsize)], b);
  });
}

__global__ void __launch_bounds__(WCA_THREADS) k_wca_list(const BoxDev* __restrict__ boxes, const int2* __restrict__ tiles,
                           int always, int* err) {
  for_tile_beads(boxes, tiles, [&](const BoxDev& B, int b) {
    if (!(always || *B.nl_stale)) return;
    const int key = B.nl_key[b];
    const int c[3] = {key % B.n[0], (key / B.n[0]) % B.n[1], key / (B.n[0] * B.n[1])};
    const double rb[3] = {B.nl_rb[3 * b], B.nl_rb[3 * b + 1], B.nl_rb[3 * b + 2]};
    int cnt = 0;
    bool over = false;
    // n_k >= 3 on every axis, so the 27 cells are distinct
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int x = (c[0] + dx + B.n[0]) % B.n[0], y = (c[1] + dy + B.n[1]) % B.n[1],
                    z = (c[2] + dz + B.n[2]) % B.n[2];
          const int k2 = x + B.n[0] * (y + B.n[1] * z);
          int j = B.nl_head[bucket_of(k2, B.nl_hsize)];
          // a bucket's list is acyclic and holds at most every bead once
          for (int guard = 0; j >= 0 && guard < B.nbead; ++guard, j = B.nl_next[j]) {
            if (j == b || B.nl_key[j] != k2) continue;
            double r2 = 0.0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              const double d = min_image(B.nl_rb[3 * j + q] - rb[q], B.L[q]);
              r2 += d * d;
            }
            if (!(r2 < B.wca_rl2)) continue;
            if (cnt < NL_MAX) B.nl_nbr[(size_t)b * NL_MAX + cnt] = j;
            else over = true;
            ++cnt;
          }
        }
    B.nl_cnt[b] = min(cnt, NL_MAX);
    if (over) atomicOr(err, ERR_NLIST);
  });
}

// Bond forces plus the WCA repulsion over the bead's list (Sec. 4.3 reading).
//
// The arithmetic is FP64, and the FP64 pipe issues a warp instruction only
// every many cycles on this GPU, so what counts is how many lanes of each
// instruction do useful work.  A warp owns 32 consecutive beads.  Each lane
// takes its own bead's two bonds.  The warp's listed pairs are then taken as
// one flat sequence (bead by bead, in list order), 32 at a time: each lane
// forms the distance of one pair, and the pairs within the cutoff go, in
// order, to a queue in shared memory.  Whenever the queue holds 32 pairs,
// every lane takes one and computes its force; the forces of each bead's run
// in the queue are added in queue order by the run's first lane (no
// atomics).  So the divisions run on full warps however the list lengths and
// hits are spread over the beads.  The list order follows the hash grid's
// insertion order, which may differ between runs, and so may the last bits
// of a sum.
namespace {
constexpr int FW = WCA_THREADS / 32;  // warps per block
constexpr int QCAP = 64;              // queue: fewer than 32 waiting plus one round of 32

struct ForceWarp {
  int off[33];          // first flat pair index of each bead; off[32] = all pairs
  int qown[QCAP];       // queued pair: the warp-local bead it acts on
  double qd[4][QCAP];   // queued pair: d (3) and r^2
  double c[3][32];      // forces of one flush, one per lane
  double F[3][32];      // sum of each bead's pair forces
  double rb[3][32];     // bead positions
};

// Forces of queue entries [0, nq): lane l takes entry l; each run of
// entries of one bead is summed, in order, by its first lane.
__device__ __forceinline__ void wca_flush(const BoxDev& B, ForceWarp& W, int nq, int lane) {
  if (lane < nq) {
    const double r2 = W.qd[3][lane];
    const double inv = 1.0 / r2;
    const double x = B.lj_sig2 * inv;
    const double x6 = x * x * x;
    const double g = 24.0 * B.lj_eps * x6 * (2.0 * x6 - 1.0) * inv;
#pragma unroll
    for (int q = 0; q < 3; ++q) W.c[q][lane] = -(g * W.qd[q][lane]);
  }
  __syncwarp();
  if (lane < nq) {
    const int own = W.qown[lane];
    if (lane == 0 || W.qown[lane - 1] != own) {
      double acc[3] = {W.c[0][lane], W.c[1][lane], W.c[2][lane]};
      for (int l = lane + 1; l < nq && W.qown[l] == own; ++l) {
#pragma unroll
        for (int q = 0; q < 3; ++q) acc[q] += W.c[q][l];
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) W.F[q][own] += acc[q];
    }
  }
  __syncwarp();
}
}  // namespace

__global__ void __launch_bounds__(WCA_THREADS) k_wca_force(const BoxDev* __restrict__ boxes, const int2* __restrict__ tiles,
                            int substep) {
  __shared__ ForceWarp fw[FW];
  const int2 tt = tiles[blockIdx.x / WCA_SPLIT];
  const BoxDev& B = boxes[tt.x];
  if (!B.wca || substep > B.md_substeps) return;  // the same for the whole block
  const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  ForceWarp& W = fw[warp];
  const int b0 = tt.y + (int)(blockIdx.x % WCA_SPLIT) * WCA_THREADS + warp * 32;
  const int b = b0 + lane;
  const bool valid = b < B.nbead;
  double F[3] = {0.0, 0.0, 0.0};
  int cnt = 0;
  if (valid) {
    if (b == 0) *B.nl_stale = 0;  // this substep's list kernels have all run
    bonds_on(B, b, F);
    cnt = B.nl_cnt[b];
#pragma unroll
    for (int q = 0; q < 3; ++q) W.rb[q][lane] = B.spos[3 * b + q];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) W.F[q][lane] = 0.0;
  // flat pair offsets: exclusive scan of the list lengths over the warp
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  W.off[lane] = incl - cnt;
  if (lane == 31) W.off[32] = incl;
  __syncwarp();
  const int total = W.off[32];  // at most 32 NL_MAX
  int nq = 0;                   // queued pairs (the same in every lane)
  for (int base = 0; base < total; base += 32) {
    const int k = base + lane;
    bool hit = false;
    int own = 0;
    double d[3] = {0.0, 0.0, 0.0}, r2 = 0.0;
    if (k < total) {
      // the bead of pair k: the last with off <= k (offsets do not decrease)
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (W.off[own + step] <= k) own += step;
      const int j = B.nl_nbr[(size_t)(b0 + own) * NL_MAX + (k - W.off[own])];
#pragma unroll
      for (int q = 0; q < 3; ++q) d[q] = min_image(B.spos[3 * j + q] - W.rb[q][own], B.L[q]);
      r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      hit = r2 < B.wca_rc2;
    }
    const unsigned m = __ballot_sync(0xFFFFFFFFu, hit);
    if (hit) {
      const int pos = nq + __popc(m & ((1u << lane) - 1u));  // < nq + 32 <= QCAP
      W.qown[pos] = own;
#pragma unroll
      for (int q = 0; q < 3; ++q) W.qd[q][pos] = d[q];
      W.qd[3][pos] = r2;
    }
    nq += __popc(m);
    __syncwarp();
    if (nq >= 32) {
      wca_flush(B, W, 32, lane);
      nq -= 32;
      // move the rest (fewer than 32) to the front
      int own2 = 0;
      double e[4] = {0.0, 0.0, 0.0, 0.0};
      if (lane < nq) {
        own2 = W.qown[32 + lane];
#pragma unroll
        for (int q = 0; q < 4; ++q) e[q] = W.qd[q][32 + lane];
      }
      __syncwarp();
      if (lane < nq) {
        W.qown[lane] = own2;
#pragma unroll
        for (int q = 0; q < 4; ++q) W.qd[q][lane] = e[q];
      }
      __syncwarp();
    }
  }
  if (nq > 0) wca_flush(B, W, nq, lane);
  if (valid) {
#pragma unroll
    for (int q = 0; q < 3; ++q) B.bF[3 * b + q] = F[q] + W.F[q][lane];
  }
}

// First half of a velocity-Verlet substep: half kick, drift (periodic), and
// the check whether the list still covers every pair within the cutoff.
// With close_prev, the closing half kick of the previous substep comes first
// (the same force, added as a separate step, as the substeps are written).
__global__ void __launch_bounds__(WCA_THREADS) k_wca_kick_drift(const BoxDev* __restrict__ boxes, const int2* __restrict__ tiles,
                                 int substep, int close_prev) {
  for_tile_beads(boxes, tiles, [&](const BoxDev& B, int b) {
    if (substep >= B.md_substeps) return;
    double m2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double v = B.svel[3 * b + k];
      if (close_prev) v = v + B.md_hh * B.bF[3 * b + k];
      v = v + B.md_hh * B.bF[3 * b + k];
      const double r = wrap(B.spos[3 * b + k] + B.md_h * v, B.L[k]);
      B.svel[3 * b + k] = v;
      B.spos[3 * b + k] = r;
      const double d = min_image(r - B.nl_rb[3 * b + k], B.L[k]);
      m2 += d * d;
    }
    if (m2 > B.wca_half_skin2) *B.nl_stale = 1;
  });
}

// Closing half kick of a box's last substep (its force is the last one computed).
__global__ void __launch_bounds__(WCA_THREADS) k_wca_kick(const BoxDev* __restrict__ boxes, const int2* __restrict__ tiles) {
  for_tile_beads(boxes, tiles, [&](const BoxDev& B, int b) {
    if (B.md_substeps <= 0) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) B.svel[3 * b + k] = B.svel[3 * b + k] + B.md_hh * B.bF[3 * b + k];
  });
}

// The whole solute MD of one collision step for the boxes with the repulsion.
void launch_wca_md(const BoxDev* boxes, const int2* tiles, int ntiles, int max_substeps, int* err,
                   cudaStream_t s) {
  if (ntiles <= 0) return;
  k_wca_clear<<<ntiles * WCA_SPLIT, WCA_THREADS, 0, s>>>(boxes, tiles, 1);
  k_wca_insert<<<ntiles * WCA_SPLIT, WCA_THREADS, 0, s>>>(boxes, tiles, 1);
  k_wca_list<<<ntiles * WCA_SPLIT, WCA_THREADS, 0, s>>>(boxes, tiles, 1, err);
  k_wca_force<<<ntiles * WCA_SPLIT, WCA_THREADS, 0, s>>>(boxes, tiles, 0);
  // substep sub: kick-drift (closing substep sub - 1 first), rebuild where
  // stale, force; the last substep's closing kick is a launch of its own, and
  // so is that of a box whose md_substeps is below the largest
  for (int sub = 0; sub < max_substeps; ++sub) {
    k_wca_kick_drift<<<ntiles * WCA_SPLIT, WCA_THREADS, 0, s>>>(boxes, tiles, sub, sub > 0);
    k_wca_clear<<<ntiles * WCA_SPLIT, WCA_THREADS, 0, s>>>(boxes, tiles, 0);  // rebuild where stale
    k_wca_insert<<<ntiles * WCA_SPLIT, WCA_THREADS, 0, s>>>(boxes, tiles, 0);
    k_wca_list<<<ntiles * WCA_SPLIT, WCA_THREADS, 0, s>>>(boxes, tiles, 0, err);
    k_wca_force<<<ntiles * WCA_SPLIT, WCA_THREADS, 0, s>>>(boxes, tiles, sub + 1);
  }
  k_wca_kick<<<ntiles * WCA_SPLIT, WCA_THREADS, 0, s>>>(boxes, tiles);
}

}  // namespace mpcd
