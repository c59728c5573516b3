// k_cells_warp.cu -- the fused SRD step of the mixed model with the members of
// 32 cells spread over the 32 lanes of a warp (arXiv:1801.10187: Sec. 2 Eqs.
// stream, srd and thermo; Sec. 3.4 cell list; Sec. 3.5 cell properties;
// Sec. 3.6 rotation and thermostat, algorithm "SRD collision rule").
//
// Same modes, records and results as k_cells (one thread per cell), for boxes
// without walls or solute.  A warp owns 32 consecutive cells.  Their row
// members are numbered 0 .. N-1 in cell order (a warp prefix sum of the row
// counts) and lane j takes members j, j + 32, ...: every lane is busy and a
// warp reads neighbouring records together, whatever the occupancy spread.
//   pass 1   each member's rne(v 2^32) = H 2^20 + L (two int32 parts from two
//            magic-number roundings) is summed per cell with segmented warp
//            reductions (redux.sync over the lanes of one cell); the sums are
//            exact, so u is the one of the per-cell loop
//   cell     lane c turns the sums of cell c into u, draws the axis (and with
//            the thermostat, after a second segmented pass for the energy
//            about u, the factor xi) and leaves them in shared memory
//   pass 2   each member collides with its cell's parameters, streams, is
//            binned under the next shift and appended to its new row
// Members beyond the row capacity (overflow list) stay with the lane of their
// cell, as in k_cells.  The int32 parts stay in range while K <= 448 and
// |v| < 1024; larger velocities take an exact int64 path through shared memory.
#include "dev_collide.cuh"
#include "dev_rows.cuh"
#include "dev_stream.cuh"
#include "kernels.h"
#include "mpcd_internal.cuh"

namespace mpcd {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int WARPS = BLOCK / 32;

struct WarpShared {
  int h[3][32];          // sum over the cell of H (momentum); h[0] reused for the energy
  int l[3][32];          // sum of L
  long long x[4][32];    // exact int64 sums of out-of-range members (momentum, energy)
  float4 prm[2][32];     // (u, xi), (axis, 0) per cell
  unsigned char own[32]; // lane of the cell whose first member sits at each window slot
};

__device__ __forceinline__ void add_split(float v, int& H, int& L, long long* slow) {
  if (!split32(v, H, L)) {
    atomicAdd(reinterpret_cast<unsigned long long*>(slow), (unsigned long long)fix32_rne(v));
    H = 0;
    L = 0;
  }
}

}  // namespace

template <bool THERMO, int MODE>
__global__ void __launch_bounds__(BLOCK, 4) k_cells_warp(const BoxDev* __restrict__ boxes,
                                                         const int2* __restrict__ spans,
                                                         int nspans, int* err) {
  using R = RecF;
  __shared__ WarpShared shw[WARPS];
  __shared__ long long sSn[3];
  const int lane = threadIdx.x & 31;
  WarpShared& W = shw[threadIdx.x >> 5];
  for (int sp = blockIdx.x; sp < nspans; sp += gridDim.x) {
    const int2 tt = spans[sp];
    const BoxDev& B = boxes[tt.x];
    const unsigned long long t = B.step;
    __syncthreads();
    if (threadIdx.x == 0 && MODE != MODE_C) shift_units(B, MODE == MODE_P ? t : t + 1ull, sSn);
    __syncthreads();
    const int c0 = tt.y + (int)(threadIdx.x & ~31u);
    if (c0 >= B.ncells) continue;  // warp-uniform
    const int cell = c0 + lane;
    const bool valid = cell < B.ncells;
    const int cur = B.cur, out = cur ^ 1;
    const int K = B.K;
    const uint32_t n = valid ? B.cnt[cur][cell] : 0u;
    if (MODE != MODE_C && n) B.cnt[cur][cell] = 0u;  // this set is written two steps on
    const int nrow = (int)n < K ? (int)n : K;
    const bool has_ovf = (int)n > K;
    int incl = nrow;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += y;
    }
    const int off = incl - nrow;
    const int N = __shfl_sync(FULL, incl, 31);
    R* rows = ((R*)B.rows[cur]) + (size_t)c0 * K;
    const R* ovf = (const R*)B.ovf_rec[cur];
    const uint32_t* ovf_cell = B.ovf_cell[cur];
    const uint32_t novf =
        __any_sync(FULL, has_ovf) ? min(B.ovf_n[cur], (uint32_t)B.ovf_cap) : 0u;

    // Visit the row members in windows of 32: f(o, k, act, seg, head) gets the
    // owning lane o, the slot k in its row, whether the lane holds a member,
    // the mask of the lanes of the same cell in this window and whether this
    // lane is the first of them.
    auto members = [&](auto&& f) {
      int carry = 0;
      for (int base = 0; base < N; base += 32) {
        const int rel = off - base;
        const bool st = nrow > 0 && rel >= 0 && rel < 32;
        if (st) W.own[rel] = (unsigned char)lane;
        const unsigned sb = __reduce_or_sync(FULL, st ? (1u << rel) : 0u);
        __syncwarp();
        const unsigned upto = FULL >> (31 - lane);  // bits 0 .. lane
        const unsigned le = sb & upto;
        const int lo = le ? 31 - __clz(le) : 0;
        const int o = le ? (int)W.own[lo] : carry;
        const unsigned gt = sb & ~upto;
        const int hi = gt ? __ffs(gt) - 2 : 31;
        const unsigned seg = ((2u << hi) - 1u) & ~((1u << lo) - 1u);
        const int k = base + lane - __shfl_sync(FULL, off, o);
        f(o, k, base + lane < N, seg, lane == lo);
        carry = __shfl_sync(FULL, o, 31);
        __syncwarp();
      }
    };

    if (MODE != MODE_P) {
      // ---- pass 1: exact momentum sums per cell (Sec. 3.5) ----
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        W.h[q][lane] = 0;
        W.l[q][lane] = 0;
        W.x[q][lane] = 0;
      }
      W.x[3][lane] = 0;
      __syncwarp();
      members([&](int o, int k, bool act, unsigned seg, bool head) {
        int H[3] = {0, 0, 0}, L[3] = {0, 0, 0};
        if (act) {
          const float* p = reinterpret_cast<const float*>(rows + (size_t)o * K + k);
          const float v0 = p[3];
          const float2 v12 = *reinterpret_cast<const float2*>(p + 4);
          add_split(v0, H[0], L[0], &W.x[0][o]);
          add_split(v12.x, H[1], L[1], &W.x[1][o]);
          add_split(v12.y, H[2], L[2], &W.x[2][o]);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int sh = __reduce_add_sync(seg, H[q]);
          const int sl = __reduce_add_sync(seg, L[q]);
          if (head) {
            W.h[q][o] += sh;
            W.l[q][o] += sl;
          }
        }
      });
      __syncwarp();

      // ---- per cell: u, then (thermostat) the energy about u, axis, xi ----
      CellAcc<true> a;
      float u[3] = {0.0f, 0.0f, 0.0f};
      if (n > 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q)
          a.q[q] = (long long)W.h[q][lane] * 1048576LL + (long long)W.l[q][lane] + W.x[q][lane];
        if (has_ovf)
          for (uint32_t j = 0; j < novf; ++j)
            if (ovf_cell[j] == (uint32_t)cell) {
              float w[3];
              load_v(ovf + j, w);
#pragma unroll
              for (int q = 0; q < 3; ++q) a.q[q] += fix32_rne(w[q]);
            }
        a.ns = (int)n;
        a.mean_velocity(B, u, false);
        W.prm[0][lane] = make_float4(u[0], u[1], u[2], 1.0f);
      }
      if (THERMO) {
        W.h[0][lane] = 0;
        W.l[0][lane] = 0;
        __syncwarp();
        members([&](int o, int k, bool act, unsigned seg, bool head) {
          int H = 0, L = 0;
          if (act) {
            const float* p = reinterpret_cast<const float*>(rows + (size_t)o * K + k);
            const float v0 = p[3];
            const float2 v12 = *reinterpret_cast<const float2*>(p + 4);
            const float4 uo = W.prm[0][o];
            const float d0 = v0 - uo.x, d1 = v12.x - uo.y, d2 = v12.y - uo.z;
            const float e = d0 * d0 + d1 * d1 + d2 * d2;
            add_split(e, H, L, &W.x[3][o]);
          }
          const int sh = __reduce_add_sync(seg, H);
          const int sl = __reduce_add_sync(seg, L);
          if (head) {
            W.h[0][o] += sh;
            W.l[0][o] += sl;
          }
        });
        __syncwarp();
        if (n > 0) {
          a.es = (long long)W.h[0][lane] * 1048576LL + (long long)W.l[0][lane] + W.x[3][lane];
          if (has_ovf)
            for (uint32_t j = 0; j < novf; ++j)
              if (ovf_cell[j] == (uint32_t)cell) {
                float w[3];
                load_v(ovf + j, w);
                a.add_solvent_energy(B, w, u);
              }
        }
      }
      CellParams<float> prm;
      if (n > 0) {
        auto no_beads = [](int, int&) { return false; };
        cell_finish<true>(B, t, (uint32_t)cell, a, u, 0, no_beads, THERMO, false, prm, err);
        W.prm[0][lane] = make_float4(prm.u[0], prm.u[1], prm.u[2], prm.xi);
        W.prm[1][lane] = make_float4(prm.n[0], prm.n[1], prm.n[2], 0.0f);
      }
      __syncwarp();
    }

    // ---- pass 2: collide (Eq. srd), stream (Eq. stream), bin (Sec. 3.4) ----
    auto process = [&](R* p, const CellParams<float>& prm) {
      float r[3], w[3];
      uint32_t tag;
      load_rec(p, r, w, tag);
      if (MODE != MODE_P) collide_one<true>(B, prm, w, THERMO);
      if (MODE == MODE_C) {
        store_rec(p, r, w, tag);
        return;
      }
      stream_one(B, r, w);
      const uint32_t c2 = cell_of(B, sSn, r, err);
      insert<true>(B, out, c2, r, w, tag, err);
    };
    auto params_of = [&](int o) {
      CellParams<float> prm;
      if (MODE != MODE_P) {
        const float4 a = W.prm[0][o], b = W.prm[1][o];
        prm.u[0] = a.x; prm.u[1] = a.y; prm.u[2] = a.z; prm.xi = a.w;
        prm.n[0] = b.x; prm.n[1] = b.y; prm.n[2] = b.z;
      }
      return prm;
    };
    members([&](int o, int k, bool act, unsigned, bool) {
      if (act) process(rows + (size_t)o * K + k, params_of(o));
    });
    if (has_ovf) {
      const CellParams<float> prm = params_of(lane);
      for (uint32_t j = 0; j < novf; ++j)
        if (ovf_cell[j] == (uint32_t)cell) process(((R*)B.ovf_rec[cur]) + j, prm);
    }
  }
}

template <bool TH, int MODE>
static void* warp_fn() {
  return (void*)k_cells_warp<TH, MODE>;
}

static void* warp_variant(bool thermo, int mode) {
  if (mode == MODE_P) return thermo ? warp_fn<true, MODE_P>() : warp_fn<false, MODE_P>();
  if (mode == MODE_F) return thermo ? warp_fn<true, MODE_F>() : warp_fn<false, MODE_F>();
  return thermo ? warp_fn<true, MODE_C>() : warp_fn<false, MODE_C>();
}

int cells_warp_blocks_per_sm(bool thermo, int mode) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, warp_variant(thermo, mode), BLOCK, 0);
  return nb;
}

void launch_cells_warp(bool thermo, int mode, const BoxDev* boxes, const int2* spans, int nspans,
                       int grid, int* err, cudaStream_t s) {
  if (nspans <= 0) return;
  void* args[] = {(void*)&boxes, (void*)&spans, (void*)&nspans, (void*)&err};
  cudaLaunchKernel(warp_variant(thermo, mode), dim3(grid), dim3(BLOCK), args, 0, s);
}

}  // namespace mpcd
