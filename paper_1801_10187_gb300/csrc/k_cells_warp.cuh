// k_cells_warp.cuh -- the fused SRD step of the mixed model with the members of
// a warp's cells spread over its 32 lanes (arXiv:1801.10187: Sec. 2 Eqs.
// stream, srd and thermo; Sec. 3.4 cell list; Sec. 3.5 cell properties;
// Sec. 3.6 rotation and thermostat, algorithm "SRD collision rule").
//
// Same modes, records and results as k_cells (one thread per cell), for boxes
// without walls (solute beads allowed).  A warp owns 32 consecutive cells (or
// 16 or 8, a launch-tuner choice; see CPW below).  Their row members are
// numbered 0 .. N-1 in cell order (a warp prefix sum of the row counts); a
// byte map gives each member's cell.
//   pass 1   the (v, tag) words of up to 192 members are copied into shared
//            memory asynchronously in member order (neighbouring lanes,
//            neighbouring records), issued as soon as the counts are scanned
//            so that they land while the bead counts and the per-cell draws
//            compute (the Andersen and angular variants load up to 256
//            velocities in windows of registers instead); then lane j takes a
//            consecutive share of them, so its members lie in one or two
//            cells.  Each velocity component gives rne(v 2^32) = H 2^20 + L,
//            two int32 parts from two magic-number roundings, summed in
//            registers while the cell stays the same and added to the cell's
//            shared sums by one atomic per part when it changes.  The sums
//            are exact, so u is the one of any order.
//   cell     lane c turns the sums of cell c into u and, with the thermostat,
//            into E_k (one pass, Sec. 3.5: pass 1 also sums the exact second
//            moment of the split velocities) and the factor xi; the axis and
//            the Gamma pair were drawn before pass 1 (they need only the
//            member count).  u, xi and the axis go to shared memory
//   pass 2   members in order across the lanes, in chunks of two to four
//            windows of 32: the chunk's records are copied into shared memory
//            asynchronously (all in flight at once), each is collided with its
//            cell's parameters, streamed and binned under the next shift while
//            its slot in the new row is requested (atomic on the row count),
//            and the records are written once every request of the chunk is
//            out
// The parameters a member needs (time step, box, rotation, the thresholds of
// the next grid shift, row pointers) are staged in shared memory when a block
// meets a new box.  Members beyond the row capacity (overflow list) stay with the lane
// of their cell, as in k_cells.  The int32 parts stay in range while K <= 448
// and |v| < 1024; a warp that meets a larger velocity (or energy) sums its
// cells again in int64, one lane per cell.
//
// The Andersen-thermostat variant (Eq. at, Sec. 3.7) has the same passes:
// pass 1 also sums each member's Gaussian random velocity dv (drawn from its
// tag) in the same exact split form, the cell phase forms the mass-weighted
// mean dv of the cell, and pass 2 draws dv again and sets v = (u + dv) - dbar.
#pragma once
#include "dev_angular.cuh"
#include "dev_bin.cuh"
#include "dev_collide.cuh"
#include "dev_rows.cuh"
#include "dev_stream.cuh"
#include "kernels.h"
#include "mpcd_internal.cuh"

namespace mpcd {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int WARPS = BLOCK / 32;

constexpr int MAP_MEMBERS = 640;  // members per warp with a byte owner map
constexpr int STAGE = 256;        // member velocities staged per block of pass 1
constexpr int STAGE4 = 192;       // the same for the SRD variants (whole 16-byte words)
constexpr int STAGE_PAD = STAGE + STAGE / 32;
constexpr int CHUNK = 3;          // windows of 32 members per chunk of pass 2 (default)

// The wait for all of this thread's outstanding asynchronous copies (16-byte
// global -> shared copies that bypass L1, issued below with an L2 policy).
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Exact int64 momentum and kinetic-energy sums of the beads in each of a
// warp's cells (bead variants), kept in the staging buffer during the cell
// phase (see BeadShared).
struct BeadSums {
  unsigned long long X[3][32];
  unsigned long long E[32];
};

// CH: windows of 32 members per chunk of pass 2 (the launch tuner picks 2, 3
// or 4 for the F mode of the SRD variants; 3 elsewhere).
template <int CH>
struct WarpShared {
  float4 prm[2][32];               // (u, xi), (axis, 0) per cell
  float2 gdv[32];                  // thermostat: accepted Gamma pair (d, v); d < 0: none
  int h[3][32];                    // sum over the cell of H (momentum)
  int l[3][32];                    // sum of L
  int offs[33];                    // first member of each cell; offs[32] = members
  int pad_[3];
  unsigned char map[MAP_MEMBERS];  // owner lane of each member
  union {
    float sv[3][STAGE_PAD];        // pass 1: staged velocities (index j + j / 32)
    float4 sv4[STAGE4];            // pass 1 of the SRD variants: staged (v, tag)
    BeadSums bx;                   // cell phase (bead variants): the beads' exact sums
    float4 buf[CH][2][32];         // pass 2: records of one chunk (two halves)
  };
};

// Thermostat variants: the exact second moment of each cell's split
// velocities, sum over members and components of H^2, H L and L^2 (V = H 2^20
// + L, so sum V^2 = 2^40 sum H^2 + 2^21 sum H L + sum L^2).
//
// A lane adds its partial P of a moment (an int64) as two 32-bit shared
// atomics instead of one 64-bit one, P = (P >> 24) 2^24 + (P & (2^24 - 1)).
// Both sums stay exact: a lane's share is at most 8
// members (24 terms: |h| < 2^22, |l| <= 2^19), so |P >> 24| < 2^24.6 for H^2,
// 2^21.6 for H L and 2^18.6 for L^2, and a cell of at most 448 members takes at
// most 4 staged blocks of 32 lane shares, 128 partials: the high sums stay
// below 2^32 (H^2, unsigned) and 2^29 in magnitude (the others), the low sums
// below 2^31.
struct ThermoShared {
  unsigned hh_lo[32], hh_hi[32];
  unsigned hl_lo[32];
  int hl_hi[32];
  unsigned ll_lo[32], ll_hi[32];
};

// Per-cell bead accumulators of one warp (bead variants only): the bead count
// of each of the 32 cells (before the draws, which need it), and their exact
// int64 momentum and kinetic-energy sums (after pass 1, in the staging
// buffer, which pass 1 no longer needs and pass 2 has not yet taken).
struct BeadShared {
  int nb[32];
};

// Andersen-rule accumulators of one warp: split sums of the random
// velocities per cell, the tags of the staged members, the beads' exact int64
// random momenta, and the random velocities of the first DV_CAP members
// (index m + m / 32), drawn once in pass 1 and used again in pass 2.  Members
// beyond DV_CAP draw theirs again in pass 2.
template <int DV_CAP>
struct ATShared {
  int h[3][32];
  int l[3][32];
  uint32_t tag[STAGE_PAD];
  unsigned long long DX[3][32];
  float dv[3][DV_CAP + DV_CAP / 32];
};
constexpr int DV_CAP = 448;        // cached members per warp
constexpr int DV_CAP_BEADS = 320;  // with the bead accumulators (two blocks per SM fit)

// Shared memory of one block: the span parameters, then one area per warp;
// kept under 48 KB so that four blocks (the register limit) fit on an SM with
// room left for L1.
template <int CH>
constexpr size_t WARP_SMEM = sizeof(WarpShared<CH>);

// Per-span parameters shared by the block.
struct SpanParams {
  float dt, ca, sa, omc, m;
  float L[3], hg[3], gdt[3];
  float lo[3], hi[3];  // binning thresholds of the next grid shift (see bin_axis)
  int n[3], K;
  RecF* rows_cur;
  RecF* rows_out;
  uint32_t* cnt_out;
  RecF* ovf_out;
  uint32_t* ovf_cell_out;
  uint32_t* ovf_n_out;
  int ovf_cap, pad;
};
constexpr size_t SPAN_SMEM = (sizeof(SpanParams) + 15) & ~(size_t)15;
template <int CH>
constexpr size_t BLOCK_SMEM = SPAN_SMEM + WARPS * WARP_SMEM<CH>;

// Angular-momentum correction (SRD without beads): the float
// frame of the collision step's shift (per block), and per warp the staged
// relative positions of the members, split sums per cell of the positions,
// of r_c x (v - v') and of the six inertia-tensor entries, and per cell the
// centre of mass and omega.
struct AngBlock {
  float sf[3], lo[3], hi[3];
  int pad_[3];
};
struct AngWarp {
  float sr[3][STAGE_PAD];
  int qh[3][32], ql[3][32];
  int lh[3][32], ll[3][32];
  int ph[6][32], pl[6][32];
  float4 rc[32];  // (centre of mass in the cell frame, 0)
  float4 om[32];  // (omega, 0)
};

template <int CH = CHUNK>
__host__ __device__ constexpr size_t block_smem(bool beads, bool at, bool ang = false,
                                                bool thermo = false) {
  return BLOCK_SMEM<CH> + (beads ? WARPS * sizeof(BeadShared) : 0) +
         (at ? WARPS * (beads ? sizeof(ATShared<DV_CAP_BEADS>) : sizeof(ATShared<DV_CAP>)) : 0) +
         (ang ? sizeof(AngBlock) + WARPS * sizeof(AngWarp) : 0) +
         (thermo ? WARPS * sizeof(ThermoShared) : 0);
}

}  // namespace

// The SRD variants run four blocks per SM (64 registers); the thermostat
// variants then spill about 50 bytes, which costs less than the fourth block
// gains (measured).  With the beads' sums in the staging buffer during the
// cell phase, four blocks of the thermostat and bead variant fit in shared
// memory.
// AT selects the Andersen rule (then THERMO is false): its two Box-Muller
// draws per member want registers for independent chains, and its cache of
// random velocities wants shared memory, so it runs two blocks per SM.
// CPW: cells per warp (32, or 16 or 8 for the F mode of the SRD variants, a
// launch-tuner choice).  A warp of CPW < 32 cells leaves lanes CPW..31
// without a cell (they still take members in the member passes); a 256-cell
// span is then taken in 32 / CPW parts, each by one block, which puts more
// blocks on a small box.  Results do not depend on CPW (exact sums).
// ANG adds the angular-momentum correction to SRD, with or without the
// thermostat (then BEADS and AT are false); its shared memory allows two
// blocks per SM.
template <bool THERMO, int MODE, bool FORCE, bool BEADS, bool AT, bool ANG, int CH = CHUNK,
          int CPW = 32>
__global__ void __launch_bounds__(BLOCK, (AT || ANG) ? 2 : 4) k_cells_warp(const BoxDev* __restrict__ boxes,
                                                         const int2* __restrict__ spans,
                                                         int nspans, int* err) {
  using R = RecF;
  extern __shared__ __align__(16) unsigned char smem_[];
  SpanParams& sp_ = *reinterpret_cast<SpanParams*>(smem_);
  const int lane = threadIdx.x & 31;
  WarpShared<CH>& W =
      reinterpret_cast<WarpShared<CH>*>(smem_ + SPAN_SMEM)[threadIdx.x >> 5];
  BeadShared& BS = reinterpret_cast<BeadShared*>(smem_ + BLOCK_SMEM<CH>)[threadIdx.x >> 5];
  constexpr int DVC = BEADS ? DV_CAP_BEADS : DV_CAP;
  ATShared<DVC>& AS = reinterpret_cast<ATShared<DVC>*>(smem_ + block_smem<CH>(BEADS, false))[threadIdx.x >> 5];
  AngBlock& AB = *reinterpret_cast<AngBlock*>(smem_ + block_smem<CH>(BEADS, AT));
  AngWarp& AG = reinterpret_cast<AngWarp*>(smem_ + block_smem<CH>(BEADS, AT) + sizeof(AngBlock))[threadIdx.x >> 5];
  ThermoShared& TS = reinterpret_cast<ThermoShared*>(smem_ + block_smem<CH>(BEADS, AT, ANG))[threadIdx.x >> 5];
  const SpanParams& H = sp_;
  // SRD variants stage pass 1 by asynchronous copies issued early (above);
  // the Andersen and angular variants load and convert in stage()
  constexpr bool EARLY = !AT && !ANG;
  constexpr int SB = EARLY ? STAGE4 : STAGE;
  int box_of_params = -1;  // the span parameters depend on the box only
  static_assert(CPW == 32 || CPW == 16 || CPW == 8, "cells per warp");
  constexpr int PARTS = 32 / CPW;  // parts of a 256-cell span
  for (int it = blockIdx.x; it < nspans * PARTS; it += gridDim.x) {
    const int sp = it / PARTS, part = it - sp * PARTS;
    const int2 tt = spans[sp];
    const BoxDev& B = boxes[tt.x];
    const unsigned long long t = B.step;
    if (tt.x != box_of_params) {  // block-uniform
      __syncthreads();
      if (threadIdx.x == 0) {
        SpanParams& P = sp_;
        P.dt = B.dt_f; P.ca = B.ca_f; P.sa = B.sa_f; P.omc = B.omc_f; P.m = B.m_f;
        for (int q = 0; q < 3; ++q) {
          P.L[q] = B.L_f[q]; P.hg[q] = B.hg_f[q]; P.gdt[q] = B.gdt_f[q]; P.n[q] = B.n[q];
        }
        P.K = B.K;
        const int out = B.cur ^ 1;
        P.rows_cur = (RecF*)B.rows[B.cur];
        P.rows_out = (RecF*)B.rows[out];
        P.cnt_out = B.cnt[out];
        P.ovf_out = (RecF*)B.ovf_rec[out];
        P.ovf_cell_out = B.ovf_cell[out];
        P.ovf_n_out = &B.ovf_n[out];
        P.ovf_cap = B.ovf_cap;
        if (MODE != MODE_C) {
          long long S[3];
          shift_units(B, MODE == MODE_P ? t : t + 1ull, S);
          for (int q = 0; q < 3; ++q) bin_thresholds(S[q], P.lo[q], P.hi[q]);
        }
        if (ANG && MODE != MODE_P) {  // frame of the collision step's cells
          long long S[3];
          shift_units(B, t, S);
          for (int q = 0; q < 3; ++q) shift_thresholds(S[q], AB.sf[q], AB.lo[q], AB.hi[q]);
        }
      }
      __syncthreads();
      box_of_params = tt.x;
    }
    const int c0 = tt.y + part * (WARPS * CPW) + (int)(threadIdx.x >> 5) * CPW;
    if (c0 >= B.ncells) continue;  // warp-uniform
    const int cell = c0 + lane;
    const bool valid = (CPW == 32 || lane < CPW) && cell < B.ncells;
    const int cur = B.cur;
    const int K = H.K;
    const uint32_t n = valid ? B.cnt[cur][cell] : 0u;
    // the bead group's bounds, loaded together with the row counts
    int gb0 = 0, gb1 = 0;
    if (BEADS && MODE != MODE_P) {
      const int g = c0 / B.tc;
      gb0 = (int)B.bstart[g];
      gb1 = (int)B.bstart[g + 1];
    }
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
    __syncwarp();  // the previous span of this warp is done with W
    W.offs[lane + 1] = incl;
    if (lane == 0) W.offs[0] = 0;
    R* rows = H.rows_cur + (size_t)c0 * K;
    const R* ovf = (const R*)B.ovf_rec[cur];
    const uint32_t* ovf_cell = B.ovf_cell[cur];
    const uint32_t novf =
        __any_sync(FULL, has_ovf) ? min(B.ovf_n[cur], (uint32_t)B.ovf_cap) : 0u;
    // owner lane of member m: a byte map for up to MAP_MEMBERS members, else a
    // binary search of the offsets (the last cell whose first member is <= m)
    const bool mapped = N <= MAP_MEMBERS;
    if (mapped)
      for (int j = 0; j < nrow; ++j) W.map[off + j] = (unsigned char)lane;
    __syncwarp();
    auto owner_of = [&](int m) -> int {
      if (mapped) return W.map[m];
      int lo = 0, hi = 32;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (W.offs[mid] <= m) lo = mid;
        else hi = mid;
      }
      return lo;
    };
    auto member = [&](int m, int o) -> R* { return rows + (size_t)o * K + (m - W.offs[o]); };
    // Velocities of members [sbase, sbase + cnt) into shared memory, read in
    // member order (neighbouring lanes, neighbouring records).
    auto stage = [&](int sbase, int cnt) {
      for (int j0 = 0; j0 < cnt; j0 += 128) {  // four windows of loads in flight
        float4 a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + (u << 5) + lane;
          if (j < cnt) a[u] = *reinterpret_cast<const float4*>(member(sbase + j, owner_of(sbase + j)));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + (u << 5) + lane;
          if (j < cnt) {
            const int js = j + (j >> 5);
            W.sv[0][js] = a[u].x;
            W.sv[1][js] = a[u].y;
            W.sv[2][js] = a[u].z;
            if (AT) AS.tag[js] = __float_as_uint(a[u].w);
          }
        }
        if (ANG && MODE != MODE_P) {  // positions relative to the collision cell
          float4 b[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = j0 + (u << 5) + lane;
            if (j < cnt) b[u] = reinterpret_cast<const float4*>(member(sbase + j, owner_of(sbase + j)))[1];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = j0 + (u << 5) + lane;
            if (j < cnt) {
              const int js = j + (j >> 5);
              AG.sr[0][js] = rel_pos_f(b[u].x, AB.sf[0], AB.lo[0], AB.hi[0]);
              AG.sr[1][js] = rel_pos_f(b[u].y, AB.sf[1], AB.lo[1], AB.hi[1]);
              AG.sr[2][js] = rel_pos_f(b[u].z, AB.sf[2], AB.lo[2], AB.hi[2]);
            }
          }
        }
        if (AT && MODE != MODE_P) {  // Eq. at: random velocities of the cached members
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = j0 + (u << 5) + lane, m = sbase + j;
            if (j < cnt && m < DVC) {
              float dv[3];
              at_draw(B, t, __float_as_uint(a[u].w), 0u, B.sig_f, dv);
              const int mp = m + (m >> 5);
              AS.dv[0][mp] = dv[0];
              AS.dv[1][mp] = dv[1];
              AS.dv[2][mp] = dv[2];
            }
          }
        }
      }
      __syncwarp();
    };
    // This lane's consecutive share of a staged block: f(o, j, last) with the
    // owner lane o, the index j in the block and whether it is the last of
    // the share in cell o.
    auto share = [&](int sbase, int cnt, auto&& f) {
      const int cs = (lane * cnt) >> 5, ce = ((lane + 1) * cnt) >> 5;
      if (cs >= ce) return;
      int o = owner_of(sbase + cs);
      int cend = W.offs[o + 1] - sbase;
      for (int j = cs; j < ce; ++j) {
        if (j == cend) {
          do {
            ++o;
            cend = W.offs[o + 1] - sbase;
          } while (cend == j);
        }
        f(o, j, j + 1 == cend || j + 1 == ce);
      }
    };

    // SRD variants: the (v, tag) words of members [sbase, sbase + cnt) are
    // copied into shared memory asynchronously.  The first block is issued
    // here, before the bead sums and the per-cell draws, which need none of
    // it, so its load latency passes while they compute.
    auto stage_async = [&](int sbase, int cnt) {
      for (int j = lane; j < cnt; j += 32)
        cp_async16(&W.sv4[j], member(sbase + j, owner_of(sbase + j)));
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (EARLY && MODE != MODE_P) stage_async(0, min(STAGE4, N));

    // Solute beads join their cell's collision with mass M (Sec. 3.6).  The
    // warp's cells lie in one bead group of 32 cells (all of it when CPW is
    // 32); the group's beads are handled one per lane (grouped copies of cell
    // and velocity), those of this warp's cells only: first their count and
    // exact int64 momentum per cell, into shared sums.
    const int gnb = gb1 - gb0;
    int nb = 0;
    auto for_beads = [&](auto&& f) {  // f(slot in the group order, local cell)
      for (int j0 = 0; j0 < gnb; j0 += 32) {
        const int j = gb0 + j0 + lane;
        if (j0 + lane < gnb) {
          const int lc = B.bgc[j] - c0;  // beads of the group's other cells: another warp's
          if (CPW == 32 || (unsigned)lc < (unsigned)CPW) f(j, lc);
        }
      }
    };
    if (BEADS && MODE != MODE_P) {
      if (gnb > 0) {
        BS.nb[lane] = 0;
        __syncwarp();
        for_beads([&](int, int lc) { atomicAdd(&BS.nb[lc], 1); });
        __syncwarp();
        nb = BS.nb[lane];
      }
    }
    // The per-cell draws of the step need only the member count, so they
    // come before the sums (less state is live here): the axis (Sec. 3.6)
    // and, with the thermostat, the accepted Gamma pair (d, v), E^ = d v kT.
    if (MODE != MODE_P && !AT && (n > 0 || nb > 0)) {
      float ax[3];
      axis_of(B, t, (uint32_t)cell, ax);
      W.prm[1][lane] = make_float4(ax[0], ax[1], ax[2], 0.0f);
      if (THERMO) {
        float d = -1.0f, v = 0.0f;
        if ((int)n + nb >= 2 && !gamma_draw_mixed(B, t, (uint32_t)cell, (int)n + nb, d, v))
          d = -1.0f;
        W.gdv[lane] = make_float2(d, v);
      }
    }

    if (MODE != MODE_P) {
      // ---- pass 1: exact momentum sums per cell (Sec. 3.5) ----
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        W.h[q][lane] = 0;
        W.l[q][lane] = 0;
        if (AT) {
          AS.h[q][lane] = 0;
          AS.l[q][lane] = 0;
        }
        if (ANG) {
          AG.qh[q][lane] = 0;
          AG.ql[q][lane] = 0;
        }
      }
      if (THERMO) {
        TS.hh_lo[lane] = 0u;
        TS.hh_hi[lane] = 0u;
        TS.hl_lo[lane] = 0u;
        TS.hl_hi[lane] = 0;
        TS.ll_lo[lane] = 0u;
        TS.ll_hi[lane] = 0u;
      }
      __syncwarp();
      bool slow = false, slow_d = false;
      for (int sbase = 0; sbase < N; sbase += SB) {
        const int cnt = min(SB, N - sbase);
        if (EARLY) {
          if (sbase > 0) stage_async(sbase, cnt);
          cp_async_wait_all();
          __syncwarp();  // every lane's copies are in shared memory
        } else {
          stage(sbase, cnt);
        }
        int Hs[3] = {0, 0, 0}, Ls[3] = {0, 0, 0};
        int Hd[3] = {0, 0, 0}, Ld[3] = {0, 0, 0};
        int Hq[3] = {0, 0, 0}, Lq[3] = {0, 0, 0};
        long long Shh = 0, Shl = 0, Sll = 0;  // thermostat: second moment
        share(sbase, cnt, [&](int o, int j, bool last) {
          const int js = j + (j >> 5);
          float vm[3];
          if (EARLY) {
            const float4 a = W.sv4[j];
            vm[0] = a.x;
            vm[1] = a.y;
            vm[2] = a.z;
          } else {
            vm[0] = W.sv[0][js];
            vm[1] = W.sv[1][js];
            vm[2] = W.sv[2][js];
          }
          if (ANG) {  // |position in the cell frame| < 2: the split never fails
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              int h, l;
              split32(AG.sr[q][js], h, l);
              Hq[q] += h;
              Lq[q] += l;
            }
          }
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            int h, l;
            if (!split32(vm[q], h, l)) {
              slow = true;
              h = 0;
              l = 0;
            }
            Hs[q] += h;
            Ls[q] += l;
            if (THERMO) {  // Sec. 3.5: the kinetic energy in the same pass, exactly
              Shh += (long long)h * h;
              Shl += (long long)h * l;
              Sll += (long long)l * l;
            }
          }
          if (AT) {  // Eq. at: this member's random velocity, summed the same way
            float dv[3];
            const int m = sbase + j, mp = m + (m >> 5);  // member, padded index
            if (m < DVC) {
              dv[0] = AS.dv[0][mp];
              dv[1] = AS.dv[1][mp];
              dv[2] = AS.dv[2][mp];
            } else {
              at_draw(B, t, AS.tag[js], 0u, B.sig_f, dv);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              int h, l;
              if (!split32(dv[q], h, l)) {
                slow_d = true;
                h = 0;
                l = 0;
              }
              Hd[q] += h;
              Ld[q] += l;
            }
          }
          if (last) {
            if (THERMO) {
              atomicAdd(&TS.hh_lo[o], (unsigned)(Shh & 0xFFFFFFLL));
              atomicAdd(&TS.hh_hi[o], (unsigned)(Shh >> 24));
              atomicAdd(&TS.hl_lo[o], (unsigned)(Shl & 0xFFFFFFLL));
              atomicAdd(&TS.hl_hi[o], (int)(Shl >> 24));
              atomicAdd(&TS.ll_lo[o], (unsigned)(Sll & 0xFFFFFFLL));
              atomicAdd(&TS.ll_hi[o], (unsigned)(Sll >> 24));
              Shh = 0;
              Shl = 0;
              Sll = 0;
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              atomicAdd(&W.h[q][o], Hs[q]);
              atomicAdd(&W.l[q][o], Ls[q]);
              Hs[q] = 0;
              Ls[q] = 0;
              if (AT) {
                atomicAdd(&AS.h[q][o], Hd[q]);
                atomicAdd(&AS.l[q][o], Ld[q]);
                Hd[q] = 0;
                Ld[q] = 0;
              }
              if (ANG) {
                atomicAdd(&AG.qh[q][o], Hq[q]);
                atomicAdd(&AG.ql[q][o], Lq[q]);
                Hq[q] = 0;
                Lq[q] = 0;
              }
            }
          }
        });
        __syncwarp();
      }
      const bool exact64 = __any_sync(FULL, slow);  // a velocity of 1024 or more
      const bool exact64_d = AT && __any_sync(FULL, slow_d);

      // the beads' exact momentum and (with the thermostat) kinetic sums per
      // cell, into the staging buffer that pass 1 is done with
      long long X[3] = {0, 0, 0};
      if (BEADS && gnb > 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) W.bx.X[q][lane] = 0ull;
        W.bx.E[lane] = 0ull;
        __syncwarp();
        for_beads([&](int j, int lc) {
          const double w0 = B.bgv[3 * j], w1 = B.bgv[3 * j + 1], w2 = B.bgv[3 * j + 2];
          atomicAdd(&W.bx.X[0][lc], (unsigned long long)__double2ll_rn((B.Mb * w0) * 4294967296.0));
          atomicAdd(&W.bx.X[1][lc], (unsigned long long)__double2ll_rn((B.Mb * w1) * 4294967296.0));
          atomicAdd(&W.bx.X[2][lc], (unsigned long long)__double2ll_rn((B.Mb * w2) * 4294967296.0));
          if (THERMO)  // kinetic term of the one-pass energy (Sec. 3.5)
            atomicAdd(&W.bx.E[lc], (unsigned long long)__double2ll_rn(
                                       (B.Mb * (w0 * w0 + w1 * w1 + w2 * w2)) * 4294967296.0));
        });
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 3; ++q) X[q] = (long long)W.bx.X[q][lane];
      }

      // ---- per cell: u (Sec. 3.5), then E_k and xi ----
      const bool occupied = n > 0 || nb > 0;
      float u[3] = {0.0f, 0.0f, 0.0f};
      long long Q[3] = {0, 0, 0};  // exact path: this cell's sums of rne(v 2^32)
      __int128 S2x = 0;            // and of their squares (thermostat)
      if (occupied) {
        auto add_v = [&](const float w[3]) {
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const long long V = fix32_rne(w[q]);
            Q[q] += V;
            if (THERMO) S2x += (__int128)V * V;
          }
        };
        if (exact64)
          for (int k = 0; k < nrow; ++k) {
            float w[3];
            load_v(rows + (size_t)lane * K + k, w);
            add_v(w);
          }
        if (has_ovf)
          for (uint32_t j = 0; j < novf; ++j)
            if (ovf_cell[j] == (uint32_t)cell) {
              float w[3];
              load_v(ovf + j, w);
              add_v(w);
            }
        float M = H.m * small_to_float((int)n);
        if (BEADS) M = M + (small_to_float(nb) * B.Mb_f + 0.0f * H.m);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          float P = H.m * (exact64 ? i64_to_float(Q[q])
                                   : split_sum_to_float(W.h[q][lane], W.l[q][lane], Q[q]));
          if (BEADS) P = P + i64_to_float(X[q]);
          u[q] = (P * 0x1p-32f) / M;
        }
        W.prm[0][lane] = make_float4(u[0], u[1], u[2], 1.0f);
      }
      if (AT) {
        // Eq. at: dbar = sum m dv / sum m over the cell's members and beads
        long long DX[3] = {0, 0, 0};
        if (BEADS && gnb > 0) {
#pragma unroll
          for (int q = 0; q < 3; ++q) AS.DX[q][lane] = 0ull;
          __syncwarp();
          for_beads([&](int j, int lc) {
            float dvf[3];
            at_draw(B, t, B.border[j], 1u, B.sigb_f, dvf);
#pragma unroll
            for (int q = 0; q < 3; ++q)
              atomicAdd(&AS.DX[q][lc],
                        (unsigned long long)__double2ll_rn((B.Mb * (double)dvf[q]) * 4294967296.0));
          });
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 3; ++q) DX[q] = (long long)AS.DX[q][lane];
        }
        if (occupied) {
          long long Qd[3] = {0, 0, 0};
          auto add_dv = [&](const R* p) {
            const float4 a = *reinterpret_cast<const float4*>(p);  // (v, tag)
            float dv[3];
            at_draw(B, t, __float_as_uint(a.w), 0u, B.sig_f, dv);
#pragma unroll
            for (int q = 0; q < 3; ++q) Qd[q] += fix32_rne(dv[q]);
          };
          if (exact64_d)
            for (int k = 0; k < nrow; ++k) add_dv(rows + (size_t)lane * K + k);
          if (has_ovf)
            for (uint32_t j = 0; j < novf; ++j)
              if (ovf_cell[j] == (uint32_t)cell) add_dv(ovf + j);
          float M = H.m * small_to_float((int)n);
          if (BEADS) M = M + (small_to_float(nb) * B.Mb_f + 0.0f * H.m);
          float dbar[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            float D = H.m * (exact64_d ? i64_to_float(Qd[q])
                                       : split_sum_to_float(AS.h[q][lane], AS.l[q][lane], Qd[q]));
            if (BEADS) D = D + i64_to_float(DX[q]);
            dbar[q] = (D * 0x1p-32f) / M;
          }
          W.prm[0][lane] = make_float4(u[0], u[1], u[2], 0.0f);
          W.prm[1][lane] = make_float4(dbar[0], dbar[1], dbar[2], 0.0f);
        }
        __syncwarp();
        if (BEADS && gnb > 0) {  // Eq. at for the beads: v = (u + dv) - dbar
          for_beads([&](int j, int lc) {
            const float4 pa = W.prm[0][lc], pb = W.prm[1][lc];
            const uint32_t b = B.border[j];
            float dvf[3];
            at_draw(B, t, b, 1u, B.sigb_f, dvf);
            B.svel[3 * b] = ((double)pa.x + (double)dvf[0]) - (double)pb.x;
            B.svel[3 * b + 1] = ((double)pa.y + (double)dvf[1]) - (double)pb.y;
            B.svel[3 * b + 2] = ((double)pa.z + (double)dvf[2]) - (double)pb.z;
          });
        }
        __syncwarp();
      }
      float xi = 1.0f;
      if (THERMO && occupied && (int)n + nb >= 2) {
        // Eq. thermo with the one pass of Sec. 3.5: E_k from the cell's exact
        // sums (momentum, second moment; beads' momentum and kinetic term),
        // xi = sqrt(E^/E_k) in FP64 from the Gamma pair drawn before pass 1
        long long Qt[3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
          Qt[q] = exact64 ? Q[q] : (long long)W.h[q][lane] * 1048576LL + (long long)W.l[q][lane] + Q[q];
        const __int128 S2 =
            exact64 ? S2x
                    : ((__int128)(((long long)TS.hh_hi[lane] << 24) + TS.hh_lo[lane]) << 40) +
                          ((__int128)((long long)TS.hl_hi[lane] * 16777216LL + TS.hl_lo[lane]) << 21) +
                          (__int128)(((long long)TS.ll_hi[lane] << 24) + TS.ll_lo[lane]) +
                          S2x;
        const long long Kx = (BEADS && gnb > 0) ? (long long)W.bx.E[lane] : 0ll;
        double Mt;
        const double Ep = mixed_ek_mt(B, (int)n, nb, 0, Qt, S2, X, Kx, Mt);
        const float2 dv = W.gdv[lane];
        if (!thermo_xi_from_draw(B, dv.x, dv.y, Ep, Mt, xi)) atomicOr(err, ERR_GAMMA_CAP);
      }
      if (occupied && !AT) W.prm[0][lane] = make_float4(u[0], u[1], u[2], xi);  // axis: prm[1]
      __syncwarp();
      if (BEADS && !AT && gnb > 0) {  // collide the beads with their cell's parameters
        for_beads([&](int j, int lc) {
          const float4 pa = W.prm[0][lc], pb = W.prm[1][lc];
          CellParams<float> prm;
          prm.u[0] = pa.x; prm.u[1] = pa.y; prm.u[2] = pa.z; prm.xi = pa.w;
          prm.n[0] = pb.x; prm.n[1] = pb.y; prm.n[2] = pb.z;
          double w[3] = {B.bgv[3 * j], B.bgv[3 * j + 1], B.bgv[3 * j + 2]};
          collide_bead<true>(B, prm, w, THERMO);
          const uint32_t b = B.border[j];
          B.svel[3 * b] = w[0];
          B.svel[3 * b + 1] = w[1];
          B.svel[3 * b + 2] = w[2];
        });
      }
      __syncwarp();
      if (ANG) {
        // ---- angular-momentum correction: centre of mass, then pass 1b ----
        auto rel_of = [&](const R* p, float x[3]) {
          const float4 b = reinterpret_cast<const float4*>(p)[1];
          x[0] = rel_pos_f(b.x, AB.sf[0], AB.lo[0], AB.hi[0]);
          x[1] = rel_pos_f(b.y, AB.sf[1], AB.lo[1], AB.hi[1]);
          x[2] = rel_pos_f(b.z, AB.sf[2], AB.lo[2], AB.hi[2]);
        };
        {
          long long Qo[3] = {0, 0, 0};
          if (has_ovf)
            for (uint32_t j = 0; j < novf; ++j)
              if (ovf_cell[j] == (uint32_t)cell) {
                float x[3];
                rel_of(ovf + j, x);
#pragma unroll
                for (int q = 0; q < 3; ++q) Qo[q] += fix32_rne(x[q]);
              }
          float rcm[3] = {0.0f, 0.0f, 0.0f};
          if (n > 0) {
#pragma unroll
            for (int q = 0; q < 3; ++q)
              rcm[q] = (split_sum_to_float(AG.qh[q][lane], AG.ql[q][lane], Qo[q]) * 0x1p-32f) /
                       small_to_float((int)n);
          }
          AG.rc[lane] = make_float4(rcm[0], rcm[1], rcm[2], 0.0f);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            AG.lh[k][lane] = 0;
            AG.ll[k][lane] = 0;
          }
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            AG.ph[k][lane] = 0;
            AG.pl[k][lane] = 0;
          }
        }
        __syncwarp();
        // r_c x (v - v') and the inertia-tensor entries of a member of cell o,
        // v' by the same operations as pass 2
        auto terms = [&](const float v[3], const float x[3], int o, float tm[9]) {
          const float4 pa = W.prm[0][o], pb = W.prm[1][o], c = AG.rc[o];
          const float nn[3] = {pb.x, pb.y, pb.z};
          const float uu[3] = {pa.x, pa.y, pa.z};
          float d[3], rr[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) d[q] = v[q] - uu[q];
          rotate(nn, H.ca, H.sa, H.omc, d, rr);
          float dv[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) dv[q] = v[q] - (uu[q] + (THERMO ? pa.w * rr[q] : rr[q]));
          const float rc[3] = {x[0] - c.x, x[1] - c.y, x[2] - c.z};
          tm[0] = rc[1] * dv[2] - rc[2] * dv[1];
          tm[1] = rc[2] * dv[0] - rc[0] * dv[2];
          tm[2] = rc[0] * dv[1] - rc[1] * dv[0];
          tm[3] = rc[1] * rc[1] + rc[2] * rc[2];
          tm[4] = rc[0] * rc[1];
          tm[5] = rc[0] * rc[2];
          tm[6] = rc[0] * rc[0] + rc[2] * rc[2];
          tm[7] = rc[1] * rc[2];
          tm[8] = rc[0] * rc[0] + rc[1] * rc[1];
        };
        bool slow_a = false;
        for (int sbase = 0; sbase < N; sbase += STAGE) {
          const int cnt = min(STAGE, N - sbase);
          if (N > STAGE) stage(sbase, cnt);  // else still staged from pass 1
          int Ha[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, La[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
          share(sbase, cnt, [&](int o, int j, bool last) {
            const int js = j + (j >> 5);
            const float v[3] = {W.sv[0][js], W.sv[1][js], W.sv[2][js]};
            const float x[3] = {AG.sr[0][js], AG.sr[1][js], AG.sr[2][js]};
            float tm[9];
            terms(v, x, o, tm);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              int h, l;
              if (!split32(tm[k], h, l)) {
                slow_a = true;
                h = 0;
                l = 0;
              }
              Ha[k] += h;
              La[k] += l;
            }
            if (last) {
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                atomicAdd(&AG.lh[k][o], Ha[k]);
                atomicAdd(&AG.ll[k][o], La[k]);
              }
#pragma unroll
              for (int k = 0; k < 6; ++k) {
                atomicAdd(&AG.ph[k][o], Ha[3 + k]);
                atomicAdd(&AG.pl[k][o], La[3 + k]);
              }
#pragma unroll
              for (int k = 0; k < 9; ++k) {
                Ha[k] = 0;
                La[k] = 0;
              }
            }
          });
          __syncwarp();
        }
        const bool exact_a = __any_sync(FULL, slow_a);  // a term of 1024 or more
        if (n > 0) {
          long long Lo[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
          auto add_terms = [&](const R* p) {
            const float4 a = reinterpret_cast<const float4*>(p)[0];
            const float v[3] = {a.x, a.y, a.z};
            float x[3], tm[9];
            rel_of(p, x);
            terms(v, x, lane, tm);
#pragma unroll
            for (int k = 0; k < 9; ++k) Lo[k] += fix32_rne(tm[k]);
          };
          if (exact_a)
            for (int k = 0; k < nrow; ++k) add_terms(rows + (size_t)lane * K + k);
          if (has_ovf)
            for (uint32_t j = 0; j < novf; ++j)
              if (ovf_cell[j] == (uint32_t)cell) add_terms(ovf + j);
          float dL[3], P6[6], om[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float tot = exact_a ? i64_to_float(Lo[k])
                                      : split_sum_to_float(AG.lh[k][lane], AG.ll[k][lane], Lo[k]);
            dL[k] = H.m * (tot * 0x1p-32f);
          }
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            const float tot = exact_a ? i64_to_float(Lo[3 + k])
                                      : split_sum_to_float(AG.ph[k][lane], AG.pl[k][lane], Lo[3 + k]);
            const float e = H.m * (tot * 0x1p-32f);
            P6[k] = (k == 1 || k == 2 || k == 4) ? -e : e;
          }
          solve_omega<float>((int)n, P6, dL, om);
          AG.om[lane] = make_float4(om[0], om[1], om[2], 0.0f);
        }
        __syncwarp();
      }
    }

    // ---- pass 2: collide (Eq. srd), stream (Eq. stream), bin (Sec. 3.4) ----
    // new state of a member and its cell for the next step
    // Eq. at: member m's random velocity, from the cache or drawn again (m < 0:
    // an overflow member)
    auto at_dv = [&](int m, uint32_t tag, float dv[3]) {
      if (m >= 0 && m < DVC) {
        const int mp = m + (m >> 5);
        dv[0] = AS.dv[0][mp];
        dv[1] = AS.dv[1][mp];
        dv[2] = AS.dv[2][mp];
      } else {
        at_draw(B, t, tag, 0u, B.sig_f, dv);
      }
    };
    auto advance = [&](float r[3], float w[3], uint32_t tag, int o, int m) -> uint32_t {
      if (MODE != MODE_P && AT) {  // Eq. at
        const float4 pa = W.prm[0][o], pb = W.prm[1][o];
        float dv[3];
        at_dv(m, tag, dv);
        w[0] = (pa.x + dv[0]) - pb.x;
        w[1] = (pa.y + dv[1]) - pb.y;
        w[2] = (pa.z + dv[2]) - pb.z;
      } else if (MODE != MODE_P) {
        const float4 pa = W.prm[0][o], pb = W.prm[1][o];
        const float nn[3] = {pb.x, pb.y, pb.z};
        const float uu[3] = {pa.x, pa.y, pa.z};
        float d[3], rr[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) d[q] = w[q] - uu[q];
        rotate(nn, H.ca, H.sa, H.omc, d, rr);
#pragma unroll
        for (int q = 0; q < 3; ++q) w[q] = uu[q] + (THERMO ? pa.w * rr[q] : rr[q]);
        if (ANG) {  // v'' = v' + omega x r_c
          const float4 c = AG.rc[o], om = AG.om[o];
          const float rc[3] = {rel_pos_f(r[0], AB.sf[0], AB.lo[0], AB.hi[0]) - c.x,
                               rel_pos_f(r[1], AB.sf[1], AB.lo[1], AB.hi[1]) - c.y,
                               rel_pos_f(r[2], AB.sf[2], AB.lo[2], AB.hi[2]) - c.z};
          w[0] = w[0] + (om.y * rc[2] - om.z * rc[1]);
          w[1] = w[1] + (om.z * rc[0] - om.x * rc[2]);
          w[2] = w[2] + (om.x * rc[1] - om.y * rc[0]);
        }
      }
      if (MODE == MODE_C) return 0u;
      // periodic box; the additions of zero keep the operation sequence of
      // the general form (they turn -0 into +0)
      bool bad = false;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (FORCE) {
          r[q] = fmaf(w[q], H.dt, r[q]) + H.hg[q];
          w[q] = w[q] + H.gdt[q];
        } else {
          r[q] = fmaf(w[q], H.dt, r[q]) + 0.0f;
          w[q] = w[q] + 0.0f;
        }
        r[q] = wrap_fast(r[q], H.L[q]);
        bad |= !(r[q] >= 0.0f && r[q] < H.L[q]);
      }
      if (bad) {  // more than one box length out, or non-finite
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (!(r[q] >= 0.0f && r[q] < H.L[q])) {
            r[q] = r[q] - H.L[q] * floorf(r[q] / H.L[q]);
            if (!(r[q] >= 0.0f && r[q] < H.L[q])) r[q] = 0.0f;
          }
      }
      const int cx = bin_axis(r[0], H.lo[0], H.hi[0], H.n[0]);
      const int cy = bin_axis(r[1], H.lo[1], H.hi[1], H.n[1]);
      const int cz = bin_axis(r[2], H.lo[2], H.hi[2], H.n[2]);
      return (uint32_t)(cx + H.n[0] * (cy + H.n[1] * cz));
    };
    // append a record to the row of cell c2 at the slot taken for it (or to
    // the overflow list beyond the row capacity)
    auto emit = [&](const float r[3], const float w[3], uint32_t tag, uint32_t c2, uint32_t slot) {
      if (slot < (uint32_t)H.K) {
        store_rec_streaming(H.rows_out + (size_t)c2 * H.K + slot, r, w, tag, l2_evict_first());
      } else {
        const uint32_t j = atomicAdd(H.ovf_n_out, 1u);
        if (j < (uint32_t)H.ovf_cap) {
          store_rec(H.ovf_out + j, r, w, tag);
          H.ovf_cell_out[j] = c2;
        } else {
          atomicOr(err, ERR_OVERFLOW_CAP);
        }
      }
    };
    // Chunks of CH windows: (a) every record of the chunk is copied into
    // shared memory by asynchronous copies (all in flight together, no
    // registers held); (b) each is advanced and, in modes P and F, written
    // back with its new cell while the slot request for it goes out; (c) once
    // all slot requests of the chunk are out, the records are written to
    // their rows.  One load latency and one slot latency per chunk.
    for (int base = 0; base < N; base += 32 * CH) {
#pragma unroll
      for (int w = 0; w < CH; ++w) {
        const int m = base + (w << 5) + lane;
        if (m < N) {
          const R* p = member(m, owner_of(m));
          const unsigned long long pol = l2_evict_first();
          cp_async16_last_use(&W.buf[w][0][lane], p, pol);
          cp_async16_last_use(&W.buf[w][1][lane], reinterpret_cast<const float4*>(p) + 1, pol);
        }
      }
      cp_async_wait_all();  // each lane reads back only its own copies
      // Slots: the lanes of a window bound for the same cell share one atomic
      // (made by the first of them) and take consecutive slots, so their
      // records land side by side.  The atomic's result is read only when
      // the chunk is written.
      uint32_t sbase[CH];
      int lr[CH];  // leader lane | rank << 8
#pragma unroll
      for (int w = 0; w < CH; ++w) {
        const int m = base + (w << 5) + lane;
        uint32_t key = 0xFFFFFFFFu;
        if (m < N) {
          const int o = owner_of(m);
          const float4 x = W.buf[w][0][lane], y = W.buf[w][1][lane];  // (v, tag), (r, pad)
          float v[3] = {x.x, x.y, x.z}, r[3] = {y.x, y.y, y.z};
          const uint32_t c2 = advance(r, v, __float_as_uint(x.w), o, m);
          if (MODE == MODE_C) {
            store_rec(member(m, o), r, v, __float_as_uint(x.w));
          } else {
            W.buf[w][0][lane] = make_float4(v[0], v[1], v[2], x.w);
            W.buf[w][1][lane] = make_float4(r[0], r[1], r[2], __uint_as_float(c2));
            key = c2;
          }
        }
        if (MODE != MODE_C) {
          const unsigned peers = __match_any_sync(FULL, key);
          const int leader = __ffs(peers) - 1;
          sbase[w] = 0u;
          if (key != 0xFFFFFFFFu && lane == leader)
            sbase[w] = atomicAdd(&H.cnt_out[key], (uint32_t)__popc(peers));
          lr[w] = leader | (__popc(peers & ((1u << lane) - 1u)) << 8);
        }
      }
      if (MODE != MODE_C) {
#pragma unroll
        for (int w = 0; w < CH; ++w) {
          const int m = base + (w << 5) + lane;
          const uint32_t slot = __shfl_sync(FULL, sbase[w], lr[w] & 255) + (uint32_t)(lr[w] >> 8);
          if (m < N) {
            const float4 x = W.buf[w][0][lane], y = W.buf[w][1][lane];
            const float v[3] = {x.x, x.y, x.z}, r[3] = {y.x, y.y, y.z};
            emit(r, v, __float_as_uint(x.w), __float_as_uint(y.w), slot);
          }
        }
      }
    }
    if (has_ovf) {
      for (uint32_t j = 0; j < novf; ++j)
        if (ovf_cell[j] == (uint32_t)cell) {
          R* p = ((R*)B.ovf_rec[cur]) + j;
          float r[3], w[3];
          uint32_t tag;
          load_rec(p, r, w, tag);
          const uint32_t c2 = advance(r, w, tag, lane, -1);
          if (MODE == MODE_C) store_rec(p, r, w, tag);
          else emit(r, w, tag, c2, atomicAdd(&H.cnt_out[c2], 1u));
        }
    }
  }
}

// The F-mode instance of the SRD variant (thermo, force, beads) with cpw = 8 or
// 16 cells per warp and pass-2 chunks of 3 windows (k_cells_warp_narrow.cu).
void* cells_warp_narrow_fn(bool thermo, bool force, bool beads, int cpw);

}  // namespace mpcd
