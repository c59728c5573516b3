// k_cells_warp_d.cu -- the fused SRD step of the FP64 model with the members
// of 32 cells spread over the lanes of a warp (arXiv:1801.10187: Sec. 2 Eqs.
// stream, srd and thermo; Sec. 3.4 cell list; Sec. 3.5 cell properties;
// Sec. 3.6 rotation and thermostat, algorithm "SRD collision rule").
//
// The FP64 counterpart of k_cells_warp (mixed model), for boxes without
// walls: same modes, 64-byte records and results within rounding of the
// per-cell loop of k_cells.  A warp owns 32 consecutive cells; their row
// members are numbered in cell order and a byte map gives each member's cell.
//   pass 1   velocities of up to 128 members are staged in shared memory in
//            member order; each lane sums a consecutive share in registers
//            (double) and adds it to its cell with one shared atomic per
//            component when the cell changes
//   cell     lane c forms u of cell c, draws the axis (and with the
//            thermostat, after the same kind of pass for the energy about u,
//            xi) and leaves the collision in shared memory as the affine
//            map v' = A v + c (A = xi R, c = u - A u)
//   pass 2   windows of 32 members: records copied to shared memory by
//            cp.async, collided, streamed, binned under the next shift; lanes
//            bound for the same cell share one slot atomic
// Solute beads of the warp's bead group are handled one per lane with shared
// per-cell sums.  The FP64 pipe bounds this kernel on GB300.
//
// The Andersen-thermostat variant (Eq. at, Sec. 3.7): pass 1 also sums each
// member's Gaussian random velocity dv (drawn from its tag), the cell phase
// forms the mass-weighted mean dbar, and pass 2 sets v = (u + dv) - dbar.
#include "dev_collide.cuh"
#include "dev_rows.cuh"
#include "dev_stream.cuh"
#include "kernels.h"
#include "mpcd_internal.cuh"

namespace mpcd {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int WARPS = BLOCK / 32;
constexpr int MAP_MEMBERS = 640;
constexpr int STAGE = 128;
constexpr int STAGE_PAD = STAGE + STAGE / 32;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

struct WarpShared {
  double2 pr[6][32];               // per cell: rows (A_i0, A_i1), (A_i2, c_i) of the collision
                                   // map; before that (u0, u1), (u2, xi), (axis0, axis1), (axis2, 0)
  double P[3][32];                 // sum of v over the cell's solvent
  double E[32];                    // sum of |v - u|^2 over the cell's solvent
  int offs[33];                    // first member of each cell; offs[32] = members
  int pad_[3];
  unsigned char map[MAP_MEMBERS];  // owner lane of each member
  union {
    double sv[3][STAGE_PAD];       // pass 1: staged velocities (index j + j / 32)
    float4 buf[4][32];             // pass 2: records of one window (four quarters)
  };
};

struct BeadShared {  // per-cell bead sums (bead variants)
  double X[3][32];
  double E[32];
  int nb[32];
};

struct ATShared {  // Andersen rule: per-cell sums of dv, staged tags, bead sums of M dv
  double D[3][32];
  uint32_t tag[STAGE_PAD];
  uint32_t pad_[4 - (STAGE_PAD & 3)];
  double DX[3][32];
};

struct SpanParams {
  double dt, ca, sa, omc, m, Mb;
  double L[3], hg[3], gdt[3];
  long long S[3];  // grid shift of the step the records are binned for
  double s[3];     // the same as doubles (S 2^-32, exact)
  int n[3], K;
  RecD* rows_cur;
  RecD* rows_out;
  uint32_t* cnt_out;
  RecD* ovf_out;
  uint32_t* ovf_cell_out;
  uint32_t* ovf_n_out;
  int ovf_cap, pad;
};
constexpr size_t SPAN_SMEM = (sizeof(SpanParams) + 15) & ~(size_t)15;
constexpr size_t BLOCK_SMEM = SPAN_SMEM + WARPS * sizeof(WarpShared);
constexpr size_t BLOCK_SMEM_BEADS = BLOCK_SMEM + WARPS * sizeof(BeadShared);

__host__ __device__ constexpr size_t block_smem(bool beads, bool at) {
  return BLOCK_SMEM + (beads ? WARPS * sizeof(BeadShared) : 0) + (at ? WARPS * sizeof(ATShared) : 0);
}

}  // namespace

template <bool THERMO, int MODE, bool FORCE, bool BEADS, bool AT>
__global__ void __launch_bounds__(BLOCK, 3) k_cells_warp_d(const BoxDev* __restrict__ boxes,
                                                           const int2* __restrict__ spans,
                                                           int nspans, int* err) {
  using R = RecD;
  extern __shared__ __align__(16) unsigned char smem_[];
  SpanParams& sp_ = *reinterpret_cast<SpanParams*>(smem_);
  const int lane = threadIdx.x & 31;
  WarpShared& W = reinterpret_cast<WarpShared*>(smem_ + SPAN_SMEM)[threadIdx.x >> 5];
  BeadShared& BS = reinterpret_cast<BeadShared*>(smem_ + BLOCK_SMEM)[threadIdx.x >> 5];
  ATShared& AS = reinterpret_cast<ATShared*>(smem_ + block_smem(BEADS, false))[threadIdx.x >> 5];
  const SpanParams& H = sp_;
  int box_of_params = -1;
  for (int sp = blockIdx.x; sp < nspans; sp += gridDim.x) {
    const int2 tt = spans[sp];
    const BoxDev& B = boxes[tt.x];
    const unsigned long long t = B.step;
    if (tt.x != box_of_params) {  // block-uniform
      __syncthreads();
      if (threadIdx.x == 0) {
        SpanParams& P = sp_;
        P.dt = B.dt; P.ca = B.ca; P.sa = B.sa; P.omc = B.omc; P.m = B.m; P.Mb = B.Mb;
        for (int q = 0; q < 3; ++q) {
          P.L[q] = B.L[q]; P.hg[q] = B.hg[q]; P.gdt[q] = B.gdt[q]; P.n[q] = B.n[q];
        }
        P.K = B.K;
        const int out = B.cur ^ 1;
        P.rows_cur = (RecD*)B.rows[B.cur];
        P.rows_out = (RecD*)B.rows[out];
        P.cnt_out = B.cnt[out];
        P.ovf_out = (RecD*)B.ovf_rec[out];
        P.ovf_cell_out = B.ovf_cell[out];
        P.ovf_n_out = &B.ovf_n[out];
        P.ovf_cap = B.ovf_cap;
        if (MODE != MODE_C) {
          shift_units(B, MODE == MODE_P ? t : t + 1ull, P.S);
          for (int q = 0; q < 3; ++q) P.s[q] = (double)P.S[q] * 0x1p-32;
        }
      }
      __syncthreads();
      box_of_params = tt.x;
    }
    const int c0 = tt.y + (int)(threadIdx.x & ~31u);
    if (c0 >= B.ncells) continue;  // warp-uniform
    const int cell = c0 + lane;
    const int cur = B.cur;
    const int K = H.K;
    const uint32_t n = cell < B.ncells ? B.cnt[cur][cell] : 0u;
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
    auto stage = [&](int sbase, int cnt) {
      for (int j0 = 0; j0 < cnt; j0 += 64) {  // two windows of loads in flight
        double a[2][3];
        uint32_t tg[2] = {0u, 0u};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int j = j0 + (u << 5) + lane;
          if (j < cnt) {
            const R* p = member(sbase + j, owner_of(sbase + j));
            load_v(p, a[u]);
            if (AT) tg[u] = p->tag;
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int j = j0 + (u << 5) + lane;
          if (j < cnt) {
            const int js = j + (j >> 5);
            W.sv[0][js] = a[u][0];
            W.sv[1][js] = a[u][1];
            W.sv[2][js] = a[u][2];
            if (AT) AS.tag[js] = tg[u];
          }
        }
      }
      __syncwarp();
    };
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
        f(o, j + (j >> 5), j + 1 == cend || j + 1 == ce);
      }
    };

    if (MODE != MODE_P) {
      // ---- pass 1: momentum sums per cell (Sec. 3.5) ----
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        W.P[q][lane] = 0.0;
        if (AT) AS.D[q][lane] = 0.0;
      }
      W.E[lane] = 0.0;
      __syncwarp();
      for (int sbase = 0; sbase < N; sbase += STAGE) {
        const int cnt = min(STAGE, N - sbase);
        stage(sbase, cnt);
        double s[3] = {0.0, 0.0, 0.0}, sd[3] = {0.0, 0.0, 0.0};
        share(sbase, cnt, [&](int o, int js, bool last) {
#pragma unroll
          for (int q = 0; q < 3; ++q) s[q] += W.sv[q][js];
          if (AT) {  // Eq. at: this member's random velocity
            double dv[3];
            at_draw(B, t, AS.tag[js], 0u, B.sig, dv);
#pragma unroll
            for (int q = 0; q < 3; ++q) sd[q] += dv[q];
          }
          if (last) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              atomicAdd(&W.P[q][o], s[q]);
              s[q] = 0.0;
              if (AT) {
                atomicAdd(&AS.D[q][o], sd[q]);
                sd[q] = 0.0;
              }
            }
          }
        });
        __syncwarp();
      }

      // ---- beads of the warp's bead group, one per lane (Sec. 3.6) ----
      int gb0 = 0, gnb = 0, nb = 0;
      auto for_beads = [&](auto&& f) {
        for (int j0 = 0; j0 < gnb; j0 += 32) {
          const int j = gb0 + j0 + lane;
          if (j0 + lane < gnb) f(j, B.bgc[j] - c0);
        }
      };
      if (BEADS) {
        const int g = c0 / B.tc;
        gb0 = (int)B.bstart[g];
        gnb = (int)B.bstart[g + 1] - gb0;
        if (gnb > 0) {
#pragma unroll
          for (int q = 0; q < 3; ++q) BS.X[q][lane] = 0.0;
          BS.E[lane] = 0.0;
          BS.nb[lane] = 0;
          __syncwarp();
          for_beads([&](int j, int lc) {
#pragma unroll
            for (int q = 0; q < 3; ++q) atomicAdd(&BS.X[q][lc], H.Mb * B.bgv[3 * j + q]);
            atomicAdd(&BS.nb[lc], 1);
          });
          __syncwarp();
          nb = BS.nb[lane];
        }
      }

      // ---- per cell: u = P / M, then the energy about u, axis and xi ----
      const bool occupied = n > 0 || nb > 0;
      double u[3] = {0.0, 0.0, 0.0};
      double M = 1.0;
      if (occupied) {
        double Pv[3] = {W.P[0][lane], W.P[1][lane], W.P[2][lane]};
        if (has_ovf)
          for (uint32_t j = 0; j < novf; ++j)
            if (ovf_cell[j] == (uint32_t)cell) {
              double w[3];
              load_v(ovf + j, w);
#pragma unroll
              for (int q = 0; q < 3; ++q) Pv[q] += w[q];
            }
        M = ll2d_exact((long long)n) * H.m + ll2d_exact((long long)nb) * H.Mb;
        const double iM = 1.0 / M;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          double P = H.m * Pv[q];
          if (BEADS && gnb > 0) P += BS.X[q][lane];
          u[q] = P * iM;
        }
        W.pr[0][lane] = make_double2(u[0], u[1]);
        W.pr[1][lane] = make_double2(u[2], 1.0);
      }
      if (AT) {
        // Eq. at: dbar = sum m dv / sum m over the cell's members and beads
        if (BEADS && gnb > 0) {
#pragma unroll
          for (int q = 0; q < 3; ++q) AS.DX[q][lane] = 0.0;
          __syncwarp();
          for_beads([&](int j, int lc) {
            double dv[3];
            at_draw(B, t, B.border[j], 1u, B.sigb, dv);
#pragma unroll
            for (int q = 0; q < 3; ++q) atomicAdd(&AS.DX[q][lc], H.Mb * dv[q]);
          });
          __syncwarp();
        }
        if (occupied) {
          double Dv[3] = {AS.D[0][lane], AS.D[1][lane], AS.D[2][lane]};
          if (has_ovf)
            for (uint32_t j = 0; j < novf; ++j)
              if (ovf_cell[j] == (uint32_t)cell) {
                double dv[3];
                at_draw(B, t, ovf[j].tag, 0u, B.sig, dv);
#pragma unroll
                for (int q = 0; q < 3; ++q) Dv[q] += dv[q];
              }
          double dbar[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            double D = H.m * Dv[q];
            if (BEADS && gnb > 0) D += AS.DX[q][lane];
            dbar[q] = D / M;
          }
          W.pr[0][lane] = make_double2(u[0], u[1]);
          W.pr[1][lane] = make_double2(u[2], 0.0);
          W.pr[2][lane] = make_double2(dbar[0], dbar[1]);
          W.pr[3][lane] = make_double2(dbar[2], 0.0);
        }
        __syncwarp();
        if (BEADS && gnb > 0) {  // Eq. at for the beads: v = (u + dv) - dbar
          for_beads([&](int j, int lc) {
            const double2 p0 = W.pr[0][lc], p1 = W.pr[1][lc], p2 = W.pr[2][lc], p3 = W.pr[3][lc];
            const uint32_t b = B.border[j];
            double dv[3];
            at_draw(B, t, b, 1u, B.sigb, dv);
            B.svel[3 * b] = (p0.x + dv[0]) - p2.x;
            B.svel[3 * b + 1] = (p0.y + dv[1]) - p2.y;
            B.svel[3 * b + 2] = (p1.x + dv[2]) - p3.x;
          });
        }
        __syncwarp();
      }
      double xi = 1.0;
      if (THERMO) {
        __syncwarp();
        if (BEADS && gnb > 0) {
          for_beads([&](int j, int lc) {
            const double2 ua = W.pr[0][lc], ub = W.pr[1][lc];
            const double d0 = B.bgv[3 * j] - ua.x, d1 = B.bgv[3 * j + 1] - ua.y,
                         d2 = B.bgv[3 * j + 2] - ub.x;
            atomicAdd(&BS.E[lc], (0.5 * H.Mb) * (d0 * d0 + d1 * d1 + d2 * d2));
          });
          __syncwarp();
        }
        for (int sbase = 0; sbase < N; sbase += STAGE) {
          const int cnt = min(STAGE, N - sbase);
          if (N > STAGE) stage(sbase, cnt);  // else still staged from pass 1
          double se = 0.0;
          share(sbase, cnt, [&](int o, int js, bool last) {
            const double2 ua = W.pr[0][o], ub = W.pr[1][o];
            const double d0 = W.sv[0][js] - ua.x, d1 = W.sv[1][js] - ua.y, d2 = W.sv[2][js] - ub.x;
            se += d0 * d0 + d1 * d1 + d2 * d2;
            if (last) {
              atomicAdd(&W.E[o], se);
              se = 0.0;
            }
          });
          __syncwarp();
        }
        if (occupied) {
          double Es = W.E[lane];
          if (has_ovf)
            for (uint32_t j = 0; j < novf; ++j)
              if (ovf_cell[j] == (uint32_t)cell) {
                double w[3];
                load_v(ovf + j, w);
                const double d0 = w[0] - u[0], d1 = w[1] - u[1], d2 = w[2] - u[2];
                Es += d0 * d0 + d1 * d1 + d2 * d2;
              }
          // Eq. thermo: E_k about u, E^ ~ Gamma(3(N_c-1)/2, kT), xi = sqrt(E^/E_k)
          double Ek = (0.5 * H.m) * Es;
          if (BEADS && gnb > 0) Ek += BS.E[lane];
          const int nc = (int)n + nb;
          if (nc >= 2 && Ek > 0.0) {
            double ehat;
            if (gamma_draw(B, t, (uint32_t)cell, nc, ehat)) xi = sqrt(ehat / Ek);
            else atomicOr(err, ERR_GAMMA_CAP);
          }
        }
      }
      // pass 2 takes the collision of Eq. srd as one affine map per cell,
      // v' = A v + c with A = xi R(axis, alpha) and c = u - A u (Rodrigues'
      // R = cos(alpha) I + sin(alpha) [n]x + (1 - cos(alpha)) n n^T): nine
      // FP64 fmas a member instead of the subtract, rotate and add.
      auto put_map = [&](const double uu[3], double x, const double nn[3]) {
        const double ca = H.ca, sa = H.sa, omc = H.omc;
        double A[3][3];
        A[0][0] = fma(omc * nn[0], nn[0], ca);
        A[1][1] = fma(omc * nn[1], nn[1], ca);
        A[2][2] = fma(omc * nn[2], nn[2], ca);
        A[0][1] = fma(omc * nn[0], nn[1], -sa * nn[2]);
        A[1][0] = fma(omc * nn[1], nn[0], sa * nn[2]);
        A[0][2] = fma(omc * nn[0], nn[2], sa * nn[1]);
        A[2][0] = fma(omc * nn[2], nn[0], -sa * nn[1]);
        A[1][2] = fma(omc * nn[1], nn[2], -sa * nn[0]);
        A[2][1] = fma(omc * nn[2], nn[1], sa * nn[0]);
        double c[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
          for (int k = 0; k < 3; ++k)
            if (THERMO) A[i][k] *= x;
          c[i] = uu[i] - fma(A[i][0], uu[0], fma(A[i][1], uu[1], A[i][2] * uu[2]));
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          W.pr[2 * i][lane] = make_double2(A[i][0], A[i][1]);
          W.pr[2 * i + 1][lane] = make_double2(A[i][2], c[i]);
        }
      };
      if (occupied && !AT) {
        double ax[3];
        axis_of(B, t, (uint32_t)cell, ax);  // Sec. 3.6
        if (BEADS) {  // the beads collide with u, xi and the axis first
          W.pr[0][lane] = make_double2(u[0], u[1]);
          W.pr[1][lane] = make_double2(u[2], xi);
          W.pr[2][lane] = make_double2(ax[0], ax[1]);
          W.pr[3][lane] = make_double2(ax[2], 0.0);
        } else {
          put_map(u, xi, ax);
        }
      }
      __syncwarp();
      if (BEADS && !AT && gnb > 0) {  // collide the beads with their cell's parameters
        for_beads([&](int j, int lc) {
          const double2 p0 = W.pr[0][lc], p1 = W.pr[1][lc], p2 = W.pr[2][lc], p3 = W.pr[3][lc];
          CellParams<double> prm;
          prm.u[0] = p0.x; prm.u[1] = p0.y; prm.u[2] = p1.x; prm.xi = p1.y;
          prm.n[0] = p2.x; prm.n[1] = p2.y; prm.n[2] = p3.x;
          double w[3] = {B.bgv[3 * j], B.bgv[3 * j + 1], B.bgv[3 * j + 2]};
          collide_bead<false>(B, prm, w, THERMO);
          const uint32_t b = B.border[j];
          B.svel[3 * b] = w[0];
          B.svel[3 * b + 1] = w[1];
          B.svel[3 * b + 2] = w[2];
        });
      }
      if (BEADS && !AT) {
        __syncwarp();
        if (occupied) {
          const double2 p0 = W.pr[0][lane], p1 = W.pr[1][lane], p2 = W.pr[2][lane],
                        p3 = W.pr[3][lane];
          const double uu[3] = {p0.x, p0.y, p1.x}, nn[3] = {p2.x, p2.y, p3.x};
          put_map(uu, p1.y, nn);
        }
      }
      __syncwarp();
    }

    // ---- pass 2: collide (Eq. srd), stream (Eq. stream), bin (Sec. 3.4) ----
    auto advance = [&](double r[3], double w[3], uint32_t tag, int o) -> uint32_t {
      if (MODE != MODE_P && AT) {  // Eq. at
        const double2 p0 = W.pr[0][o], p1 = W.pr[1][o], p2 = W.pr[2][o], p3 = W.pr[3][o];
        double dv[3];
        at_draw(B, t, tag, 0u, B.sig, dv);
        w[0] = (p0.x + dv[0]) - p2.x;
        w[1] = (p0.y + dv[1]) - p2.y;
        w[2] = (p1.x + dv[2]) - p3.x;
      } else if (MODE != MODE_P) {  // Eq. srd as v' = A v + c
        double v2[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const double2 a = W.pr[2 * i][o], b = W.pr[2 * i + 1][o];
          v2[i] = fma(a.x, w[0], fma(a.y, w[1], fma(b.x, w[2], b.y)));
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) w[i] = v2[i];
      }
      if (MODE == MODE_C) return 0u;
      int c[3];
      bool bad = false;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (FORCE) {
          r[q] = fma(w[q], H.dt, r[q]) + H.hg[q];
          w[q] = w[q] + H.gdt[q];
        } else {
          r[q] = fma(w[q], H.dt, r[q]);  // FP64 parity is to rounding: no -0 -> +0 step
        }
        r[q] = wrap_bits(r[q], H.L[q]);  // finite, in [0, L) (or -0)
        int i = floor_minus_shift(r[q], H.S[q], H.s[q]);  // in [-1, n] (Sec. 3.4)
        if (i < 0) i += H.n[q];
        if (i >= H.n[q]) i -= H.n[q];
        if (i < 0 || i >= H.n[q]) {
          bad = true;
          i = 0;
        }
        c[q] = i;
      }
      if (bad) atomicOr(err, ERR_CELL_RANGE);
      return (uint32_t)(c[0] + H.n[0] * (c[1] + H.n[1] * c[2]));
    };
    auto emit = [&](const double r[3], const double w[3], uint32_t tag, uint32_t c2, uint32_t slot) {
      if (slot < (uint32_t)H.K) {
        store_rec(H.rows_out + (size_t)c2 * H.K + slot, r, w, tag);
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
    for (int base = 0; base < N; base += 32) {
      const int m = base + lane;
      const bool act = m < N;
      int o = 0;
      if (act) {
        o = owner_of(m);
        const float4* p = reinterpret_cast<const float4*>(member(m, o));
#pragma unroll
        for (int q = 0; q < 4; ++q) cp_async16(&W.buf[q][lane], p + q);
      }
      cp_async_wait_all();  // each lane reads back only its own copies
      double r[3], w[3];
      uint32_t tag = 0u, c2 = 0xFFFFFFFFu;
      if (act) {
        // the record's four 16-byte quarters sit 512 bytes apart in shared memory
        const double2 a = *reinterpret_cast<const double2*>(&W.buf[0][lane]);
        const double2 b = *reinterpret_cast<const double2*>(&W.buf[1][lane]);
        const double2 cq = *reinterpret_cast<const double2*>(&W.buf[2][lane]);
        const uint4 dq = *reinterpret_cast<const uint4*>(&W.buf[3][lane]);
        r[0] = a.x; r[1] = a.y; r[2] = b.x;
        w[0] = b.y; w[1] = cq.x; w[2] = cq.y;
        tag = dq.x;
        c2 = advance(r, w, tag, o);
        if (MODE == MODE_C) store_rec(member(m, o), r, w, tag);
      }
      if (MODE != MODE_C) {
        const uint32_t key = act ? c2 : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(FULL, key);
        const int leader = __ffs(peers) - 1;
        uint32_t sbase = 0u;
        if (act && lane == leader) sbase = atomicAdd(&H.cnt_out[c2], (uint32_t)__popc(peers));
        const uint32_t slot = __shfl_sync(FULL, sbase, leader) +
                              (uint32_t)__popc(peers & ((1u << lane) - 1u));
        if (act) emit(r, w, tag, c2, slot);
      }
      __syncwarp();  // buf is refilled by the next window
    }
    if (has_ovf) {
      for (uint32_t j = 0; j < novf; ++j)
        if (ovf_cell[j] == (uint32_t)cell) {
          R* p = ((R*)B.ovf_rec[cur]) + j;
          double r[3], w[3];
          uint32_t tag;
          load_rec(p, r, w, tag);
          const uint32_t c2 = advance(r, w, tag, lane);
          if (MODE == MODE_C) store_rec(p, r, w, tag);
          else emit(r, w, tag, c2, atomicAdd(&H.cnt_out[c2], 1u));
        }
    }
  }
}

template <bool TH, int MODE, bool FO, bool BE, bool AT>
static void* warpd_fn() {
  return (void*)k_cells_warp_d<TH, MODE, FO, BE, AT>;
}

template <int MODE, bool BE>
static void* warpd_variant_mb(bool thermo, bool force, bool at) {
  if (at) return force ? warpd_fn<false, MODE, true, BE, true>() : warpd_fn<false, MODE, false, BE, true>();
  if (thermo) return force ? warpd_fn<true, MODE, true, BE, false>() : warpd_fn<true, MODE, false, BE, false>();
  return force ? warpd_fn<false, MODE, true, BE, false>() : warpd_fn<false, MODE, false, BE, false>();
}

static void* warpd_variant(bool thermo, bool force, bool beads, bool at, int mode) {
  if (mode == MODE_P)
    return beads ? warpd_variant_mb<MODE_P, true>(thermo, force, at)
                 : warpd_variant_mb<MODE_P, false>(thermo, force, at);
  if (mode == MODE_F)
    return beads ? warpd_variant_mb<MODE_F, true>(thermo, force, at)
                 : warpd_variant_mb<MODE_F, false>(thermo, force, at);
  return beads ? warpd_variant_mb<MODE_C, true>(thermo, force, at)
               : warpd_variant_mb<MODE_C, false>(thermo, force, at);
}

int cells_warpd_blocks_per_sm(bool thermo, bool force, bool beads, bool at, int mode) {
  const void* fn = warpd_variant(thermo, force, beads, at, mode);
  const size_t smem = block_smem(beads, at);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, BLOCK, smem);
  return nb;
}

void launch_cells_warpd(bool thermo, bool force, bool beads, bool at, int mode, const BoxDev* boxes,
                        const int2* spans, int nspans, int grid, int* err, cudaStream_t s) {
  if (nspans <= 0) return;
  void* args[] = {(void*)&boxes, (void*)&spans, (void*)&nspans, (void*)&err};
  cudaLaunchKernel(warpd_variant(thermo, force, beads, at, mode), dim3(grid), dim3(BLOCK), args,
                   block_smem(beads, at), s);
}

}  // namespace mpcd
