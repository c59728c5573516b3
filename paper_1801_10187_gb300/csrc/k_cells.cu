// k_cells.cu -- the fused SRD step on cell rows (arXiv:1801.10187: Sec. 2
// Eqs. stream, srd and thermo; Sec. 3.4 cell list; Sec. 3.5 cell properties;
// Sec. 3.6 rotation and thermostat, algorithm "SRD collision rule").
//
// One thread owns one cell.  Its members are the records of its row (plus,
// rarely, overflow records).  Mode F is one whole step boundary in one pass:
//   collide step t      pass 1 forms the exact cell sums (and, with the
//                       thermostat, a second pass the energy about u); the
//                       thread draws the axis and xi; pass 2 rotates each member
//   stream step t + 1   the rotated velocity streams the position
//   bin step t + 1      with the next grid shift; the record is appended to the
//                       row of its new cell in the other buffer (atomic slot)
// Mode P only streams and bins (the first step after the state was read or
// set), mode C only collides, in place (to complete a step before the state is
// read).  Nothing else touches the particles: no separate sort, scan or
// reorder pass exists, and every record moves as one 32-byte sector.
//
// This kernel also carries the Andersen rule (Eq. at, Sec. 3.7) for rows too
// long for the warp-spread kernel, and the angular-momentum-conserving form
// of either rule (Sec. 2: the constraint the paper cites after Eqs. srd and
// at): a second pass over the cell's members forms dL = sum m r_c x (v - v')
// and the inertia tensor about the cell's centre of mass, and every member
// then receives omega x r_c with Pi omega = dL.
#include "dev_angular.cuh"
#include "dev_collide.cuh"
#include "dev_rows.cuh"
#include "dev_stream.cuh"
#include "kernels.h"
#include "mpcd_internal.cuh"

namespace mpcd {

namespace {

// Coordinate of x relative to the shifted cell whose index along the axis is
// i (in [0, 1); a member wrapped across the box edge is brought back).
__device__ __forceinline__ double rel_pos(double x, double s, int i, double L) {
  double d = (x - s) - (double)i;
  if (d < 0.0) d += L;
  else if (d >= 1.0) d -= L;
  return d;
}

// Per-cell sums of the angular correction: positions (centre of mass), then
// r_c x (v - v') and the inertia tensor entries (|r_c|^2 - r_c r_c^T: xx, xy,
// xz, yy, yz, zz with the off-diagonal products summed positive).  Mixed
// model: int64 sums of rne(term 2^32) of float terms; FP64: double sums.
template <bool MIXED> struct AngAcc;
template <> struct AngAcc<true> {
  long long q[3] = {0, 0, 0}, l[3] = {0, 0, 0}, p[6] = {0, 0, 0, 0, 0, 0};
};
template <> struct AngAcc<false> {
  double q[3] = {0, 0, 0}, l[3] = {0, 0, 0}, p[6] = {0, 0, 0, 0, 0, 0};
};

}  // namespace

template <bool MIXED, bool THERMO, bool EXTRA, int MODE, bool AT, bool ANG>
__global__ void __launch_bounds__(BLOCK) k_cells(const BoxDev* __restrict__ boxes,
                                                 const int2* __restrict__ spans, int nspans,
                                                 int* err) {
  using T = real_t<MIXED>;
  using R = rec_t<MIXED>;
  __shared__ long long sSn[3];  // shift of the step the records are binned for
  __shared__ long long sSz;     // z shift of the collision step (wall-cut cells)
  __shared__ long long sSc[3];  // shift of the collision step (angular correction)
  __shared__ float sCf[3][3];   // its float form and thresholds (mixed model)
  for (int sp = blockIdx.x; sp < nspans; sp += gridDim.x) {
    const int2 tt = spans[sp];
    const BoxDev& B = boxes[tt.x];
    const unsigned long long t = B.step;
    __syncthreads();
    if (threadIdx.x == 0) {
      if (MODE != MODE_C) shift_units(B, MODE == MODE_P ? t : t + 1ull, sSn);
      if (EXTRA && MODE != MODE_P) {
        long long S[3];
        shift_units(B, t, S);
        sSz = S[2];
      }
      if (ANG && MODE != MODE_P) {
        shift_units(B, t, sSc);
        for (int k = 0; k < 3; ++k) shift_thresholds(sSc[k], sCf[0][k], sCf[1][k], sCf[2][k]);
      }
    }
    __syncthreads();
    const int cell = tt.y + (int)threadIdx.x;
    if (cell >= B.ncells) continue;
    const int cur = B.cur, out = cur ^ 1;
    const int K = B.K;
    const uint32_t n = B.cnt[cur][cell];
    if (MODE != MODE_C && n) B.cnt[cur][cell] = 0u;  // this set is written two steps on
    const int nrow = (int)n < K ? (int)n : K;
    const bool has_ovf = (int)n > K;
    R* row = ((R*)B.rows[cur]) + (size_t)cell * K;
    R* ovf = (R*)B.ovf_rec[cur];
    const uint32_t* ovf_cell = B.ovf_cell[cur];
    const uint32_t novf = has_ovf ? min(B.ovf_n[cur], (uint32_t)B.ovf_cap) : 0u;
    int b0 = 0, nbt = 0;
    if (EXTRA && MODE != MODE_P && B.nbead > 0) {
      const int g = cell / B.tc;
      b0 = (int)B.bstart[g];
      nbt = (int)B.bstart[g + 1] - b0;
    }
    auto bead_in = [&](int j, int& b) {
      b = (int)B.border[b0 + j];
      return B.bcell[b] == cell;
    };
    bool any = n > 0;
    if (EXTRA)
      for (int j = 0; j < nbt && !any; ++j) {
        int b;
        any = bead_in(j, b);
      }
    if (!any) continue;

    CellParams<T> prm;  // the Andersen rule keeps the mean random velocity in prm.n
    T om[3] = {(T)0, (T)0, (T)0}, rcm[3] = {(T)0, (T)0, (T)0};
    int ic[3] = {0, 0, 0};
    double sc[3] = {0.0, 0.0, 0.0};
    if (ANG && MODE != MODE_P) {
      ic[0] = cell % B.n[0];
      ic[1] = (cell / B.n[0]) % B.n[1];
      ic[2] = cell / (B.n[0] * B.n[1]);
#pragma unroll
      for (int k = 0; k < 3; ++k) sc[k] = (double)sSc[k] * 0x1p-32;
    }
    // position of a member relative to its cell, in the model's type
    auto rel = [&](const T r[3], T o[3]) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if constexpr (MIXED) o[k] = rel_pos_f(r[k], sCf[0][k], sCf[1][k], sCf[2][k]);
        else o[k] = rel_pos(r[k], sc[k], ic[k], B.L[k]);
      }
    };
    // Eq. at: random velocity of a member
    auto draw_dv = [&](uint32_t tag, T dv[3]) {
      if constexpr (MIXED) at_draw(B, t, tag, 0u, B.sig_f, dv);
      else at_draw(B, t, tag, 0u, B.sig, dv);
    };
    // the collision rule without the angular correction
    auto base_rule = [&](T w[3], uint32_t tag) {
      if (AT) {
        T dv[3];
        draw_dv(tag, dv);
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = (prm.u[k] + dv[k]) - prm.n[k];
      } else {
        collide_one<MIXED>(B, prm, w, THERMO);
      }
    };
    if (MODE != MODE_P) {
      // ---- cell properties (Sec. 3.5) ----
      CellAcc<MIXED> a;
      CellAcc<MIXED> ad;  // Andersen rule: sums of the random velocities
      AngAcc<MIXED> g;
      auto add_member = [&](const R* p) {
        if (AT || ANG) {
          T r[3], w[3];
          uint32_t tag;
          load_rec(p, r, w, tag);
          a.add_solvent(B, w);
          if (AT) {
            T dv[3];
            draw_dv(tag, dv);
            ad.add_solvent(B, dv);
          }
          if (ANG) {
            T x[3];
            rel(r, x);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              if constexpr (MIXED) g.q[k] += fix32_rne(x[k]);
              else g.q[k] += x[k];
            }
          }
        } else {
          T w[3];
          load_v(p, w);
          a.add_solvent(B, w);
        }
      };
#pragma unroll 4
      for (int k = 0; k < nrow; ++k) add_member(row + k);
      if (has_ovf)
        for (uint32_t j = 0; j < novf; ++j)
          if (ovf_cell[j] == (uint32_t)cell) add_member(ovf + j);
      // the FP64 model's energy about u (the mixed model has E_k from the
      // exact sums of the first pass)
      auto solvent_energy = [&](const T u[3], CellAcc<MIXED>& acc) {
        if constexpr (!MIXED) {
#pragma unroll 4
          for (int k = 0; k < nrow; ++k) {
            T w[3];
            load_v(row + k, w);
            acc.add_solvent_energy(B, w, u);
          }
          if (has_ovf)
            for (uint32_t j = 0; j < novf; ++j)
              if (ovf_cell[j] == (uint32_t)cell) {
                T w[3];
                load_v(ovf + j, w);
                acc.add_solvent_energy(B, w, u);
              }
        }
      };
      const double sz = EXTRA ? (double)sSz * 0x1p-32 : 0.0;
      T u[3];
      cell_mean<MIXED>(B, t, (uint32_t)cell, sz, a, EXTRA ? nbt : 0, bead_in, EXTRA, u);
      if (AT) {  // Eq. at: u and dbar = sum m dv / sum m
        T dbar[3];
        ad.mean_velocity(B, dbar, false);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          prm.u[k] = u[k];
          prm.n[k] = dbar[k];
        }
        prm.xi = (T)1;
      } else {
        if (THERMO) solvent_energy(u, a);
        cell_finish<MIXED>(B, t, (uint32_t)cell, a, u, EXTRA ? nbt : 0, bead_in, THERMO, EXTRA, prm,
                           err);
      }
      if (ANG) {
        // centre of mass in the cell frame, then dL = sum m r_c x (v - v')
        // and the inertia tensor about it
        const int ns = a.ns;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (MIXED) rcm[k] = (i64_to_float(g.q[k]) * 0x1p-32f) / small_to_float(ns);
          else rcm[k] = g.q[k] / (double)ns;
        }
        auto add_moment = [&](const R* p) {
          T r[3], w[3];
          uint32_t tag;
          load_rec(p, r, w, tag);
          T x[3], rc[3], v2[3] = {w[0], w[1], w[2]};
          rel(r, x);
          base_rule(v2, tag);
          T d[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            rc[k] = x[k] - rcm[k];
            d[k] = w[k] - v2[k];
          }
          const T cx[3] = {rc[1] * d[2] - rc[2] * d[1], rc[2] * d[0] - rc[0] * d[2],
                           rc[0] * d[1] - rc[1] * d[0]};
          const T te[6] = {rc[1] * rc[1] + rc[2] * rc[2], rc[0] * rc[1], rc[0] * rc[2],
                           rc[0] * rc[0] + rc[2] * rc[2], rc[1] * rc[2],
                           rc[0] * rc[0] + rc[1] * rc[1]};
          if constexpr (MIXED) {
#pragma unroll
            for (int k = 0; k < 3; ++k) g.l[k] += fix32_rne(cx[k]);
#pragma unroll
            for (int k = 0; k < 6; ++k) g.p[k] += fix32_rne(te[k]);
          } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) g.l[k] += B.m * cx[k];
#pragma unroll
            for (int k = 0; k < 6; ++k) g.p[k] += B.m * te[k];
          }
        };
        for (int k = 0; k < nrow; ++k) add_moment(row + k);
        if (has_ovf)
          for (uint32_t j = 0; j < novf; ++j)
            if (ovf_cell[j] == (uint32_t)cell) add_moment(ovf + j);
        T P[6], dL[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (MIXED) dL[k] = B.m_f * (i64_to_float(g.l[k]) * 0x1p-32f);
          else dL[k] = g.l[k];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          T e;
          if constexpr (MIXED) e = B.m_f * (i64_to_float(g.p[k]) * 0x1p-32f);
          else e = g.p[k];
          P[k] = (k == 1 || k == 2 || k == 4) ? -e : e;
        }
        solve_omega<T>(ns, P, dL, om);
      }
    }

    // ---- members: collide, then stream and bin for the next step ----
    auto process = [&](R* p) {
      T r[3], w[3];
      uint32_t tag;
      load_rec(p, r, w, tag);
      if (MODE != MODE_P) {
        if (AT || ANG) base_rule(w, tag);
        else collide_one<MIXED>(B, prm, w, THERMO);
        if (ANG) {  // v'' = v' + omega x r_c
          T x[3], rc[3];
          rel(r, x);
#pragma unroll
          for (int k = 0; k < 3; ++k) rc[k] = x[k] - rcm[k];
          w[0] = w[0] + (om[1] * rc[2] - om[2] * rc[1]);
          w[1] = w[1] + (om[2] * rc[0] - om[0] * rc[2]);
          w[2] = w[2] + (om[0] * rc[1] - om[1] * rc[0]);
        }
      }
      if (MODE == MODE_C) {
        store_rec(p, r, w, tag);
        return;
      }
      stream_one(B, r, w);
      const uint32_t c2 = cell_of(B, sSn, r, err);
      insert<MIXED>(B, out, c2, r, w, tag, err);
    };
#pragma unroll 2
    for (int k = 0; k < nrow; ++k) process(row + k);
    if (has_ovf)
      for (uint32_t j = 0; j < novf; ++j)
        if (ovf_cell[j] == (uint32_t)cell) process(ovf + j);
    if (EXTRA && MODE != MODE_P) {
      for (int j = 0; j < nbt; ++j) {
        int b;
        if (!bead_in(j, b)) continue;
        double w[3] = {B.svel[3 * b], B.svel[3 * b + 1], B.svel[3 * b + 2]};
        collide_bead<MIXED>(B, prm, w, THERMO);
        B.svel[3 * b] = w[0];
        B.svel[3 * b + 1] = w[1];
        B.svel[3 * b + 2] = w[2];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// State in and out.  The input is placed in the rows of the unshifted grid
// (any placement works: the next step re-bins after streaming).  Positions
// are stored as given; only the placement uses a wrapped copy.
// ---------------------------------------------------------------------------
template <bool MIXED>
__global__ void k_load(const BoxDev* __restrict__ box, const real_t<MIXED>* __restrict__ pos,
                       const real_t<MIXED>* __restrict__ vel, int* err) {
  using T = real_t<MIXED>;
  const BoxDev& B = *box;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.nsol; i += gridDim.x * blockDim.x) {
    const T r[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    const T v[3] = {vel[3 * i], vel[3 * i + 1], vel[3 * i + 2]};
    int c[3];
    for (int k = 0; k < 3; ++k) {
      const double L = B.L[k];
      double x = (double)r[k];
      x = x - L * floor(x / L);
      int q = (x >= 0.0 && x < L) ? (int)x : 0;
      if (q >= B.n[k]) q = B.n[k] - 1;
      c[k] = q;
    }
    if (B.walls) c[2] += 1;  // channel layers are 1 .. n_z of the n_z + 2 layers
    const uint32_t cell = (uint32_t)(c[0] + B.n[0] * (c[1] + B.n[1] * c[2]));
    insert<MIXED>(B, B.cur, cell, r, v, (uint32_t)i, err);
  }
}

// Records of the current set, written in input order; cell_out (optional)
// receives each particle's cell.
template <bool MIXED>
__global__ void k_extract(const BoxDev* __restrict__ box, real_t<MIXED>* __restrict__ pos,
                          real_t<MIXED>* __restrict__ vel, int32_t* __restrict__ cell_out) {
  using T = real_t<MIXED>;
  using R = rec_t<MIXED>;
  const BoxDev& B = *box;
  const int cur = B.cur;
  const int stride = gridDim.x * blockDim.x;
  const int K = B.K;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < B.ncells; cell += stride) {
    const uint32_t n = B.cnt[cur][cell];
    const int nrow = (int)n < K ? (int)n : K;
    const R* row = ((const R*)B.rows[cur]) + (size_t)cell * K;
    for (int k = 0; k < nrow; ++k) {
      T r[3], v[3];
      uint32_t tag;
      load_rec(row + k, r, v, tag);
      for (int q = 0; q < 3; ++q) {
        pos[3 * tag + q] = r[q];
        vel[3 * tag + q] = v[q];
      }
      if (cell_out) cell_out[tag] = cell;
    }
  }
  const uint32_t novf = min(B.ovf_n[cur], (uint32_t)B.ovf_cap);
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < novf; j += stride) {
    T r[3], v[3];
    uint32_t tag;
    load_rec(((const R*)B.ovf_rec[cur]) + j, r, v, tag);
    for (int q = 0; q < 3; ++q) {
      pos[3 * tag + q] = r[q];
      vel[3 * tag + q] = v[q];
    }
    if (cell_out) cell_out[tag] = (int32_t)B.ovf_cell[cur][j];
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <bool M, bool TH, bool EX, int MODE, bool AT, bool ANG>
static void* cells_fn() {
  return (void*)k_cells<M, TH, EX, MODE, AT, ANG>;
}

// variant bits: 1 thermostat, 2 walls or beads, 16 Andersen rule, 32 angular
// correction (the last two without walls or beads; the Andersen rule without
// the thermostat).
template <bool M, int MODE>
static void* cells_variant_m(int variant) {
  const bool th = (variant & 1) != 0, ex = (variant & 2) != 0;
  const bool at = (variant & 16) != 0, ang = (variant & 32) != 0;
  if (at) return ang ? cells_fn<M, false, false, MODE, true, true>()
                     : cells_fn<M, false, false, MODE, true, false>();
  if (ang) return th ? cells_fn<M, true, false, MODE, false, true>()
                     : cells_fn<M, false, false, MODE, false, true>();
  if (th) return ex ? cells_fn<M, true, true, MODE, false, false>()
                    : cells_fn<M, true, false, MODE, false, false>();
  return ex ? cells_fn<M, false, true, MODE, false, false>()
            : cells_fn<M, false, false, MODE, false, false>();
}

template <int MODE>
static void* cells_variant_mode(bool mixed, int variant) {
  return mixed ? cells_variant_m<true, MODE>(variant) : cells_variant_m<false, MODE>(variant);
}

static void* cells_variant(bool mixed, int variant, int mode) {
  if (mode == MODE_P) return cells_variant_mode<MODE_P>(mixed, variant);
  if (mode == MODE_F) return cells_variant_mode<MODE_F>(mixed, variant);
  return cells_variant_mode<MODE_C>(mixed, variant);
}

int cells_blocks_per_sm(bool mixed, int variant, int mode) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cells_variant(mixed, variant, mode), BLOCK, 0);
  return nb;
}

void launch_cells(bool mixed, int variant, int mode, const BoxDev* boxes, const int2* spans,
                  int nspans, int grid, int* err, cudaStream_t s) {
  if (nspans <= 0) return;
  void* args[] = {(void*)&boxes, (void*)&spans, (void*)&nspans, (void*)&err};
  cudaLaunchKernel(cells_variant(mixed, variant, mode), dim3(grid), dim3(BLOCK), args, 0, s);
}

static int grid_for_n(int n) {
  int g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 8192) g = 8192;
  return g;
}

void launch_load(bool mixed, const BoxDev* box, const void* pos, const void* vel, int n, int* err,
                 cudaStream_t s) {
  if (n <= 0) return;
  if (mixed)
    k_load<true><<<grid_for_n(n), 256, 0, s>>>(box, (const float*)pos, (const float*)vel, err);
  else
    k_load<false><<<grid_for_n(n), 256, 0, s>>>(box, (const double*)pos, (const double*)vel, err);
}

void launch_extract(bool mixed, const BoxDev* box, void* pos, void* vel, int32_t* cell_out,
                    int ncells, cudaStream_t s) {
  if (mixed)
    k_extract<true><<<grid_for_n(ncells), 256, 0, s>>>(box, (float*)pos, (float*)vel, cell_out);
  else
    k_extract<false><<<grid_for_n(ncells), 256, 0, s>>>(box, (double*)pos, (double*)vel, cell_out);
}

}  // namespace mpcd

namespace mpcd {

// ---------------------------------------------------------------------------
// Thermal initial state drawn on the device (input generation for batched and
// served jobs, not part of a step): positions uniform in the box, velocity
// components Gaussian with variance kT/m (Box-Muller), then the mean velocity
// removed, as the benchmark set-up of Sec. 4 / 4.1 does.  Particle i uses
// counters (i, 0..2) under its own purpose; the mean comes from exact int64
// fixed-point sums, so the state is reproducible.
// ---------------------------------------------------------------------------
constexpr uint32_t PURPOSE_INIT = 0x494E4954u;

struct InitParams {
  uint32_t seed_lo, seed_hi;
  double L[3];
  double sigma;
  int n;
};

__device__ __forceinline__ void init_draw(const InitParams& P, int i, double r[3], double v[3]) {
  const uint2 key = make_uint2(P.seed_lo, P.seed_hi ^ PURPOSE_INIT);
  const uint4 a = philox(make_uint4((uint32_t)i, 0u, 0u, 0u), key);
  const uint4 b = philox(make_uint4((uint32_t)i, 1u, 0u, 0u), key);
  const uint4 c = philox(make_uint4((uint32_t)i, 2u, 0u, 0u), key);
  r[0] = P.L[0] * ((double)a.x * 0x1p-32);
  r[1] = P.L[1] * ((double)a.y * 0x1p-32);
  r[2] = P.L[2] * ((double)a.z * 0x1p-32);
  const double u1 = unit53(b.x, b.y), u2 = unit53(b.z, b.w);
  const double u3 = unit53(c.x, c.y), u4 = unit53(c.z, c.w);
  const double rho1 = sqrt(-2.0 * log(1.0 - u1)), rho2 = sqrt(-2.0 * log(1.0 - u3));
  v[0] = P.sigma * (rho1 * cos(kTwoPi * u2));
  v[1] = P.sigma * (rho1 * sin(kTwoPi * u2));
  v[2] = P.sigma * (rho2 * cos(kTwoPi * u4));
}

__global__ void k_init_sum(InitParams P, unsigned long long* sums) {
  long long s[3] = {0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    double r[3], v[3];
    init_draw(P, i, r, v);
    for (int k = 0; k < 3; ++k) s[k] += __double2ll_rn(v[k] * 4294967296.0);
  }
  for (int k = 0; k < 3; ++k) {
    long long x = s[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sums[k], (unsigned long long)x);
  }
}

template <bool MIXED>
__global__ void k_init_write(InitParams P, const unsigned long long* sums, real_t<MIXED>* pos,
                             real_t<MIXED>* vel) {
  using T = real_t<MIXED>;
  double mean[3];
  for (int k = 0; k < 3; ++k)
    mean[k] = P.n > 0 ? ((double)(long long)sums[k] * 0x1p-32) / (double)P.n : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    double r[3], v[3];
    init_draw(P, i, r, v);
    for (int k = 0; k < 3; ++k) {
      T x = (T)r[k];
      if (!((double)x < P.L[k])) x = (T)0;  // rounding up to L wraps to 0
      pos[3 * i + k] = x;
      vel[3 * i + k] = (T)(v[k] - mean[k]);
    }
  }
}

void launch_init_thermal(bool mixed, int n, uint64_t seed, const double L[3], double sigma,
                         void* pos, void* vel, unsigned long long* sums, cudaStream_t s) {
  if (n <= 0) return;
  InitParams P;
  P.seed_lo = (uint32_t)seed;
  P.seed_hi = (uint32_t)(seed >> 32);
  for (int k = 0; k < 3; ++k) P.L[k] = L[k];
  P.sigma = sigma;
  P.n = n;
  int g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  cudaMemsetAsync(sums, 0, 3 * sizeof(unsigned long long), s);
  k_init_sum<<<g, 256, 0, s>>>(P, sums);
  if (mixed) k_init_write<true><<<g, 256, 0, s>>>(P, sums, (float*)pos, (float*)vel);
  else k_init_write<false><<<g, 256, 0, s>>>(P, sums, (double*)pos, (double*)vel);
}

}  // namespace mpcd
