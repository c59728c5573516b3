// k_obs.cu -- observables (arXiv:1801.10187, Sec. 3.5 last paragraph: net
// momentum, energy and temperature), the z profile of v_x used for the
// Poiseuille check, and the member counts of the last step.  They read the
// state in input order, as k_extract writes it.
#include <type_traits>

#include "kernels.h"
#include "mpcd_internal.cuh"

namespace mpcd {

// Per-particle pass: block partial sums of P and KE (double, fixed block
// decomposition) and fixed-point sums per cell of the unshifted grid.
template <bool MIXED>
__global__ void __launch_bounds__(256) k_obs_particles(const BoxDev* __restrict__ box,
                                                       const real_t<MIXED>* __restrict__ pos,
                                                       const real_t<MIXED>* __restrict__ vel,
                                                       ObsCells oc, double* __restrict__ partials) {
  const BoxDev& B = *box;
  __shared__ double red[4][256];
  double acc[4] = {0, 0, 0, 0};
  const int ntot = B.nsol + B.nbead;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ntot; i += gridDim.x * blockDim.x) {
    double x[3], w[3], m;
    if (i < B.nsol) {
      for (int k = 0; k < 3; ++k) {
        x[k] = (double)pos[3 * i + k];
        w[k] = (double)vel[3 * i + k];
      }
      m = B.m;
    } else {
      const int b = i - B.nsol;
      for (int k = 0; k < 3; ++k) {
        x[k] = B.spos[3 * b + k];
        w[k] = B.svel[3 * b + k];
      }
      m = B.Mb;
    }
    const double e = (0.5 * m) * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int k = 0; k < 3; ++k) acc[k] += m * w[k];
    acc[3] += e;
    int c[3];
    for (int k = 0; k < 3; ++k) {
      int q = (int)floor(x[k]);
      if (q < 0) q = 0;
      if (q >= B.n[k]) q = B.n[k] - 1;
      c[k] = q;
    }
    const int cell = c[0] + B.n[0] * (c[1] + B.n[1] * c[2]);
    atomicAdd(&oc.cnt[cell], 1u);
    atomicAdd((unsigned long long*)&oc.mass[cell], (unsigned long long)__double2ll_rn(m * 4294967296.0));
    for (int k = 0; k < 3; ++k)
      atomicAdd((unsigned long long*)&oc.p[3 * cell + k],
                (unsigned long long)__double2ll_rn((m * w[k]) * 4294967296.0));
    atomicAdd((unsigned long long*)&oc.k[cell], (unsigned long long)__double2ll_rn(e * 4294967296.0));
  }
  for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) partials[4 * blockIdx.x + q] = red[q][0];
}

// Per-cell pass: sum of cell temperatures over cells with >= 2 members, the
// number of such cells and the number of occupied cells (block partials).
__global__ void __launch_bounds__(256) k_obs_cells(ObsCells oc, double* __restrict__ partials) {
  __shared__ double red[3][256];
  double a[3] = {0, 0, 0};
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < oc.ncells; c += gridDim.x * blockDim.x) {
    const uint32_t n = oc.cnt[c];
    if (n >= 1) a[2] += 1.0;
    if (n >= 2) {
      const double M = (double)oc.mass[c] * 0x1p-32;
      const double P0 = (double)oc.p[3 * c] * 0x1p-32, P1 = (double)oc.p[3 * c + 1] * 0x1p-32,
                   P2 = (double)oc.p[3 * c + 2] * 0x1p-32;
      const double K = (double)oc.k[c] * 0x1p-32;
      const double pp = P0 * P0 + P1 * P1 + P2 * P2;
      const double Ek = K - pp / (2.0 * M);
      a[0] += 2.0 * Ek / (3.0 * (double)(n - 1));
      a[1] += 1.0;
    }
  }
  for (int q = 0; q < 3; ++q) red[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) partials[3 * blockIdx.x + q] = red[q][0];
}

template <bool MIXED>
__global__ void k_profile(const real_t<MIXED>* __restrict__ pos, const real_t<MIXED>* __restrict__ vel,
                          int n, int nbins, double* sum, unsigned long long* cnt, double H) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    long long b = (long long)floor((double)pos[3 * i + 2] / H * (double)nbins);
    if (b < 0) b = 0;
    if (b >= nbins) b = nbins - 1;
    atomicAdd(&sum[b], (double)vel[3 * i]);
    atomicAdd(&cnt[b], 1ull);
  }
}

// Member counts of the current cells: solvent from the row counts, then the
// beads of the step.
__global__ void k_cell_counts(const BoxDev* __restrict__ box, int32_t* count_out) {
  const BoxDev& B = *box;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < B.ncells; c += gridDim.x * blockDim.x)
    count_out[c] = (int32_t)B.cnt[B.cur][c];
}
__global__ void k_bead_cells(const BoxDev* __restrict__ box, int32_t* cell_out, int32_t* count_out) {
  const BoxDev& B = *box;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B.nbead; b += gridDim.x * blockDim.x) {
    const int32_t c = B.bcell[b];
    if (cell_out) cell_out[B.nsol + b] = c;
    if (count_out) atomicAdd(&count_out[c], 1);
  }
}

static int grid_for(int n, int per_block) {
  int g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return g;
}

void launch_obs_particles(bool mixed, const BoxDev* box, const void* pos, const void* vel,
                          ObsCells oc, double* partials, int nblocks, cudaStream_t s) {
  if (mixed)
    k_obs_particles<true><<<nblocks, 256, 0, s>>>(box, (const float*)pos, (const float*)vel, oc, partials);
  else
    k_obs_particles<false><<<nblocks, 256, 0, s>>>(box, (const double*)pos, (const double*)vel, oc,
                                                   partials);
}

void launch_obs_cells(ObsCells oc, double* partials, int nblocks, cudaStream_t s) {
  k_obs_cells<<<nblocks, 256, 0, s>>>(oc, partials);
}

void launch_profile(bool mixed, const void* pos, const void* vel, int n, int nbins, double* sum,
                    unsigned long long* cnt, double H, cudaStream_t s) {
  const int g = grid_for(n, 256);
  if (mixed) k_profile<true><<<g, 256, 0, s>>>((const float*)pos, (const float*)vel, n, nbins, sum, cnt, H);
  else k_profile<false><<<g, 256, 0, s>>>((const double*)pos, (const double*)vel, n, nbins, sum, cnt, H);
}

void launch_cell_counts(const BoxDev* box, int ncells, int nbead, int32_t* cell_out,
                        int32_t* count_out, cudaStream_t s) {
  if (count_out) k_cell_counts<<<grid_for(ncells, 256), 256, 0, s>>>(box, count_out);
  if (nbead > 0) k_bead_cells<<<grid_for(nbead, 256), 256, 0, s>>>(box, cell_out, count_out);
}

}  // namespace mpcd
