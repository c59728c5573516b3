// kernels.h -- host-side launchers of the libmpcd kernels (internal).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "mpcd_internal.cuh"

namespace mpcd {

void launch_stream_bin(bool mixed, const BoxDev* boxes, const int2* tiles, int ntiles, int grid,
                       int* err, cudaStream_t s);
void launch_md_bin(const BoxDev* boxes, const int2* tiles, int ntiles, int chains_per_block,
                   int threads, int* err, cudaStream_t s);
void launch_scan(const ScanSeg* segs, const int2* tiles, int ntiles, uint32_t* tsum,
                 unsigned long long* gscan, uint32_t* toff, int grid, cudaStream_t s);
void launch_scatter(const BoxDev* boxes, const int2* tiles, int ntiles, int grid, cudaStream_t s);
void launch_bead_scatter(const BoxDev* boxes, const int2* tiles, int ntiles, cudaStream_t s);
// reorder every sort_period steps, then swap the buffers in (two launches)
void launch_permute(bool mixed, BoxDev* boxes, int nboxes, const int2* tiles, int ntiles,
                    int grid, cudaStream_t s);
// advance the step counters and clear the overflow queue
void launch_end_step(BoxDev* boxes, int nboxes, int* novf, cudaStream_t s);

size_t collide_smem_bytes(bool mixed, int cap, int bcap);
cudaError_t prepare_collide(bool mixed, size_t smem);
// variant = (thermostat ? 1 : 0) | (solute beads or walls ? 2 : 0)
int collide_blocks_per_sm(bool mixed, int variant, size_t smem);
void launch_collide(bool mixed, int variant, const BoxDev* boxes, const int2* tiles, int ntiles,
                    int grid, int cap, int bcap, size_t smem, int2* ovf, int* novf, int* err,
                    cudaStream_t s);
// tiles the fast path queued in ovf[0 .. *novf)
void launch_collide_overflow(bool mixed, const BoxDev* boxes, const int2* ovf, const int* novf,
                             int grid, int* err, cudaStream_t s);

// observables / diagnostics / state movement (k_obs.cu)
struct ObsCells {
  uint32_t* cnt;
  long long* mass;
  long long* p;  // 3 per cell
  long long* k;
  int ncells;
};
void launch_iota(uint32_t* a, int n, cudaStream_t s);
void launch_obs_particles(bool mixed, const BoxDev* box, ObsCells oc, double* partials,
                          int nblocks, cudaStream_t s);
void launch_obs_cells(ObsCells oc, double* partials, int nblocks, cudaStream_t s);
void launch_profile(bool mixed, const BoxDev* box, int nbins, double* sum, unsigned long long* cnt,
                    int n, double H, cudaStream_t s);
void launch_unpermute(bool mixed, const BoxDev* box, int n, cudaStream_t s);
void launch_last_cells(const BoxDev* box, int nsol, int nbead, int ncells, int32_t* cell_out,
                       int32_t* count_out, cudaStream_t s);

}  // namespace mpcd
