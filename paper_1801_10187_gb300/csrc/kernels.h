// kernels.h -- host-side launchers of the libmpcd kernels (internal).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "mpcd_internal.cuh"

namespace mpcd {

// ---- fused step on cell rows (k_cells.cu) ----
// mode: MODE_P stream + bin, MODE_F collide + stream + bin, MODE_C collide in place.
// variant = (thermostat ? 1 : 0) | (solute beads or walls ? 2 : 0) |
// (Andersen rule ? 16 : 0) | (angular-momentum correction ? 32 : 0); the last
// two without solute or walls.
// Solute MD of one collision step for the boxes with the non-bonded WCA
// repulsion (k_wca.cu): neighbour-list build, then max_substeps velocity-
// Verlet substeps (each box takes its own md_substeps).
void launch_wca_md(const BoxDev* boxes, const int2* tiles, int ntiles, int max_substeps, int* err,
                   cudaStream_t s);
int cells_blocks_per_sm(bool mixed, int variant, int mode);
void launch_cells(bool mixed, int variant, int mode, const BoxDev* boxes, const int2* spans,
                  int nspans, int grid, int* err, cudaStream_t s);
// The same step for mixed-model boxes without walls, members spread over the
// lanes of a warp (k_cells_warp.cu); valid for row capacities up to
// WARP_MAX_K and boxes below 2^22 cells per axis.  force: nonzero body force;
// beads: the box has solute beads; at: Andersen-thermostat rule (Eq. at)
// instead of the rotation (thermo is then false).
constexpr int WARP_MAX_K = 448;
// ang (mixed model, SRD without beads): the angular-momentum correction.
// chunk: windows of 32 members whose loads and slot requests pass 2 keeps in
// flight together (2, 3 or 4; used by the F mode of the SRD variants, 3
// elsewhere); cpw: cells per warp (8, 16 or 32; 8 and 16 only in the F mode
// of the SRD variants, with chunks of 3, 32 elsewhere).  Both are launch-tuner
// choices.  With cpw < 32 a 256-cell span is taken in 32 / cpw parts, each by
// one block: grid sizes count parts.
int cells_warp_blocks_per_sm(bool thermo, bool force, bool beads, bool at, bool ang, int mode,
                             int chunk, int cpw);
void launch_cells_warp(bool thermo, bool force, bool beads, bool at, bool ang, int mode,
                       const BoxDev* boxes, const int2* spans, int nspans, int grid, int chunk,
                       int cpw, int* err, cudaStream_t s);
// The FP64 model's counterpart (k_cells_warp_d.cu), same conditions.
int cells_warpd_blocks_per_sm(bool thermo, bool force, bool beads, bool at, int mode);
void launch_cells_warpd(bool thermo, bool force, bool beads, bool at, int mode, const BoxDev* boxes,
                        const int2* spans, int nspans, int grid, int* err, cudaStream_t s);
// Place n particles (device arrays of float (mixed) or double, n x 3) in the
// current rows of a box whose counts are zero.
void launch_load(bool mixed, const BoxDev* box, const void* pos, const void* vel, int n, int* err,
                 cudaStream_t s);
// Current state into device arrays in input order (cell_out optional).
void launch_extract(bool mixed, const BoxDev* box, void* pos, void* vel, int32_t* cell_out,
                    int ncells, cudaStream_t s);

// Thermal initial state drawn on the device into pos/vel (n x 3 of the storage
// type); sums: 3 device words of scratch.
void launch_init_thermal(bool mixed, int n, uint64_t seed, const double L[3], double sigma,
                         void* pos, void* vel, unsigned long long* sums, cudaStream_t s);

// ---- solute and pass bookkeeping (k_step.cu) ----
// Allows k_md_bin the shared memory of 1024-thread blocks; returns a cudaError_t.
int md_bin_prepare();
void launch_md_bin(const BoxDev* boxes, const int2* tiles, int ntiles, int chains_per_block,
                   int threads, int* err, cudaStream_t s);
void launch_scan(const ScanSeg* segs, const int2* tiles, int ntiles, uint32_t* tsum,
                 unsigned long long* gscan, uint32_t* toff, int grid, cudaStream_t s);
void launch_bead_scatter(const BoxDev* boxes, const int2* tiles, int ntiles, cudaStream_t s);
// flip: the output set becomes current (after modes P and F); advance: step += 1
// (after modes F and C).
void launch_after_pass(BoxDev* boxes, int nboxes, bool flip, bool advance, cudaStream_t s);

// ---- observables (k_obs.cu) ----
struct ObsCells {
  uint32_t* cnt;
  long long* mass;
  long long* p;  // 3 per cell
  long long* k;
  int ncells;
};
void launch_obs_particles(bool mixed, const BoxDev* box, const void* pos, const void* vel,
                          ObsCells oc, double* partials, int nblocks, cudaStream_t s);
void launch_obs_cells(ObsCells oc, double* partials, int nblocks, cudaStream_t s);
void launch_profile(bool mixed, const void* pos, const void* vel, int n, int nbins, double* sum,
                    unsigned long long* cnt, double H, cudaStream_t s);
void launch_cell_counts(const BoxDev* box, int ncells, int nbead, int32_t* cell_out,
                        int32_t* count_out, cudaStream_t s);

}  // namespace mpcd
