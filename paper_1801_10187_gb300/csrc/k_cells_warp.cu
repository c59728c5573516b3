// k_cells_warp.cu -- launch dispatch of the fused SRD step of the mixed model
// (the kernel template is in k_cells_warp.cuh), and its instances with 32
// cells per warp; k_cells_warp_narrow.cu holds those with 8 and 16.
#include "k_cells_warp.cuh"

namespace mpcd {

template <bool TH, int MODE, bool FO, bool BE, bool AT, bool ANG = false, int CH = CHUNK>
static void* warp_fn() {
  return (void*)k_cells_warp<TH, MODE, FO, BE, AT, ANG, CH>;
}

// pass-2 chunk depth of the F mode of the SRD variants (tuned); 3 elsewhere
template <bool TH, bool FO, bool BE>
static void* warp_fn_chunk(int ch) {
  if (ch == 2) return warp_fn<TH, MODE_F, FO, BE, false, false, 2>();
  if (ch == 4) return warp_fn<TH, MODE_F, FO, BE, false, false, 4>();
  return warp_fn<TH, MODE_F, FO, BE, false, false, 3>();
}

template <int MODE, bool BE>
static void* warp_variant_mb(bool thermo, bool force, bool at, int ch) {
  if (at) return force ? warp_fn<false, MODE, true, BE, true>() : warp_fn<false, MODE, false, BE, true>();
  if (MODE == MODE_F) {
    if (thermo) return force ? warp_fn_chunk<true, true, BE>(ch) : warp_fn_chunk<true, false, BE>(ch);
    return force ? warp_fn_chunk<false, true, BE>(ch) : warp_fn_chunk<false, false, BE>(ch);
  }
  if (thermo) return force ? warp_fn<true, MODE, true, BE, false>() : warp_fn<true, MODE, false, BE, false>();
  return force ? warp_fn<false, MODE, true, BE, false>() : warp_fn<false, MODE, false, BE, false>();
}

template <int MODE>
static void* warp_variant_mode(bool thermo, bool force, bool beads, bool at, bool ang, int ch) {
  if (ang && thermo) return force ? warp_fn<true, MODE, true, false, false, true>()
                                  : warp_fn<true, MODE, false, false, false, true>();
  if (ang) return force ? warp_fn<false, MODE, true, false, false, true>()
                        : warp_fn<false, MODE, false, false, false, true>();
  return beads ? warp_variant_mb<MODE, true>(thermo, force, at, ch)
               : warp_variant_mb<MODE, false>(thermo, force, at, ch);
}

// ang: the angular-momentum correction (SRD without beads only).
static void* warp_variant(bool thermo, bool force, bool beads, bool at, bool ang, int mode, int ch) {
  if (mode == MODE_P) return warp_variant_mode<MODE_P>(thermo, force, beads, at, ang, ch);
  if (mode == MODE_F) return warp_variant_mode<MODE_F>(thermo, force, beads, at, ang, ch);
  return warp_variant_mode<MODE_C>(thermo, force, beads, at, ang, ch);
}

// the cells per warp and the chunk depth a launch actually uses: 8 or 16
// cells per warp (with chunks of 3) only in the F mode of the SRD variants
static int used_cpw(bool at, bool ang, int mode, int cpw) {
  return (mode == MODE_F && !at && !ang && (cpw == 8 || cpw == 16)) ? cpw : 32;
}
static int used_chunk(bool at, bool ang, int mode, int ch, int cpw) {
  if (used_cpw(at, ang, mode, cpw) != 32) return CHUNK;
  return (mode == MODE_F && !at && !ang && (ch == 2 || ch == 4)) ? ch : CHUNK;
}
static void* warp_kernel(bool thermo, bool force, bool beads, bool at, bool ang, int mode, int ch,
                         int cpw) {
  const int c = used_cpw(at, ang, mode, cpw);
  if (c != 32) return cells_warp_narrow_fn(thermo, force, beads, c);
  return warp_variant(thermo, force, beads, at, ang, mode, used_chunk(at, ang, mode, ch, c));
}
static size_t warp_smem(bool thermo, bool beads, bool at, bool ang, int ch) {
  if (ch == 2) return block_smem<2>(beads, at, ang, thermo);
  if (ch == 4) return block_smem<4>(beads, at, ang, thermo);
  return block_smem<3>(beads, at, ang, thermo);
}

int cells_warp_blocks_per_sm(bool thermo, bool force, bool beads, bool at, bool ang, int mode,
                             int chunk, int cpw) {
  const int ch = used_chunk(at, ang, mode, chunk, cpw);
  const void* fn = warp_kernel(thermo, force, beads, at, ang, mode, chunk, cpw);
  const size_t smem = warp_smem(thermo, beads, at, ang, ch);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, BLOCK, smem);
  return nb;
}

void launch_cells_warp(bool thermo, bool force, bool beads, bool at, bool ang, int mode,
                       const BoxDev* boxes, const int2* spans, int nspans, int grid, int chunk,
                       int cpw, int* err, cudaStream_t s) {
  if (nspans <= 0) return;
  const int ch = used_chunk(at, ang, mode, chunk, cpw);
  void* args[] = {(void*)&boxes, (void*)&spans, (void*)&nspans, (void*)&err};
  cudaLaunchKernel(warp_kernel(thermo, force, beads, at, ang, mode, chunk, cpw), dim3(grid),
                   dim3(BLOCK), args, warp_smem(thermo, beads, at, ang, ch), s);
}

}  // namespace mpcd
