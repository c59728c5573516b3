// k_cells_warp_narrow.cu -- the fused SRD step of the mixed model with 8 or 16
// cells per warp (F mode of the SRD variants, pass-2 chunks of 3 windows): the
// launch tuner's candidates for boxes that 32 cells per warp spread over too
// few blocks.  Kernel template: k_cells_warp.cuh.
#include "k_cells_warp.cuh"

namespace mpcd {

template <bool TH, bool FO, bool BE, int CPW>
static void* narrow_fn() {
  return (void*)k_cells_warp<TH, MODE_F, FO, BE, false, false, 3, CPW>;
}

template <int CPW>
static void* narrow_cpw(bool thermo, bool force, bool beads) {
  if (thermo) {
    if (force) return beads ? narrow_fn<true, true, true, CPW>() : narrow_fn<true, true, false, CPW>();
    return beads ? narrow_fn<true, false, true, CPW>() : narrow_fn<true, false, false, CPW>();
  }
  if (force) return beads ? narrow_fn<false, true, true, CPW>() : narrow_fn<false, true, false, CPW>();
  return beads ? narrow_fn<false, false, true, CPW>() : narrow_fn<false, false, false, CPW>();
}

void* cells_warp_narrow_fn(bool thermo, bool force, bool beads, int cpw) {
  return cpw == 8 ? narrow_cpw<8>(thermo, force, beads) : narrow_cpw<16>(thermo, force, beads);
}

}  // namespace mpcd
