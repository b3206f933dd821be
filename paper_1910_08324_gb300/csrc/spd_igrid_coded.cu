// spd_igrid_coded.cu -- launches of the coded IGRID grids (at most 32 widths:
// DIT, IG(0) with 2 layers, IG(1) with 2 or 4 layers), whose width index rides
// in the SNRs' low mantissa bits.  float32 input has its own instantiation with
// the input type fixed at compile time (no per-chunk type dispatch); other input
// types read it from the parameters.  Kernel templates: spd_igrid.cuh.
#include "spd_igrid.cuh"

namespace spd {

cudaError_t launch_igrid_coded(const spd_plan& plan, const SearchParams& p, size_t smem, cudaStream_t s) {
  const bool table = p.table != 0;
  const bool f32 = p.dtype == kDtF32;
  switch (plan.d * 8 + plan.pl) {
#define SPD_IGC_LAUNCH(D, PL)                                                                        \
  case D * 8 + PL:                                                                                   \
    static_assert(IgS<D, PL>::ENC, "coded grid");                                                    \
    if (f32)                                                                                         \
      return table ? launch_ig<D, PL, true, kDtF32>(plan, p, smem, s)                                \
                   : launch_ig<D, PL, false, kDtF32>(plan, p, smem, s);                              \
    return table ? launch_ig<D, PL, true, -1>(plan, p, smem, s) : launch_ig<D, PL, false, -1>(plan, p, smem, s);
    SPD_IGC_LAUNCH(0, 0)
    SPD_IGC_LAUNCH(0, 1)
    SPD_IGC_LAUNCH(1, 1)
    SPD_IGC_LAUNCH(1, 2)
#undef SPD_IGC_LAUNCH
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace spd
