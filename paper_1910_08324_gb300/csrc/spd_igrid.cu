// spd_igrid.cu -- IGRID search launches: the grids with more than 32 widths
// (IG(2), IG(3) and their layer variants), the batched search of every IGRID
// grid, and the dispatch of the coded grids to spd_igrid_coded.cu.  The kernel
// templates are in spd_igrid.cuh.
#include "spd_igrid.cuh"

namespace spd {

size_t igrid_smem_bytes(const spd_plan& plan, bool table) {
  switch (plan.d * 8 + plan.pl) {
#define SPD_IG_CASE(D, PL) \
  case D * 8 + PL:         \
    return ig_smem_bytes<D, PL>(plan, table);
    SPD_IG_CASE(0, 0)
    SPD_IG_CASE(0, 1)
    SPD_IG_CASE(1, 1)
    SPD_IG_CASE(1, 2)
    SPD_IG_CASE(2, 2)
    SPD_IG_CASE(2, 3)
    SPD_IG_CASE(3, 3)
    SPD_IG_CASE(3, 4)
#undef SPD_IG_CASE
    default: return 0;
  }
}

cudaError_t launch_igrid_batch(const spd_plan& plan, const SearchParams& p, cudaStream_t s) {
  const size_t smem = igrid_smem_bytes(plan, false);
  const bool coarse = plan.top >= kRing0;
  switch (plan.d * 8 + plan.pl) {
#define SPD_IG_BATCH(D, PL)                                                                   \
  case D * 8 + PL:                                                                            \
    return coarse ? launch_persistent(igrid_batch_kernel<D, PL, true>, smem, p.n_units, p, s) \
                  : launch_persistent(igrid_batch_kernel<D, PL, false>, smem, p.n_units, p, s);
    SPD_IG_BATCH(0, 0)
    SPD_IG_BATCH(0, 1)
    SPD_IG_BATCH(1, 1)
    SPD_IG_BATCH(1, 2)
    SPD_IG_BATCH(2, 2)
    SPD_IG_BATCH(2, 3)
    SPD_IG_BATCH(3, 3)
    SPD_IG_BATCH(3, 4)
#undef SPD_IG_BATCH
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_igrid(const spd_plan& plan, const SearchParams& p, cudaStream_t s) {
  const bool table = p.table != 0;
  const size_t smem = igrid_smem_bytes(plan, table);
  switch (plan.d * 8 + plan.pl) {
#define SPD_IG_LAUNCH(D, PL)                                                       \
  case D * 8 + PL:                                                                 \
    return table ? launch_ig<D, PL, true, -1>(plan, p, smem, s) : launch_ig<D, PL, false, -1>(plan, p, smem, s);
    SPD_IG_LAUNCH(2, 2)
    SPD_IG_LAUNCH(2, 3)
    SPD_IG_LAUNCH(3, 3)
    SPD_IG_LAUNCH(3, 4)
#undef SPD_IG_LAUNCH
    default: return launch_igrid_coded(plan, p, smem, s);
  }
}

}  // namespace spd
