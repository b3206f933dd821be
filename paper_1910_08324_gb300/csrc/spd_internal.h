// spd_internal.h -- plan representation and kernel parameter blocks shared by the
// host side (spd_api.cu) and the kernels of libspd.so.  Not part of the ABI.
//
// The searched grids are all written as "levels" (GPU restatement of the
// paper's iterations/steps):
//
//   level j has unit u = 2^j samples; its start samples are s = p * u
//   (p = level position, so the boxcar separation is L_s = u), and each
//   candidate width is   L = base_j + m * u   for the block counts m of the level.
//
//   * exhaustive (Sec. 3.1, ideal search): one level, u = 1, base 0, m = 1..L_max.
//   * BoxDIT BD-K (Alg. 1): level i = iteration i, base c_i = K (2^i - 1)
//     (= L^{i-1}_MAX), m = 1..K; the base sum X_{c_i}[s] is the previous
//     level's widest boxcar at the same start (X^{i-1} of Alg. 1).
//   * IGRID IG(d) with P = 2^p layers (Sec. 3.2): steps i <= p all have L_s = 1
//     and form level 0, with the widths [1, 2^d) and 2^i + q 2^(i-d)
//     (q < 2^d, d <= i <= p); step p + j (j >= 1) is level j with unit 2^j and
//     block counts m = 2^p + q 2^(p-d), q < 2^d (Eq. boxcarsize, Table 1).
//
// Widths of level j are larger than those of level j-1, so the plan's
// ascending width table lists the levels one after the other.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "spd.h"

namespace spd {

constexpr int kThreads = 256;      // threads per search CTA
constexpr int kChunk = 2048;       // starts per sub-chunk of a tile (fine levels)
constexpr int kMaxLevels = 24;     // levels a plan may have
constexpr int kMaxLend = 32768;    // largest width a plan may reach
constexpr int kMaxExhaustive = 4096;
constexpr int kMaxGridWidths = 512;  // widths of a BoxDIT / IGRID plan
constexpr int kMaxRanges = 8;        // DM ranges of one batched search

// One range of a batched search (spd_batch_execute): its own series, outputs,
// white-noise statistics, tile maxima (in the workspace) and optional ready flag.
struct BatchRange {
  const void* x;
  float* snr;
  uint16_t* widx;
  const float* mu;
  const float* sigma;
  float* tile_max;          // [ndm * cand_tiles_per_row] ordered-int keys
  const int32_t* ready;     // nullptr, or a flag the units of this range wait for
  int64_t ndm, nt, ld;
  int64_t unit_first;       // index of the range's first unit (row-major: row, segment)
  int32_t tile, tiles_per_row, cand_tiles_per_row, vec, vec_x, pad;
};
constexpr int kCandTile = 16384;   // starts per candidate tile (tile maxima granularity)
constexpr int kMaxPeakRadius = 64;
constexpr int kCandGroup = 32;     // candidate tiles per warp of the candidate passes
constexpr int64_t kStaticCandTiles = 262144;  // candidate tiles spd_candidates_static can hold

enum Family { kExhaustive = 0, kBoxdit = 1, kIgrid = 2 };

// General BoxDIT kernel (spd_boxdit_gen.cu): offsets of its shared-memory
// regions in SearchParams::gen_off, and the largest L^i_max of a plan.
enum BdgRegion { kBdgX0 = 0, kBdgXA, kBdgXB, kBdgBA, kBdgBB, kBdgY, kBdgW, kBdgYC, kBdgWC, kBdgAB, kBdgOffsets };
constexpr int kMaxBoxditK = 256;

// Search kernel parameters (passed by value; lives in the constant bank).
struct SearchParams {
  const void* x;        // [ndm][ld] samples of type dtype
  float* snr;
  uint16_t* widx;
  float* tile_max;      // [ndm * cand_tiles_per_row] ordered-int keys of tile maxima (or nullptr)
  const float* mu;      // white: [ndm]; table: [ndm][n_widths]
  const float* sigma;
  int64_t ndm, nt, ld;
  int64_t n_starts;     // starts evaluated per row (<= nt; samples up to nt feed them)
  int32_t tile;         // starts per CTA (multiple of kChunk; streaming kernels: of kCandTile)
  int32_t tiles_per_row;
  int32_t cand_tiles_per_row;  // ceil(nt / kCandTile)
  int32_t halo;         // samples read past the segment (widest boxcar, whole 2048-sample chunks)
  int32_t top;          // index of the last level
  int32_t n_top;        // block counts used on the last level (a prefix of its set)
  int32_t vec;          // 1: vector stores of Y and W are legal (16-byte Y rows, 8-byte W rows)
  int32_t vec_x;        // 1: x rows and base are 16-byte aligned (vector loads)
  int32_t dtype;        // spd_dtype of x
  int32_t esize;        // bytes per sample of x
  int32_t lmax;         // exhaustive: widest boxcar
  int32_t lvl_first[kMaxLevels];  // width-table index of each level's first width
  float lvl_scale[kMaxLevels];    // IGRID: 2^(-j/2), the unit factor of level j
  float rs[64];                   // rs[m] = 1/sqrt(m) (IGRID block-count factor)
  float bscale[kMaxLevels][33];   // BoxDIT: 1/sqrt(c_j + m 2^j), m = 1..K; IGRID: 1/sqrt(m 2^j), every level
  int32_t table;                  // 1: per-row, per-width noise statistics (spd_noise mode 1)
  int32_t n_widths;               // widths of the plan
  int32_t unit_widths;            // 1: width index w is width w + 1 (exhaustive grid)
  int32_t wtab[kMaxGridWidths];   // widths of the plan (table noise, unit_widths == 0)
  int32_t grid;                   // 1: explicit width set (spd_plan_create_grid), exhaustive kernel
  int32_t wsep[kMaxGridWidths];   // explicit set: start separation of each width (a power of two)
  // batched search: units are (range, row, segment); 0 ranges: the single series above
  int32_t n_ranges;
  int64_t n_units;
  int32_t* status;                // bit r: a wait for range r's ready flag ran out
  int64_t wait_ns;                // limit of one wait
  int32_t ctas_per_sm;            // persistent CTAs per SM (0: as many as fit)
  // general BoxDIT: block counts k_i of every level, window lengths of the
  // decimated series, shared-memory offsets (floats) and 1/sqrt(L) per width
  int32_t lvl_k[kMaxLevels];
  int32_t gen_len[kMaxLevels];
  int32_t gen_off[kBdgOffsets];
  float wscale[kMaxGridWidths];
  // the two-kernel form of larger plans: the first kernel runs levels below
  // gen_h and writes x^gen_h and the bases X^{gen_h - 1} of every row to gen_xh /
  // gen_bh and its SNRs and width indices at the starts of level gen_h to gen_yh
  // / gen_wh (all [ndm][gen_ldh]); the second runs levels gen_h..top on them
  int32_t gen_h;
  float* gen_xh;
  float* gen_bh;
  float* gen_yh;
  uint16_t* gen_wh;
  int64_t gen_ldh;
  BatchRange ranges[kMaxRanges];
};

// Noise-statistics kernels (spd_msd.cu).
constexpr int kMsdMaxLevels = 16;  // decimation levels 2^0 .. 2^15 (kMaxLend = 2^15)
struct MsdParams {
  const void* x;
  int64_t ndm, nt, ld;
  int32_t dtype, esize, vec_x;
  int32_t nlev;         // levels computed (2^(nlev-1) >= the widest boxcar)
  float thr;            // outlier threshold in deviations; <= 0: no rejection
  void* state;          // workspace: [ndm][kMsdMaxLevels] level statistics
  float* out_mu;        // [ndm][n_widths]
  float* out_sigma;
  int32_t n_widths, unit_widths;
  int32_t wtab[kMaxGridWidths];
};

struct CandParams {
  const float* snr;
  const uint16_t* widx;
  const float* tile_max;   // ordered-int keys (see fkey) of tile maxima; nullptr: scan every tile
  int32_t* counts;         // [tiles] candidates per tile
  int32_t* gsum;           // [groups] candidates per group of kCandGroup tiles
  int64_t* goff;           // [groups] record offset of each group
  spd_candidate* out;
  int64_t* d_count;
  int64_t ndm, nt, ld, cap;
  int32_t tile, tiles_per_row;
  int32_t radius;
  float thr;
  int32_t width_mode;      // 0: width = index + 1 (exhaustive); 1: width_tab[index]
  int32_t width_tab[512];  // plan widths (index -> samples) when width_mode == 1
  // only starts in [s_lo, s_hi) are candidates (their peak test still reads the
  // neighbours below nt); default [0, nt)
  int64_t s_lo, s_hi;
  // proposal search (spd_propose_search): row k of the searched series is block
  // row_ids[k] = r * map_bpr + b of the original one; records are written with
  // row r and start b * map_block + s - s_lo.  nullptr: records as searched.
  // The peak test of a mapped row only reads neighbours inside the original
  // series (map_nt samples per row), as a search of the whole row would.
  const int64_t* row_ids;
  int64_t map_bpr, map_nt;
  int32_t map_block;
};

}  // namespace spd

struct spd_plan {
  spd_plan_desc desc;
  int family;
  int k;          // BoxDIT L^i_max of the streaming kernel (8, 16 or 32); 0: general kernel
  bool bd_general = false;  // BoxDIT served by the general kernel (spd_boxdit_gen.cu)
  std::vector<int32_t> lvl_k;  // BoxDIT L^i_max of every level
  int d, pl;      // IGRID depth and log2(layers)
  int top;        // last level index
  int n_top;      // block counts used on the last level
  int lend;       // largest width
  int64_t n_starts;  // starts evaluated per row (spd_plan_set_starts; default nt)
  bool explicit_grid = false;  // widths and separations given by the caller (spd_plan_create_grid)
  int tile;       // starts per search CTA
  int halo;
  int64_t tiles_per_row;       // search CTAs per row
  int64_t cand_tiles_per_row;  // candidate tiles (kCandTile starts) per row
  std::vector<int32_t> widths, seps;
  std::vector<int32_t> lvl_first;
  std::vector<int32_t> lvl_base;  // base width of each level (BoxDIT c_j)
};

namespace spd {
// kernel launchers (spd_search.cu, spd_igrid.cu, spd_igrid_coded.cu, spd_boxdit.cu, spd_candidates.cu, spd_msd.cu)
cudaError_t launch_search(const spd_plan& plan, const SearchParams& p, cudaStream_t s);
cudaError_t launch_igrid(const spd_plan& plan, const SearchParams& p, cudaStream_t s);
cudaError_t launch_igrid_coded(const spd_plan& plan, const SearchParams& p, size_t smem, cudaStream_t s);
size_t igrid_smem_bytes(const spd_plan& plan, bool table);
cudaError_t launch_boxdit(const spd_plan& plan, const SearchParams& p, cudaStream_t s);
size_t boxdit_smem_bytes(const spd_plan& plan, bool table);
// general BoxDIT (spd_boxdit_gen.cu): layout of a plan with tiles of T starts
// (window lengths into len[kMaxLevels], offsets into off[kBdgOffsets]; returns floats)
// part 0: every level in one kernel; 1: levels below h (writing x^h, the bases
// X^{h-1} and a copy of the results at level h's starts); 2: levels h..top of
// the series x^h, in tiles of T positions
int bdg_layout(const spd_plan& plan, int T, bool table, int32_t* len, int32_t* off, int part = 0, int h = 0);
constexpr int kBdgSplit = 4;     // general BoxDIT plans above this level run in two kernels
constexpr int kBdgTile2 = 2048;  // level-kBdgSplit positions per tile of the second
constexpr size_t kBdgMaxSmem = 227 * 1024;  // shared memory of one CTA at most
// positions of x^h kept per row (the first kernel covers the row in tiles of T starts)
inline int64_t bdg_ldh(int64_t nt, int T) { return ((nt + T - 1) / T) * (int64_t)(T >> kBdgSplit); }
// whether a plan runs in the two-kernel form (general BoxDIT above level
// kBdgSplit, both kernels' layouts within kBdgMaxSmem)
bool bdg_two_part(const spd_plan& plan);
size_t boxdit_gen_smem_bytes(const spd_plan& plan, bool table);
cudaError_t launch_boxdit_gen(const spd_plan& plan, const SearchParams& p, cudaStream_t s);
cudaError_t launch_boxdit_gen_batch(const spd_plan& plan, const SearchParams& p, cudaStream_t s);
// Shared-memory attribute, CTAs per SM (of `threads` threads each) and SM count
// of a persistent kernel, set and queried on the first call per (kernel, device,
// shared memory, threads) and
// cached, so that later launches (e.g. during stream capture) make no queries.
cudaError_t persistent_config(const void* kernel, size_t smem, int* per_sm, int* sms, int threads = kThreads);
cudaError_t launch_igrid_batch(const spd_plan& plan, const SearchParams& p, cudaStream_t s);
// proposal network (spd_net.cu)
int net_param_count();
cudaError_t launch_net_forward(const float* P, const float* X, int64_t nb, float* logits, cudaStream_t s);
cudaError_t launch_net_grad(const float* P, const float* X, const float* Y, int64_t nb, float* G, float* loss,
                            float* partials, cudaStream_t s);
size_t net_grad_workspace_bytes();
cudaError_t launch_net_adam(float* P, float* M, float* V, const float* G, int64_t nb, float lr, int step,
                            cudaStream_t s);
cudaError_t launch_net_decimate(const void* x, int dtype, int esize, int64_t ndm, int64_t nt, int64_t ld,
                                bool vec, const float* mu, const float* sigma, float* out, cudaStream_t s);
cudaError_t launch_net_select(const float* logits, int64_t n, float thr, int64_t* list, int64_t cap,
                              int64_t* count, cudaStream_t s);
cudaError_t launch_net_gather(const void* x, int dtype, int esize, int64_t ndm, int64_t nt, int64_t ld,
                              const int64_t* list, int64_t n, int block, int left, int width, void* out,
                              int64_t ld_out, bool vec, cudaStream_t s);
cudaError_t launch_gather_rows(const float* src, int64_t len, const int64_t* ids, int64_t n, int64_t bpr,
                               int64_t ndm, float fill, float* dst, cudaStream_t s);
cudaError_t launch_boxdit_batch(const spd_plan& plan, const SearchParams& p, cudaStream_t s);
cudaError_t launch_candidates(const spd_plan& plan, CandParams& p, cudaStream_t s);
cudaError_t launch_candidates_static(const spd_plan& plan, CandParams& p, cudaStream_t s);
size_t search_smem_bytes(const spd_plan& plan, bool table);
size_t msd_state_bytes(int64_t ndm);
cudaError_t launch_msd(const spd_plan& plan, const MsdParams& p, int max_passes, cudaStream_t s);
}  // namespace spd
