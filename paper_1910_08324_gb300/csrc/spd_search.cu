// spd_search.cu -- the exhaustive search kernel and the search dispatch (sm_103a).
//
// What every search kernel computes (Eq. boxcar, Eq. SNRlong with Eq.
// whitenoise, Eq. MSD03): for every row and start s, the largest SNR over the
// plan's eligible widths and the index of the smallest width reaching it.  Each
// sample is normalised once on load, z = (x - mu_r) / sigma_r, so a width-L
// boxcar's SNR is (sum of L z-values) / sqrt(L).  Samples past the end of a row
// load as -inf, so a boxcar that would need them sums to -inf and can never be
// the maximum: that is the rule s + L <= nt.
//
// The exhaustive search (Sec. 3.1, the ideal grid: every width 1..L_max at
// every start) runs one CTA per 2048-start tile: the tile and its lookahead are
// staged once in shared memory, each thread owns 4 starts and extends their
// running sums width by width in register windows (32 widths per window),
// with 1/sqrt(L) from a shared table; each candidate of a window carries its
// rank in the 5 low mantissa bits, so the window's maximum is one three-input
// max per two candidates, decoded and merged with a strict '>' after the window.  The tile maximum goes to the workspace
// for the candidate step.  Only starts below the plan's n_starts are stored;
// samples up to nt feed them.  BoxDIT and IGRID have streaming kernels of their
// own (spd_boxdit.cu, spd_igrid.cu).
#include "spd_common.cuh"

namespace spd {
namespace {

constexpr int kItems0 = kChunk / 4 / kThreads;  // 4-start items per thread per tile
static_assert(kItems0 * 4 * kThreads == kChunk, "tile must split evenly");

// ============================================================================ exhaustive
// table: the scale table holds (a, b) float2 pairs (table noise) instead of 1/sqrt(L)
static_assert(kAbPad <= 33, "the exhaustive scale table pads 33 entries");
// grid: an explicit width set, with per-block-count tables of the width index
// (-1 outside the set) and of the start mask (separation - 1)
struct ExLayout {
  int f0, rs, red, ix, ms, total;
  __host__ __device__ ExLayout(int lmax, bool table, bool grid) {
    int o = 0;
    f0 = o;
    o += al4(kChunk + ((lmax + 36 + 127) / 128) * 128 + 8);
    rs = o;
    o += al4((lmax + 33) * (table ? 2 : 1));  // table: lmax widths + kAbPad (<= 33) padding pairs
    red = o;
    o += 32;
    ix = o;
    o += grid ? al4(lmax + 33) : 0;
    ms = o;
    o += grid ? al4(lmax + 33) : 0;
    total = o;
  }
};

// GRID: the widths of an explicit set only (p.wtab, p.wsep; width 1 at every
// start): the running sums still advance one sample per block count m, and
// width m is a candidate at start s iff it is in the set and s is a multiple of
// its separation; the stored width index is its index in the set.
template <bool TABLE, bool GRID>
__global__ void __launch_bounds__(kThreads, 2) exhaustive_kernel(const SearchParams p) {
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t row = blockIdx.x / p.tiles_per_row;
  const int64_t tile = blockIdx.x % p.tiles_per_row;
  const int64_t t0 = tile * (int64_t)kChunk;
  const int lmax = p.lmax;
  const unsigned char* __restrict__ xrow = static_cast<const unsigned char*>(p.x) + row * p.ld * p.esize;

  const bool vec = p.vec != 0;
  const ExLayout L(lmax, TABLE, GRID);
  float* F0 = smem + L.f0;
  float* RS = smem + L.rs;  // white noise: RS[m] = 1/sqrt(m); table noise: AB[m - 1] = (a, b)
  float2* AB = reinterpret_cast<float2*>(smem + L.rs);
  float mu, inv;
  row_noise<TABLE>(p, p.mu, p.sigma, row, AB, mu, inv);
  if constexpr (!TABLE)
    for (int m = tid; m <= lmax + 32; m += kThreads)
      RS[m] = (m >= 1 && m <= lmax) ? (float)(1.0 / sqrt((double)m)) : 0.0f;
  int* IX = reinterpret_cast<int*>(smem + L.ix);
  int* MS = reinterpret_cast<int*>(smem + L.ms);
  if constexpr (GRID) {
    for (int m = tid; m <= lmax + 32; m += kThreads) {
      IX[m] = -1;
      MS[m] = 0;
    }
    __syncthreads();
    for (int i = tid; i < p.n_widths; i += kThreads) {
      IX[p.wtab[i]] = i;
      MS[p.wtab[i]] = p.wsep[i] - 1;
    }
  }
  const int nchunk = (kChunk + ((lmax + 36 + 127) / 128) * 128) / 128;
  for (int c = warp; c < nchunk; c += kThreads / 32) {
    const float4 z = load_z4d(xrow, t0 + c * 128 + lane * 4, p.nt, p.dtype, p.vec_x != 0, mu, inv);
    *reinterpret_cast<float4*>(F0 + c * 128 + lane * 4) = z;
  }
  __syncthreads();
  float* yrow = p.snr + row * p.ld;
  uint16_t* wrow = p.widx + row * p.ld;
  float tmax = ninf();
  const int nfull = lmax / 32;  // chunks of 32 widths without a tail check
#pragma unroll 1
  for (int k = 0; k < kItems0; ++k) {
    const int p0 = (tid + k * kThreads) * 4;
    float S[4] = {0.f, 0.f, 0.f, 0.f}, best[4];
    float acc[4] = {ninf(), ninf(), ninf(), ninf()}, cw[4];  // the coded window maxima (explicit set: unused)
    int q[4] = {0, 0, 0, 0};
#pragma unroll
    for (int r = 0; r < 4; ++r) best[r] = ninf();
#pragma unroll 1
    for (int c = 0; c <= nfull; ++c) {
      const int mbase = c * 32;
      if (mbase >= lmax) break;
      float w[36];
      static_for<0, 9>([&](auto KK) {
        constexpr int kk = decltype(KK)::value;
        const float4 t = *reinterpret_cast<const float4*>(F0 + p0 + mbase + 4 * kk);
        w[4 * kk + 0] = t.x;
        w[4 * kk + 1] = t.y;
        w[4 * kk + 2] = t.z;
        w[4 * kk + 3] = t.w;
      });
      const bool tail = (c == nfull);
      static_for<0, 32>([&](auto MI) {
        constexpr int mi = decltype(MI)::value;
        const int m = mbase + mi + 1;
        if constexpr (GRID) {
          if (!tail || m <= lmax) {
            const int ix = IX[m], ms = MS[m];
            static_for<0, 4>([&](auto R) {
              constexpr int r = decltype(R)::value;
              S[r] += w[r + mi];
            });
            if (ix >= 0) {
              const auto sc = [&] {
                if constexpr (TABLE)
                  return AB[ix];
                else
                  return RS[m];
              }();
              static_for<0, 4>([&](auto R) {
                constexpr int r = decltype(R)::value;
                const float v = snr_of(S[r], sc);
                if (((t0 + p0 + r) & ms) == 0 && v > best[r]) {
                  best[r] = v;
                  q[r] = ix;
                }
              });
            }
          }
        } else {
          // every candidate of the window carries its rank mi in the 5 low
          // mantissa bits (enc_w: the smaller rank wins a tie), the window's
          // maximum is kept running with three-input max instructions and merged
          // with a strict '>' after the window
          if (!tail || m <= lmax) {
            const auto sc = [&] {
              if constexpr (TABLE)
                return AB[m - 1];
              else
                return RS[m];
            }();
            static_for<0, 4>([&](auto R) {
              constexpr int r = decltype(R)::value;
              S[r] += w[r + mi];
              const float e = enc_w<5>(snr_of(S[r], sc), 31 - mi);
              if constexpr ((mi & 1) == 0)
                cw[r] = e;
              else
                acc[r] = fmax3(acc[r], cw[r], e);
            });
          } else {
            static_for<0, 4>([&](auto R) {
              constexpr int r = decltype(R)::value;
              if constexpr ((mi & 1) == 0)
                cw[r] = ninf();
              else
                acc[r] = fmaxf(acc[r], cw[r]);
            });
          }
        }
      });
      if constexpr (!GRID) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {  // a NaN (no candidate) never passes '>'
          const float v = dec_v<5>(acc[r]);
          const bool take = v > best[r];
          best[r] = take ? v : best[r];
          q[r] = take ? mbase + dec_w<5>(acc[r]) : q[r];
          acc[r] = ninf();
        }
      }
    }
    const int64_t s0 = t0 + p0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (s0 + r < p.n_starts) tmax = fmaxf(tmax, best[r]);
    store4(yrow, wrow, s0, p.n_starts, vec, best, q);  // samples to nt feed starts below n_starts
  }
  tile_max_atomic(p.tile_max ? reinterpret_cast<int*>(p.tile_max) + row * p.cand_tiles_per_row : nullptr,
                  t0, tmax);
}

}  // namespace

size_t search_smem_bytes(const spd_plan& plan, bool table) {
  switch (plan.family) {
    case kExhaustive: return sizeof(float) * (size_t)ExLayout(plan.lend, table, plan.explicit_grid).total;
    case kIgrid: return igrid_smem_bytes(plan, table);
    default: return boxdit_smem_bytes(plan, table);
  }
}

cudaError_t launch_search(const spd_plan& plan, const SearchParams& p, cudaStream_t s) {
  if (plan.family == kExhaustive) {
    const size_t smem = search_smem_bytes(plan, p.table != 0);
    const int64_t nblk = plan.desc.ndm * plan.tiles_per_row;
    if (plan.explicit_grid)
      return p.table ? launch_one(exhaustive_kernel<true, true>, smem, nblk, p, s)
                     : launch_one(exhaustive_kernel<false, true>, smem, nblk, p, s);
    return p.table ? launch_one(exhaustive_kernel<true, false>, smem, nblk, p, s)
                   : launch_one(exhaustive_kernel<false, false>, smem, nblk, p, s);
  }
  if (plan.family == kBoxdit) return launch_boxdit(plan, p, s);
  return launch_igrid(plan, p, s);
}

}  // namespace spd
