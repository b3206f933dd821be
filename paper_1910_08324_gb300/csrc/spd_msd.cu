// spd_msd.cu -- noise statistics of the rows for table-noise searches (sm_103a).
//
// Sec. 4.5 ("calculation of mean and standard deviation"): the mean and the
// standard deviation of the base-level noise, estimated with point-wise outlier
// rejection repeated until convergence, computed only for the series decimated
// in time by powers of two and interpolated to the widths in between.
//
// Level k of a row is the series of sums of its complete blocks of 2^k samples,
// k = 0..nlev-1 (nlev covers the plan's widest boxcar).  Every pass streams the
// row once and updates all levels together:
//   * one CTA per row, 2048-sample chunks, 8 samples per thread; levels 0..3 in
//     registers, 4..8 by warp shuffles, 9..11 from the warps' level-8 sums,
//     12.. accumulated over chunks;
//   * a value of level k is kept when |v - mu_k| <= thr sigma_k of the previous
//     pass (the first pass keeps every value);
//   * each thread sums the kept values shifted by the previous mean (w = v - c_k,
//     so the sums stay small: a numerically stable form, Chan et al.), w and w^2,
//     per chunk in registers and across chunks with compensated (Kahan) adds;
//   * at the end, an FP64 reduction over the CTA gives n, mean and deviation
//     (population form); a level is converged when a pass keeps as many values
//     as the one before.
// Passes are separate launches; a row whose levels have all converged returns
// at once.  The table kernel then interpolates every width of the plan: the
// per-sample mean mu_k / 2^k and the white-normalised deviation sigma_k / 2^(k/2)
// are interpolated linearly in log2(L) (white noise therefore keeps Eq.
// whitenoise exactly; a power-of-two width gets its level's values).
#include <cfloat>

#include "spd_common.cuh"

namespace spd {
namespace {

constexpr int kC = kChunk;

struct MsdLevel {  // per row and level, in the workspace
  double mu, sd;
  long long n;
  int conv;  // 1: the last pass kept as many values as the one before (or no rejection)
  int pad;
};
static_assert(sizeof(MsdLevel) == 32, "MsdLevel layout");

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

__global__ void __launch_bounds__(kThreads, 3) msd_pass_kernel(const MsdParams p, int pass) {
  __shared__ float cshift[kMsdMaxLevels], clim[kMsdMaxLevels];
  __shared__ float s8[2][kThreads / 32];
  __shared__ double red[kThreads / 32][kMsdMaxLevels][2];
  __shared__ long long redn[kThreads / 32][kMsdMaxLevels];
  __shared__ int done;
  __shared__ float blk[kMsdMaxLevels];  // partial blocks of levels >= 12 (one thread)
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t row = blockIdx.x;
  const int nlev = p.nlev;
  MsdLevel* st = reinterpret_cast<MsdLevel*>(p.state) + row * kMsdMaxLevels;
  const unsigned char* __restrict__ xrow = static_cast<const unsigned char*>(p.x) + row * p.ld * p.esize;
  const int64_t nt = p.nt;
  const bool vx = p.vec_x != 0;

  if (pass > 0) {
    if (t == 0) {
      int all = 1;
      for (int k = 0; k < nlev; ++k) all &= st[k].conv;
      done = all;
    }
    __syncthreads();
    if (done) return;
    if (t < nlev) {
      cshift[t] = (float)st[t].mu;
      clim[t] = (float)(p.thr * st[t].sd);
    }
  } else {
    // pilot shift: the mean of the row's first chunk, times 2^k
    const int n0 = nt < kC ? (int)nt : kC;
    float v0, v1;
    {
      float4 a, b;
      cvt8(load_raw8(xrow, 8 * t, n0, p.dtype, vx), 8 * t, n0, p.dtype, 0.0f, 1.0f, a, b);
      float f[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      v0 = 0.0f;
#pragma unroll
      for (int i = 0; i < 8; ++i) v0 += (8 * t + i < n0) ? f[i] : 0.0f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v0 += __shfl_xor_sync(kFull, v0, o);
    if (lane == 0) s8[0][warp] = v0;
    __syncthreads();
    v1 = 0.0f;
    for (int w = 0; w < kThreads / 32; ++w) v1 += s8[0][w];
    const float c0 = v1 / (float)n0;
    if (t < nlev) {
      cshift[t] = c0 * (float)(1 << t);
      clim[t] = FLT_MAX;
    }
  }
  __syncthreads();

  float sw[kMsdMaxLevels], sw2[kMsdMaxLevels], cw[4], cw2[4];  // compensation: levels 0..3
  int cn[kMsdMaxLevels];
#pragma unroll
  for (int k = 0; k < kMsdMaxLevels; ++k) sw[k] = sw2[k] = 0.0f, cn[k] = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) cw[k] = cw2[k] = 0.0f;
  // levels 0..3 (several values per thread and chunk): chunk-local sums, folded
  // into the compensated sums once per chunk; levels >= 4: one value per chunk
  float pw[4] = {0.0f, 0.0f, 0.0f, 0.0f}, pw2[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  auto keep = [&](auto K, float v, bool valid) {
    constexpr int k = decltype(K)::value;
    const float w = v - cshift[k];
    const bool in = valid && fabsf(w) <= clim[k];
    if constexpr (k < 4) {
      pw[k] += in ? w : 0.0f;
      pw2[k] += in ? w * w : 0.0f;
    } else {  // at most one value per chunk: plain sums (<= 512 adds per row and lane)
      sw[k] += in ? w : 0.0f;
      sw2[k] += in ? w * w : 0.0f;
    }
    cn[k] += in ? 1 : 0;
  };
  if (t < kMsdMaxLevels) blk[t] = 0.0f;
  __syncthreads();

  const int64_t nch = (nt + kC - 1) / kC;
  auto chunk_n = [&](int64_t c) {  // samples of chunk c that exist
    const int64_t left = nt - c * kC;
    return left < kC ? (int)left : kC;
  };
  Raw8 nx = load_raw8(xrow, 8 * t, chunk_n(0), p.dtype, vx);  // one chunk ahead
  for (int64_t c = 0; c < nch; ++c) {
#pragma unroll
    for (int k = 0; k < 4; ++k) pw[k] = pw2[k] = 0.0f;
    const int64_t base = c * kC + 8 * t;  // first sample of this thread
    float f[8];
    {
      const Raw8 cx = nx;
      if (c + 1 < nch) nx = load_raw8(xrow + (c + 1) * kC * p.esize, 8 * t, chunk_n(c + 1), p.dtype, vx);
      const int nrel = chunk_n(c);
      float4 a, b;
      cvt8(cx, 8 * t, nrel, p.dtype, 0.0f, 1.0f, a, b);
      f[0] = a.x, f[1] = a.y, f[2] = a.z, f[3] = a.w, f[4] = b.x, f[5] = b.y, f[6] = b.z, f[7] = b.w;
#pragma unroll
      for (int i = 0; i < 8; ++i) f[i] = (base + i < nt) ? f[i] : 0.0f;  // sums stay finite
    }
    // levels 0..3 from this thread's samples; a block counts when it ends by nt
    static_for<0, 8>([&](auto I) {
      constexpr int i = decltype(I)::value;
      keep(std::integral_constant<int, 0>{}, f[i], base + i + 1 <= nt);
    });
    float p1[4], p2[2];
    static_for<0, 4>([&](auto I) {
      constexpr int i = decltype(I)::value;
      p1[i] = f[2 * i] + f[2 * i + 1];
      if (nlev > 1) keep(std::integral_constant<int, 1>{}, p1[i], base + 2 * i + 2 <= nt);
    });
    static_for<0, 2>([&](auto I) {
      constexpr int i = decltype(I)::value;
      p2[i] = p1[2 * i] + p1[2 * i + 1];
      if (nlev > 2) keep(std::integral_constant<int, 2>{}, p2[i], base + 4 * i + 4 <= nt);
    });
    float s = p2[0] + p2[1];
    if (nlev > 3) keep(std::integral_constant<int, 3>{}, s, base + 8 <= nt);
    // levels 4..8: lanes of a block share its sum; its first lane keeps it
    static_for<4, 9>([&](auto K) {
      constexpr int k = decltype(K)::value;
      s += __shfl_xor_sync(kFull, s, 1 << (k - 4));
      if (nlev > k && (lane & ((1 << (k - 3)) - 1)) == 0) keep(K, s, base + (1 << k) <= nt);
    });
    // levels 9..11 from the warps' level-8 sums (lanes 0..3, 4..5 and 6 of warp 0)
    if (lane == 0) s8[c & 1][warp] = s;
    __syncthreads();
    if (warp == 0 && lane < 7 && nlev > 9) {
      const int lj = lane < 4 ? 9 : (lane < 6 ? 10 : 11);
      const int lb = lane < 4 ? lane : (lane < 6 ? lane - 4 : 0);
      const int nw = 1 << (lj - 8);
      float v = 0.0f;
      for (int i = 0; i < nw; ++i) v += s8[c & 1][lb * nw + i];
      const bool valid = c * kC + (int64_t)(lb + 1) * (1 << lj) <= nt;
      if (lj == 9) keep(std::integral_constant<int, 9>{}, v, valid);
      else if (lj == 10) {
        if (nlev > 10) keep(std::integral_constant<int, 10>{}, v, valid);
      } else {
        if (nlev > 11) keep(std::integral_constant<int, 11>{}, v, valid);
        // levels >= 12: blocks of 2^(k-11) chunks
        static_for<12, kMsdMaxLevels>([&](auto K) {
          constexpr int k = decltype(K)::value;
          if (nlev > k) {
            blk[k] += v;
            if (((c + 1) & ((1 << (k - 11)) - 1)) == 0) {
              keep(K, blk[k], (c + 1) * kC <= nt);
              blk[k] = 0.0f;
            }
          }
        });
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      kahan_add(sw[k], cw[k], pw[k]);
      kahan_add(sw2[k], cw2[k], pw2[k]);
    }
  }

  // FP64 reduction over the CTA, then the new statistics of every level
#pragma unroll
  for (int k = 0; k < kMsdMaxLevels; ++k) {
    double a = sw[k], b = sw2[k];
    if (k < 4) a -= (double)cw[k < 4 ? k : 0], b -= (double)cw2[k < 4 ? k : 0];
    long long n = cn[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(kFull, a, o);
      b += __shfl_xor_sync(kFull, b, o);
      n += __shfl_xor_sync(kFull, n, o);
    }
    if (lane == 0) {
      red[warp][k][0] = a;
      red[warp][k][1] = b;
      redn[warp][k] = n;
    }
  }
  __syncthreads();
  if (t < nlev) {
    double a = 0.0, b = 0.0;
    long long n = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
      a += red[w][t][0];
      b += red[w][t][1];
      n += redn[w][t];
    }
    MsdLevel L = st[t];
    if (pass > 0 && L.conv) return;  // this level has stopped; keep its statistics
    const double m1 = n > 0 ? a / (double)n : 0.0;
    const double var = n > 0 ? b / (double)n - m1 * m1 : 0.0;
    const long long prev = L.n;
    L.mu = n > 0 ? (double)cshift[t] + m1 : 0.0;
    L.sd = sqrt(var > 0.0 ? var : 0.0);
    L.n = n;
    L.conv = (!(p.thr > 0.0f) || (pass > 0 && n == prev)) ? 1 : 0;
    st[t] = L;
  }
}

// mu_L, sigma_L of every width of the plan from the level statistics.
__global__ void __launch_bounds__(kThreads) msd_table_kernel(const MsdParams p) {
  const int64_t row = blockIdx.x;
  const MsdLevel* st = reinterpret_cast<const MsdLevel*>(p.state) + row * kMsdMaxLevels;
  int h = -1;
  while (h + 1 < p.nlev && st[h + 1].n >= 2) ++h;
  for (int w = threadIdx.x; w < p.n_widths; w += kThreads) {
    const int L = p.unit_widths ? w + 1 : p.wtab[w];
    double m = 0.0, r = 0.0;
    if (h >= 0) {
      const double lg = log2((double)L);
      const int a = (int)floor(lg);
      if (a >= h) {
        m = st[h].mu / ldexp(1.0, h);
        r = st[h].sd / sqrt(ldexp(1.0, h));
      } else {
        const double fr = lg - (double)a;
        const double ma = st[a].mu / ldexp(1.0, a), mb = st[a + 1].mu / ldexp(1.0, a + 1);
        const double ra = st[a].sd / sqrt(ldexp(1.0, a)), rb = st[a + 1].sd / sqrt(ldexp(1.0, a + 1));
        m = ma + fr * (mb - ma);
        r = ra + fr * (rb - ra);
      }
    }
    p.out_mu[row * p.n_widths + w] = (float)((double)L * m);
    p.out_sigma[row * p.n_widths + w] = (float)(sqrt((double)L) * r);
  }
}

__global__ void msd_reset_kernel(const MsdParams p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < p.ndm * kMsdMaxLevels) {
    MsdLevel L;
    L.mu = 0.0, L.sd = 0.0, L.n = -1, L.conv = 0, L.pad = 0;
    reinterpret_cast<MsdLevel*>(p.state)[i] = L;
  }
}

}  // namespace

size_t msd_state_bytes(int64_t ndm) { return (size_t)ndm * kMsdMaxLevels * sizeof(MsdLevel); }

cudaError_t launch_msd(const spd_plan& plan, const MsdParams& p, int max_passes, cudaStream_t s) {
  const int64_t n = plan.desc.ndm * kMsdMaxLevels;
  msd_reset_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  for (int pass = 0; pass < max_passes && e == cudaSuccess; ++pass) {
    msd_pass_kernel<<<(unsigned)plan.desc.ndm, kThreads, 0, s>>>(p, pass);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  msd_table_kernel<<<(unsigned)plan.desc.ndm, kThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace spd
