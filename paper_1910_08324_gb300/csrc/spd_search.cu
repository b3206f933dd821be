// spd_search.cu -- the boxcar search kernels (sm_103a).
//
// What is computed (Eq. boxcar, Eq. SNRlong with Eq. whitenoise, Eq. MSD03):
// for every row and start s, the largest SNR over the plan's eligible widths
// and the index of the smallest width reaching it.  Each sample is normalised
// once on load, z = (x - mu_r) / sigma_r, so a width-L boxcar's SNR is
// (sum of L z-values) / sqrt(L).
//
// GB300 structure (one CTA per (row, tile of T starts), 256 threads):
//   * the grid is split into levels (see spd_internal.h): level j has unit
//     2^j, evaluates starts that are multiples of 2^j, and sums block series
//     of 2^j-sample blocks held in shared memory;
//   * coarse levels (unit >= 8 for IGRID, >= K for BoxDIT K) are built once per
//     tile from a single pass over [t0, t0 + T + halo) (float4 loads, warp
//     shuffle reductions) and evaluated for the whole tile;
//   * fine levels are rebuilt per 2048-start sub-chunk from a second pass over
//     the sub-chunk (an L2 hit: the tile pass read it moments before), so the
//     shared-memory footprint stays small;
//   * every candidate is a running-sum add, one multiply by a compile-time
//     indexed constant and a compare/select; block counts are compile-time, the
//     loops fully unrolled; nothing intermediate reaches HBM;
//   * per-start maxima of the levels merge in shared memory (strict '>' in
//     increasing width order keeps the smallest width on ties) and leave the
//     CTA as one coalesced float4 / 4 x uint16 store per thread;
//   * the tile's largest SNR goes to the workspace for the candidate step.
// Samples past the end of a row load as -inf, so a boxcar that would need
// them sums to -inf and can never be the maximum: that is the rule s + L <= nt.
#include "spd_common.cuh"

namespace spd {
namespace {

constexpr int kItems0 = kChunk / 4 / kThreads;  // level-0 items (4 starts) per thread per sub-chunk
static_assert(kItems0 * 4 * kThreads == kChunk, "sub-chunk must split evenly");

// Evaluate 4 consecutive positions p0..p0+3 (p0 % 4 == 0) of one level whose
// block series `blk` is in shared memory (see eval_window).
template <int MMAX, class Pred, bool PARTIAL, bool HAS_BASE, class Scale>
__device__ __forceinline__ void eval4(const float* __restrict__ blk, int p0, int n_used,
                                      Scale&& scale, const float (&base)[4], float (&bv)[4],
                                      int (&bq)[4], float (&full)[4]) {
  constexpr int NW = (MMAX + 6) / 4;
  float w[NW * 4];
  load_window4<NW>(blk + p0, w);
  eval_window<4, MMAX, Pred, PARTIAL, HAS_BASE>(w, n_used, scale, base, bv, bq, full);
}

__device__ __forceinline__ void rmw(float* by, uint16_t* bw, int idx, float y, int w) {
  if (y > by[idx]) {
    by[idx] = y;
    bw[idx] = (uint16_t)w;
  }
}

// ============================================================================ BoxDIT
template <int K>
struct BdLayout {
  static constexpr int KAP = (K == 8) ? 3 : (K == 16) ? 4 : 5;
  static constexpr int E = ((K * (K - 1)) + 127) / 128 * 128;  // fine halo: c_kappa
  int lvl[kMaxLevels], bas[kMaxLevels];
  int sk, bc_y, bc_w, f[KAP], fb[KAP], be_y, be_w, red, total;
  __host__ __device__ BdLayout(int T, int H, int top) {
    int o = 0;
    for (int j = 0; j < kMaxLevels; ++j) lvl[j] = bas[j] = 0;
    sk = bc_y = bc_w = 0;
    if (top >= KAP) {
      sk = o;
      o += al4((T + H) / K + 1 + 40);
      lvl[KAP] = sk + K;  // blk_kappa[n] = A_kappa[n + K - 1], A stored at sk + 1
      for (int j = KAP + 1; j <= top; ++j) {
        lvl[j] = o;
        o += al4(((T + H) >> j) + K + 40);
      }
      for (int j = KAP; j <= top; ++j) {
        bas[j] = o;
        o += al4((T >> j) + 4);
      }
      bc_y = o;
      o += al4(T / K);
      bc_w = o;
      o += al4((T / K + 1) / 2);
    }
    for (int i = 0; i < KAP; ++i) {
      f[i] = o;
      o += al4(((kChunk + E) >> i) + K + 8);
    }
    fb[0] = 0;
    for (int i = 1; i < KAP; ++i) {
      fb[i] = o;
      o += al4((kChunk >> i) + 4);
    }
    be_y = o;
    o += kChunk / 2;
    be_w = o;
    o += kChunk / 4;
    red = o;
    o += 32;
    total = o;
  }
};

template <int K>
__global__ void __launch_bounds__(kThreads, 2) boxdit_kernel(const SearchParams p) {
  using LY = BdLayout<K>;
  constexpr int KAP = LY::KAP;
  constexpr int E = LY::E;
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t row = blockIdx.x / p.tiles_per_row;
  const int64_t tile = blockIdx.x % p.tiles_per_row;
  const int T = p.tile, H = p.halo, top = p.top;
  const int64_t t0 = tile * (int64_t)T;
  const float* __restrict__ xrow = p.x + row * p.ld;
  const float mu = p.mu[row];
  const float inv = 1.0f / p.sigma[row];
  const bool vec = p.vec != 0;
  const LY L(T, H, top);
  const float zero4[4] = {0.f, 0.f, 0.f, 0.f};

  // ---- coarse iterations kappa..top ---------------------------------------
  float* BCY = smem + L.bc_y;
  uint16_t* BCW = reinterpret_cast<uint16_t*>(smem + L.bc_w);
  if (top >= KAP) {
    float* SK = smem + L.sk;  // SK[q + 1] = aligned K-sum q of the tile pass
    const int nchunk = (T + H) / 128;
    for (int c = warp; c < nchunk; c += kThreads / 32) {
      const float4 z = load_z4(xrow, t0 + c * 128 + lane * 4, p.nt, vec, mu, inv);
      float s = (z.x + z.y) + (z.z + z.w);
      s += __shfl_xor_sync(kFull, s, 1);
      if (K >= 16) s += __shfl_xor_sync(kFull, s, 2);
      if (K >= 32) s += __shfl_xor_sync(kFull, s, 4);
      constexpr int LPK = K / 4;  // lanes per K-block
      if ((lane % LPK) == 0) SK[1 + c * (128 / K) + lane / LPK] = s;
    }
    __syncthreads();
    // base of iteration kappa: X_{c_kappa}[t0 + nK] = sum of K-1 K-blocks
    {
      float* B = smem + L.bas[KAP];
      const int P = T >> KAP;
      for (int n = tid; n < P; n += kThreads) {
        float b = 0.f;
        for (int t = 0; t < K - 1; ++t) b += SK[1 + n + t];
        B[n] = b;
      }
    }
    // shifted decimation (Sec. 3.1): blk_j[n] = blk_{j-1}[2n + K] + blk_{j-1}[2n + K + 1]
    {
      int valid = (T + H) / K - (K - 1);
      for (int j = KAP + 1; j <= top; ++j) {
        const int nv = (valid - K) / 2;
        float* dst = smem + L.lvl[j];
        const float* src = smem + L.lvl[j - 1];
        for (int i = tid; i < nv; i += kThreads) dst[i] = src[2 * i + K] + src[2 * i + K + 1];
        valid = nv;
        __syncthreads();
      }
    }
    __syncthreads();
    for (int j = KAP; j <= top; ++j) {
      const float* blk = smem + L.lvl[j];
      const float* B = smem + L.bas[j];
      float* Bn = (j < top) ? smem + L.bas[j + 1] : nullptr;
      const int P = T >> j;
      const int items = (P + 3) >> 2;
      const int first = p.lvl_first[j];
      auto scl = [&](auto M) { return p.bscale[j][decltype(M)::value]; };
      for (int it = tid; it < items; it += kThreads) {
        const int p0 = it * 4;
        const float4 b4 = *reinterpret_cast<const float4*>(B + p0);
        const float base[4] = {b4.x, b4.y, b4.z, b4.w};
        float bv[4], full[4];
        int bq[4];
        if (j == top)
          eval4<K, AllM, true, true>(blk, p0, p.n_top, scl, base, bv, bq, full);
        else
          eval4<K, AllM, false, true>(blk, p0, p.n_top, scl, base, bv, bq, full);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int pp = p0 + r;
          if (pp < P) {
            const int idx = pp << (j - KAP);
            if (j == KAP) {
              BCY[idx] = bv[r];
              BCW[idx] = (uint16_t)(first + bq[r]);
            } else {
              rmw(BCY, BCW, idx, bv[r], first + bq[r]);
            }
            if (Bn && !(pp & 1)) Bn[pp >> 1] = full[r];
          }
        }
      }
      __syncthreads();
    }
  }

  // ---- fine iterations 0..kappa-1, one sub-chunk at a time -----------------
  float* BEY = smem + L.be_y;
  uint16_t* BEW = reinterpret_cast<uint16_t*>(smem + L.be_w);
  float* yrow = p.snr + row * p.ld;
  uint16_t* wrow = p.widx + row * p.ld;
  const int ftop = top < KAP - 1 ? top : KAP - 1;  // last fine iteration
  float tmax = ninf();
  const int nsub = T / kChunk;
  for (int sub = 0; sub < nsub; ++sub) {
    const int64_t sc = t0 + (int64_t)sub * kChunk;
    if (sc >= p.nt) break;
    // A_i of the sub-chunk, stored shifted by c_i / 2^i = K - K/2^i (Sec. 3.1 shifted decimation)
    for (int c = warp; c < (kChunk + E) / 128; c += kThreads / 32) {
      const int o = c * 128 + lane * 4;
      const float4 z = load_z4(xrow, sc + o, p.nt, vec, mu, inv);
      *reinterpret_cast<float4*>(smem + L.f[0] + o) = z;
      const float a = z.x + z.y, b = z.z + z.w;
      {
        const int n = (o >> 1) - K / 2;
        if (n >= 0) *reinterpret_cast<float2*>(smem + L.f[1] + n) = make_float2(a, b);
      }
      float s = a + b;
      {
        const int n = (o >> 2) - (K - K / 4);
        if (n >= 0) smem[L.f[2] + n] = s;
      }
      if (KAP >= 4) {
        s += __shfl_xor_sync(kFull, s, 1);
        const int n = (o >> 3) - (K - K / 8);
        if (!(lane & 1) && n >= 0) smem[L.f[KAP >= 4 ? 3 : 0] + n] = s;
      }
      if (KAP >= 5) {
        s += __shfl_xor_sync(kFull, s, 2);
        const int n = (o >> 4) - (K - K / 16);
        if (!(lane & 3) && n >= 0) smem[L.f[KAP >= 5 ? 4 : 0] + n] = s;
      }
    }
    __syncthreads();
    float y0[kItems0][4];
    int w0[kItems0][4];
    {
      auto scl = [&](auto M) { return p.bscale[0][decltype(M)::value]; };
#pragma unroll
      for (int k = 0; k < kItems0; ++k) {
        const int p0 = (tid + k * kThreads) * 4;
        float full[4];
        if (top == 0)
          eval4<K, AllM, true, false>(smem + L.f[0], p0, p.n_top, scl, zero4, y0[k], w0[k], full);
        else
          eval4<K, AllM, false, false>(smem + L.f[0], p0, p.n_top, scl, zero4, y0[k], w0[k], full);
        if (ftop >= 1) {
          float* Bn = smem + L.fb[1];
          *reinterpret_cast<float2*>(Bn + (p0 >> 1)) = make_float2(full[0], full[2]);
        }
      }
    }
    __syncthreads();
    static_for<1, KAP>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if (i <= ftop) {
        const float* blk = smem + L.f[i];
        const float* B = smem + L.fb[i];
        float* Bn = (i < ftop) ? smem + L.fb[i < KAP - 1 ? i + 1 : i] : nullptr;
        const int first = p.lvl_first[i];
        auto scl = [&](auto M) { return p.bscale[i][decltype(M)::value]; };
        for (int it = tid; it < (kChunk >> i) / 4; it += kThreads) {
          const int p0 = it * 4;
          const float4 b4 = *reinterpret_cast<const float4*>(B + p0);
          const float base[4] = {b4.x, b4.y, b4.z, b4.w};
          float bv[4], full[4];
          int bq[4];
          if (i == top)
            eval4<K, AllM, true, true>(blk, p0, p.n_top, scl, base, bv, bq, full);
          else
            eval4<K, AllM, false, true>(blk, p0, p.n_top, scl, base, bv, bq, full);
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int idx = (p0 + r) << (i - 1);
            if (i == 1) {
              BEY[idx] = bv[r];
              BEW[idx] = (uint16_t)(first + bq[r]);
            } else {
              rmw(BEY, BEW, idx, bv[r], first + bq[r]);
            }
          }
          if (Bn) *reinterpret_cast<float2*>(Bn + (p0 >> 1)) = make_float2(full[0], full[2]);
        }
        __syncthreads();
      }
    });
    if (top >= KAP) {  // coarse results at starts = 0 mod K
      const int cbase = (int)((sc - t0) / K);
      for (int n = tid; n < kChunk / K; n += kThreads) rmw(BEY, BEW, n * (K / 2), BCY[cbase + n], BCW[cbase + n]);
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kItems0; ++k) {
      const int p0 = (tid + k * kThreads) * 4;
      if (top >= 1) {
#pragma unroll
        for (int r = 0; r < 4; r += 2) {
          const int idx = (p0 + r) >> 1;
          if (BEY[idx] > y0[k][r]) {
            y0[k][r] = BEY[idx];
            w0[k][r] = BEW[idx];
          }
        }
      }
      const int64_t s0 = sc + p0;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (s0 + r < p.nt) tmax = fmaxf(tmax, y0[k][r]);
      store4(yrow, wrow, s0, p.nt, vec, y0[k], w0[k]);
    }
    tile_max_atomic(p, row, sc, tmax);
    tmax = ninf();
    __syncthreads();
  }
}

// ============================================================================ exhaustive
struct ExLayout {
  int f0, rs, red, total;
  __host__ __device__ explicit ExLayout(int lmax) {
    int o = 0;
    f0 = o;
    o += al4(kChunk + ((lmax + 36 + 127) / 128) * 128 + 8);
    rs = o;
    o += al4(lmax + 33);
    red = o;
    o += 32;
    total = o;
  }
};

__global__ void __launch_bounds__(kThreads, 2) exhaustive_kernel(const SearchParams p) {
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t row = blockIdx.x / p.tiles_per_row;
  const int64_t tile = blockIdx.x % p.tiles_per_row;
  const int64_t t0 = tile * (int64_t)kChunk;
  const int lmax = p.lmax;
  const float* __restrict__ xrow = p.x + row * p.ld;
  const float mu = p.mu[row];
  const float inv = 1.0f / p.sigma[row];
  const bool vec = p.vec != 0;
  const ExLayout L(lmax);
  float* F0 = smem + L.f0;
  float* RS = smem + L.rs;
  for (int m = tid; m <= lmax + 32; m += kThreads)
    RS[m] = (m >= 1 && m <= lmax) ? (float)(1.0 / sqrt((double)m)) : 0.0f;
  const int nchunk = (kChunk + ((lmax + 36 + 127) / 128) * 128) / 128;
  for (int c = warp; c < nchunk; c += kThreads / 32) {
    const float4 z = load_z4(xrow, t0 + c * 128 + lane * 4, p.nt, vec, mu, inv);
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
        if (!tail || m <= lmax) {
          const float sc = RS[m];
          static_for<0, 4>([&](auto R) {
            constexpr int r = decltype(R)::value;
            S[r] += w[r + mi];
            const float v = S[r] * sc;
            if (v > best[r]) {
              best[r] = v;
              q[r] = m - 1;
            }
          });
        }
      });
    }
    const int64_t s0 = t0 + p0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (s0 + r < p.nt) tmax = fmaxf(tmax, best[r]);
    store4(yrow, wrow, s0, p.nt, vec, best, q);
  }
  tile_max_atomic(p, row, t0, tmax);
}

}  // namespace

size_t search_smem_bytes(const spd_plan& plan) {
  switch (plan.family) {
    case kExhaustive: return sizeof(float) * (size_t)ExLayout(plan.lend).total;
    case kIgrid: return igrid_smem_bytes(plan);
    default:
      switch (plan.k) {
        case 8: return sizeof(float) * (size_t)BdLayout<8>(plan.tile, plan.halo, plan.top).total;
        case 16: return sizeof(float) * (size_t)BdLayout<16>(plan.tile, plan.halo, plan.top).total;
        default: return sizeof(float) * (size_t)BdLayout<32>(plan.tile, plan.halo, plan.top).total;
      }
  }
}

cudaError_t launch_search(const spd_plan& plan, const SearchParams& p, cudaStream_t s) {
  const size_t smem = search_smem_bytes(plan);
  const int64_t nblk = plan.desc.ndm * plan.tiles_per_row;
  if (plan.family == kExhaustive) return launch_one(exhaustive_kernel, smem, nblk, p, s);
  if (plan.family == kBoxdit) {
    switch (plan.k) {
      case 8: return launch_one(boxdit_kernel<8>, smem, nblk, p, s);
      case 16: return launch_one(boxdit_kernel<16>, smem, nblk, p, s);
      case 32: return launch_one(boxdit_kernel<32>, smem, nblk, p, s);
      default: return cudaErrorInvalidValue;
    }
  }
  return launch_igrid(plan, p, s);
}

}  // namespace spd
