// spd_common.cuh -- device helpers shared by the search kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "spd_internal.h"

namespace spd {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float ninf() { return __int_as_float(0xff800000u); }

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

__host__ __device__ constexpr int al4(int v) { return (v + 3) & ~3; }
__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ constexpr int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// SNR of a boxcar sum S of normalised samples.  White noise: S times the
// width's 1/sqrt(L).  Table noise: the width's affine map a S + b (row_noise).
__device__ __forceinline__ float snr_of(float S, float sc) { return S * sc; }
__device__ __forceinline__ float snr_of(float S, float2 ab) { return fmaf(S, ab.x, ab.y); }

// Per-row noise constants of a search CTA (Eq. SNRlong).
//   White noise (Eq. whitenoise): samples are normalised as z = (x - mu_r) / sigma_r
//   and a width-L sum Z of z-values has SNR Z / sqrt(L).
//   Table noise (mu_L, sigma_L per row and width index; index 0 is width 1 in
//   every grid): samples are centred and scaled by the width-1 entry,
//   z = (x - mu_1) / sigma_1, so that (X_L - mu_L) / sigma_L = a_L Z + b_L with
//   a_L = sigma_1 / sigma_L and b_L = (L mu_1 - mu_L) / sigma_L, computed in
//   FP64 and stored as AB[w] = (a, b) in shared memory (caller synchronises).
//   AB holds kAbPad zero entries past the last width: the masked block counts
//   of a partial last level (ranks >= n_top) still load their entry.
constexpr int kAbPad = 32;
template <bool TABLE>
__device__ __forceinline__ void row_noise(const SearchParams& p, int64_t row, float2* AB, float& mu,
                                          float& inv) {
  if constexpr (!TABLE) {
    mu = p.mu[row];
    inv = 1.0f / p.sigma[row];
  } else {
    const float* m = p.mu + row * p.n_widths;
    const float* s = p.sigma + row * p.n_widths;
    const double c = m[0], d = s[0];
    mu = m[0];
    inv = (float)(1.0 / d);
    for (int w = threadIdx.x; w < p.n_widths + kAbPad; w += blockDim.x) {
      if (w < p.n_widths) {
        const double L = p.unit_widths ? (double)(w + 1) : (double)p.wtab[w];
        const double sg = s[w];
        AB[w] = make_float2((float)(d / sg), (float)((L * c - (double)m[w]) / sg));
      } else {
        AB[w] = make_float2(0.0f, 0.0f);
      }
    }
  }
}

// Order-preserving int key of a float (signed compare): used for atomic maxima.
__device__ __forceinline__ int fkey(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7fffffff;
}
__host__ __device__ __forceinline__ float fkey_inv(int k) {
#ifdef __CUDA_ARCH__
  return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff);
#else
  union {
    int i;
    float f;
  } u;
  u.i = k >= 0 ? k : k ^ 0x7fffffff;
  return u.f;
#endif
}

// Warp-reduced maximum of v folded into the candidate-tile maximum of start s.
__device__ __forceinline__ void tile_max_atomic(const SearchParams& p, int64_t row, int64_t s,
                                                float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  if ((threadIdx.x & 31) == 0 && p.tile_max)
    atomicMax(reinterpret_cast<int*>(p.tile_max) + row * p.cand_tiles_per_row + s / kCandTile, fkey(v));
}

// z-values of samples [pos, pos + 4) of one row; -inf at and past nt.
__device__ __forceinline__ float4 load_z4(const float* __restrict__ row, int64_t pos, int64_t nt,
                                          bool vec, float mu, float inv) {
  float4 v;
  if (vec && pos + 4 <= nt) {
    v = __ldg(reinterpret_cast<const float4*>(row + pos));
    v.x = (v.x - mu) * inv;
    v.y = (v.y - mu) * inv;
    v.z = (v.z - mu) * inv;
    v.w = (v.w - mu) * inv;
  } else {
    v.x = (pos + 0 < nt) ? (__ldg(row + pos + 0) - mu) * inv : ninf();
    v.y = (pos + 1 < nt) ? (__ldg(row + pos + 1) - mu) * inv : ninf();
    v.z = (pos + 2 < nt) ? (__ldg(row + pos + 2) - mu) * inv : ninf();
    v.w = (pos + 3 < nt) ? (__ldg(row + pos + 3) - mu) * inv : ninf();
  }
  return v;
}

// Raw samples [pos, pos + 4) (no normalisation); -inf marks positions past nt.
__device__ __forceinline__ float4 load_x4(const float* __restrict__ row, int64_t pos, int64_t nt,
                                          bool vec) {
  float4 v;
  if (vec && pos + 4 <= nt) {
    v = __ldg(reinterpret_cast<const float4*>(row + pos));
  } else {
    v.x = (pos + 0 < nt) ? __ldg(row + pos + 0) : ninf();
    v.y = (pos + 1 < nt) ? __ldg(row + pos + 1) : ninf();
    v.z = (pos + 2 < nt) ? __ldg(row + pos + 2) : ninf();
    v.w = (pos + 3 < nt) ? __ldg(row + pos + 3) : ninf();
  }
  return v;
}

__device__ __forceinline__ float4 norm4(float4 v, float mu, float inv) {
  // -inf stays -inf: (-inf - mu) * inv with inv > 0
  v.x = (v.x - mu) * inv;
  v.y = (v.y - mu) * inv;
  v.z = (v.z - mu) * inv;
  v.w = (v.w - mu) * inv;
  return v;
}

__device__ __forceinline__ void store4(float* __restrict__ yrow, uint16_t* __restrict__ wrow,
                                       int64_t s0, int64_t nt, bool vec, const float (&y)[4],
                                       const int (&w)[4]) {
  if (vec && s0 + 4 <= nt) {
    __stcs(reinterpret_cast<float4*>(yrow + s0), make_float4(y[0], y[1], y[2], y[3]));
    uint2 pk;
    pk.x = (uint32_t)(w[0] & 0xffff) | ((uint32_t)w[1] << 16);
    pk.y = (uint32_t)(w[2] & 0xffff) | ((uint32_t)w[3] << 16);
    __stcs(reinterpret_cast<uint2*>(wrow + s0), pk);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (s0 + k < nt) {
        yrow[s0 + k] = y[k];
        wrow[s0 + k] = (uint16_t)w[k];
      }
  }
}

// vec: x/Y bases 16-byte aligned, W base 8-byte aligned, ld % 4 == 0 (so Y rows
// are 16-byte and W rows 8-byte aligned); s0 % 8 == 0.
__device__ __forceinline__ void store8(float* __restrict__ yrow, uint16_t* __restrict__ wrow,
                                       int64_t s0, int64_t nt, bool vec, const float (&y)[8],
                                       const int (&w)[8]) {
  if (vec && s0 + 8 <= nt) {
    __stcs(reinterpret_cast<float4*>(yrow + s0), make_float4(y[0], y[1], y[2], y[3]));
    __stcs(reinterpret_cast<float4*>(yrow + s0 + 4), make_float4(y[4], y[5], y[6], y[7]));
    uint4 pk;
    pk.x = (uint32_t)(w[0] & 0xffff) | ((uint32_t)w[1] << 16);
    pk.y = (uint32_t)(w[2] & 0xffff) | ((uint32_t)w[3] << 16);
    pk.z = (uint32_t)(w[4] & 0xffff) | ((uint32_t)w[5] << 16);
    pk.w = (uint32_t)(w[6] & 0xffff) | ((uint32_t)w[7] << 16);
    // a row of W starts at 2 * row * ld bytes: only 8-byte aligned when ld % 8 == 4
    if ((reinterpret_cast<uintptr_t>(wrow + s0) & 15) == 0) {
      __stcs(reinterpret_cast<uint4*>(wrow + s0), pk);
    } else {
      __stcs(reinterpret_cast<uint2*>(wrow + s0), make_uint2(pk.x, pk.y));
      __stcs(reinterpret_cast<uint2*>(wrow + s0 + 4), make_uint2(pk.z, pk.w));
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (s0 + k < nt) {
        yrow[s0 + k] = y[k];
        wrow[s0 + k] = (uint16_t)w[k];
      }
  }
}

// Candidate block-count sets --------------------------------------------------
struct AllM {  // every block count 1..MMAX (BoxDIT iterations, the exhaustive search)
  __host__ __device__ static constexpr bool in(int) { return true; }
  __host__ __device__ static constexpr int rank(int m) { return m - 1; }
};

template <int D, int PL>
struct IgM {  // IGRID levels j >= 1: m = 2^p + q 2^(p-d), q < 2^d (Eq. boxcarsize)
  static constexpr int MM = 1 << D, MBASE = 1 << PL, MSTEP = 1 << (PL - D);
  static constexpr int MMAX = MBASE + (MM - 1) * MSTEP;
  __host__ __device__ static constexpr bool in(int m) {
    return m >= MBASE && m <= MMAX && (m - MBASE) % MSTEP == 0;
  }
  __host__ __device__ static constexpr int rank(int m) { return (m - MBASE) / MSTEP; }
};

template <int D, int PL>
struct Ig0 {  // IGRID level 0: steps 0..p, all at separation 1
  static constexpr int MMAX = IgM<D, PL>::MMAX;
  __host__ __device__ static constexpr int ilog2(int m) {
    int i = 0;
    while ((2 << i) <= m) ++i;
    return i;
  }
  __host__ __device__ static constexpr bool in(int m) {
    return m >= 1 && m <= MMAX &&
           (m < (1 << D) ||
            (ilog2(m) <= PL && ((m - (1 << ilog2(m))) % (1 << (ilog2(m) - D))) == 0));
  }
  __host__ __device__ static constexpr int rank(int m) {
    int r = 0;
    for (int q = 1; q < m; ++q) r += in(q) ? 1 : 0;
    return r;
  }
};

// Evaluate NP consecutive positions of one level from a register window w[]
// (w[r + m - 1] is block m of position r).  Running sums start from base[r] (or
// 0) and add block counts m = 1..MMAX in order; at every m of the set the sum
// times scale(m) is compared (strict '>') against the best so far.  Returns
// the best value and its rank within the set, and the full MMAX-block sum.
// PARTIAL: only ranks below n_used count (the last level of a grid).
template <int NP, int MMAX, class Pred, bool PARTIAL, bool HAS_BASE, class Scale>
__device__ __forceinline__ void eval_window(const float* w, int n_used, Scale&& scale,
                                            const float* base, float (&bv)[NP], int (&bq)[NP],
                                            float (&full)[NP]) {
  static_for<0, NP>([&](auto R) {
    constexpr int r = decltype(R)::value;
    float S = HAS_BASE ? base[r] : 0.0f;
    float best = ninf();
    int q = 0;
    static_for<1, MMAX + 1>([&](auto M) {
      constexpr int m = decltype(M)::value;
      S += w[r + m - 1];
      if constexpr (Pred::in(m)) {
        constexpr int rk = Pred::rank(m);
        const float v = snr_of(S, scale(M));
        if constexpr (rk == 0) {
          best = v;
          q = 0;
        } else {
          if (!PARTIAL || rk < n_used) {
            if (v > best) {
              best = v;
              q = rk;
            }
          }
        }
      }
    });
    bv[r] = best;
    bq[r] = q;
    full[r] = S;
  });
}

// Three-input maximum (one instruction on sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

template <class Pred, int MMAX>
__host__ __device__ constexpr int count_in() {
  int n = 0;
  for (int m = 1; m <= MMAX; ++m) n += Pred::in(m) ? 1 : 0;
  return n;
}

// Maximum of v[0..N) with three-input max instructions.
template <int N>
__device__ __forceinline__ float tree_max(const float (&v)[N]) {
  if constexpr (N == 1) {
    return v[0];
  } else if constexpr (N == 2) {
    return fmaxf(v[0], v[1]);
  } else {
    float acc = fmax3(v[0], v[1], v[2]);
    static_for<0, (N - 3) / 2>([&](auto I) {
      constexpr int i = 3 + 2 * decltype(I)::value;
      acc = fmax3(acc, v[i], v[i + 1]);
    });
    if constexpr (((N - 3) % 2) == 1) acc = fmaxf(acc, v[N - 1]);
    return acc;
  }
}

// eval_window without PARTIAL, computed another way: the candidates' scaled
// sums are kept, their maximum is taken with three-input max instructions, and
// the rank is the first candidate equal to it (the smallest width on ties, as
// with the strict '>' scan in increasing width order).  Running sums start from
// base[r] when HAS_BASE; full[r] receives the MMAX-block sum.
template <int NP, int MMAX, class Pred, bool HAS_BASE, class Scale>
__device__ __forceinline__ void eval_window_mxb(const float* w, const float* base, Scale&& scale,
                                                float (&bv)[NP], int (&bq)[NP], float (&full)[NP]) {
  constexpr int NC = count_in<Pred, MMAX>();
  static_for<0, NP>([&](auto R) {
    constexpr int r = decltype(R)::value;
    float v[NC];
    float S = HAS_BASE ? base[r] : 0.0f;
    static_for<1, MMAX + 1>([&](auto M) {
      constexpr int m = decltype(M)::value;
      S += w[r + m - 1];
      if constexpr (Pred::in(m)) v[Pred::rank(m)] = snr_of(S, scale(M));
    });
    const float best = tree_max<NC>(v);
    int q = NC - 1;
    static_for<0, NC - 1>([&](auto C) {
      constexpr int c = NC - 2 - decltype(C)::value;
      if (v[c] == best) q = c;
    });
    bv[r] = best;
    bq[r] = q;
    full[r] = S;
  });
}

template <int NP, int MMAX, class Pred, class Scale>
__device__ __forceinline__ void eval_window_mx(const float* w, Scale&& scale, float (&bv)[NP],
                                               int (&bq)[NP]) {
  float full[NP];
  eval_window_mxb<NP, MMAX, Pred, false>(w, nullptr, scale, bv, bq, full);
}

// Like eval_window_mx for one position, but only ranks below n_used count
// (the last level of a grid); the others are set to -inf without branching.
template <int MMAX, class Pred, class Scale>
__device__ __forceinline__ void eval_one_masked(const float* w, int n_used, Scale&& scale,
                                                float& bv, int& bq) {
  constexpr int NC = count_in<Pred, MMAX>();
  float v[NC];
  float S = 0.0f;
  static_for<1, MMAX + 1>([&](auto M) {
    constexpr int m = decltype(M)::value;
    S += w[m - 1];
    if constexpr (Pred::in(m)) {
      constexpr int rk = Pred::rank(m);
      const float x = snr_of(S, scale(M));
      v[rk] = (rk == 0 || rk < n_used) ? x : ninf();
    }
  });
  const float best = tree_max<NC>(v);
  int q = NC - 1;
  static_for<0, NC - 1>([&](auto C) {
    constexpr int c = NC - 2 - decltype(C)::value;
    if (v[c] == best) q = c;
  });
  bv = best;
  bq = q;
}

// Load a window of NW float4s from 16-byte aligned shared memory.
template <int NW>
__device__ __forceinline__ void load_window4(const float* src, float (&w)[NW * 4]) {
  static_for<0, NW>([&](auto K) {
    constexpr int k = decltype(K)::value;
    const float4 t = *reinterpret_cast<const float4*>(src + 4 * k);
    w[4 * k + 0] = t.x;
    w[4 * k + 1] = t.y;
    w[4 * k + 2] = t.z;
    w[4 * k + 3] = t.w;
  });
}

template <int NW>
__device__ __forceinline__ void load_window2(const float* src, float (&w)[NW * 2]) {
  static_for<0, NW>([&](auto K) {
    constexpr int k = decltype(K)::value;
    const float2 t = *reinterpret_cast<const float2*>(src + 2 * k);
    w[2 * k + 0] = t.x;
    w[2 * k + 1] = t.y;
  });
}

template <int NW>
__device__ __forceinline__ void load_window1(const float* src, float (&w)[NW]) {
  static_for<0, NW>([&](auto K) {
    constexpr int k = decltype(K)::value;
    w[k] = src[k];
  });
}

__device__ __forceinline__ void merge1(float& y, int& w, float ny, int nw) {
  if (ny > y) {
    y = ny;
    w = nw;
  }
}

// launch helper
template <class KernelT>
cudaError_t launch_one(KernelT kern, size_t smem, int64_t nblk, const SearchParams& p,
                       cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)nblk, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace spd
