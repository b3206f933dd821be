// spd_common.cuh -- device helpers shared by the search kernels.
#pragma once

#include <cuda_fp16.h>
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
// The same for two sums at once (packed f32x2: identical roundings).
__device__ __forceinline__ float2 snr_of2(float2 S, float sc) { return __fmul2_rn(S, make_float2(sc, sc)); }
__device__ __forceinline__ float2 snr_of2(float2 S, float2 ab) {
  return __ffma2_rn(S, make_float2(ab.x, ab.x), make_float2(ab.y, ab.y));
}

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
__device__ __forceinline__ void row_noise(const SearchParams& p, const float* mu_tab,
                                          const float* sigma_tab, int64_t row, float2* AB, float& mu,
                                          float& inv) {
  if constexpr (!TABLE) {
    mu = mu_tab[row];
    inv = 1.0f / sigma_tab[row];
  } else {
    const float* m = mu_tab + row * p.n_widths;
    const float* s = sigma_tab + row * p.n_widths;
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

// Warp-reduced maximum of v folded into the candidate-tile maximum of start s
// (tm_row: the row's tile keys, or null).
__device__ __forceinline__ void tile_max_atomic(int* tm_row, int64_t s, float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  if ((threadIdx.x & 31) == 0 && tm_row) atomicMax(tm_row + s / kCandTile, fkey(v));
}

// One unit of a streaming search: segment [t0, t0 + T) of one row (plus the
// halo after it), with the row's pointers, length and noise.
struct Unit {
  const unsigned char* xrow;  // the row's first sample (bytes)
  float* yrow;
  uint16_t* wrow;
  const float* mu;            // noise table base and the row index into it
  const float* sigma;
  int* tm_row;                // the row's candidate-tile keys (or null)
  int64_t row, nt, t0;
  int64_t ns;                 // starts of the row that are evaluated (<= nt)
  int32_t T;
  bool vec, vec_x;
};

// Unit u of a single-series search: row u / tiles_per_row, segment u % tiles_per_row.
__device__ __forceinline__ Unit plan_unit(const SearchParams& p, int64_t u) {
  Unit U;
  U.row = u / p.tiles_per_row;
  U.t0 = (u % p.tiles_per_row) * (int64_t)p.tile;
  U.T = p.tile;
  U.nt = p.nt;
  U.ns = p.n_starts;
  U.xrow = static_cast<const unsigned char*>(p.x) + U.row * p.ld * p.esize;
  U.yrow = p.snr + U.row * p.ld;
  U.wrow = p.widx + U.row * p.ld;
  U.mu = p.mu;
  U.sigma = p.sigma;
  U.tm_row = p.tile_max ? reinterpret_cast<int*>(p.tile_max) + U.row * p.cand_tiles_per_row : nullptr;
  U.vec = p.vec != 0;
  U.vec_x = p.vec_x != 0;
  return U;
}

// Unit u of a batched search (ranges in unit order).  If the range has a ready
// flag, thread 0 waits for it (nanosleep polling, at most p.wait_ns by the
// global timer, and at most 2^26 polls); when a wait runs out, the range's bit
// of *p.status is set and this and every later unit of the range are skipped.
// Returns false when the unit is skipped (uniform over the CTA).
__device__ __forceinline__ bool batch_unit(const SearchParams& p, int64_t u, Unit& U, int* flag) {
  int r = 0;
  while (r + 1 < p.n_ranges && u >= p.ranges[r + 1].unit_first) ++r;
  const BatchRange& g = p.ranges[r];
  if (g.ready) {
    if (threadIdx.x == 0) {
      int ok = (atomicOr(p.status, 0) >> r) & 1 ? 0 : 1;
      if (ok && *reinterpret_cast<const volatile int32_t*>(g.ready) == 0) {
        unsigned long long t_start, t_now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
        ok = 0;
        for (int it = 0; it < (1 << 26); ++it) {
          if (*reinterpret_cast<const volatile int32_t*>(g.ready) != 0) {
            ok = 1;
            break;
          }
          asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_now));
          if ((long long)(t_now - t_start) > p.wait_ns) break;
          __nanosleep(1000);
        }
        if (!ok) atomicOr(p.status, 1 << r);
      }
      *flag = ok;
    }
    __syncthreads();
    const bool ok = *flag != 0;
    __syncthreads();  // the flag is reused by the next unit
    if (!ok) return false;
  }
  const int64_t local = u - g.unit_first;
  U.row = local / g.tiles_per_row;
  U.t0 = (local % g.tiles_per_row) * (int64_t)g.tile;
  U.T = g.tile;
  U.nt = g.nt;
  U.ns = g.nt;
  U.xrow = static_cast<const unsigned char*>(g.x) + U.row * g.ld * p.esize;
  U.yrow = g.snr + U.row * g.ld;
  U.wrow = g.widx + U.row * g.ld;
  U.mu = g.mu;
  U.sigma = g.sigma;
  U.tm_row = reinterpret_cast<int*>(g.tile_max) + U.row * g.cand_tiles_per_row;
  U.vec = g.vec != 0;
  U.vec_x = g.vec_x != 0;
  return true;
}

// ---------------------------------------------------------------- input samples
// Input sample types (the spd_dtype values).  Rows are addressed as bytes.
constexpr int kDtF32 = 0, kDtF16 = 1, kDtBF16 = 2, kDtU8 = 3;

__device__ __forceinline__ float f16_bits(uint32_t h) { return __half2float(__ushort_as_half((unsigned short)h)); }

// Eight consecutive samples of one row as stored: f32 in a and b, f16/bf16 in
// a (two per word, the earlier sample in the low half), u8 in a.x, a.y (four
// per word, the earliest in the low byte).
struct Raw8 {
  uint4 a, b;
};

// Raw samples [pos, pos + 8) of the row at byte pointer `row`; n = samples that
// exist.  One 32/16/8-byte vector load per thread when vec (row and samples
// 16-byte aligned) and all 8 exist; element loads otherwise (missing ones 0).
__device__ __forceinline__ Raw8 load_raw8(const unsigned char* __restrict__ row, int pos, int n,
                                          int dtype, bool vec) {
  Raw8 r;
  if (vec && pos + 8 <= n) {
    if (dtype == kDtF32) {
      const uint4* q = reinterpret_cast<const uint4*>(row + 4 * pos);
      r.a = __ldg(q);
      r.b = __ldg(q + 1);
    } else if (dtype == kDtU8) {
      const uint2 v = __ldg(reinterpret_cast<const uint2*>(row + pos));
      r.a = make_uint4(v.x, v.y, 0u, 0u);
      r.b = make_uint4(0u, 0u, 0u, 0u);
    } else {
      r.a = __ldg(reinterpret_cast<const uint4*>(row + 2 * pos));
      r.b = make_uint4(0u, 0u, 0u, 0u);
    }
    return r;
  }
  uint32_t w[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (pos + i < n) {
      if (dtype == kDtF32) {
        w[i] = __ldg(reinterpret_cast<const unsigned int*>(row) + pos + i);
      } else if (dtype == kDtU8) {
        w[i >> 2] |= (uint32_t)__ldg(row + pos + i) << (8 * (i & 3));
      } else {
        w[i >> 1] |= (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(row) + pos + i) << (16 * (i & 1));
      }
    }
  }
  r.a = make_uint4(w[0], w[1], w[2], w[3]);
  r.b = make_uint4(w[4], w[5], w[6], w[7]);
  return r;
}

// The samples of load_raw8 as floats, normalised to (x - mu) * inv (NORM; the
// raw values otherwise); samples at or past n are -inf.
template <bool NORM = true>
__device__ __forceinline__ void cvt8(const Raw8& r, int pos, int n, int dtype, float mu, float inv,
                                     float4& v0, float4& v1) {
  float f[8];
  const uint32_t wa[4] = {r.a.x, r.a.y, r.a.z, r.a.w};
  if (dtype == kDtF32) {
    const uint32_t wb[4] = {r.b.x, r.b.y, r.b.z, r.b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[i] = __uint_as_float(wa[i]);
      f[4 + i] = __uint_as_float(wb[i]);
    }
  } else if (dtype == kDtF16) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[2 * i] = f16_bits(wa[i] & 0xffffu);
      f[2 * i + 1] = f16_bits(wa[i] >> 16);
    }
  } else if (dtype == kDtBF16) {  // bf16 is the high half of an f32
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[2 * i] = __uint_as_float(wa[i] << 16);
      f[2 * i + 1] = __uint_as_float(wa[i] & 0xffff0000u);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) f[i] = __uint2float_rn((wa[i >> 2] >> (8 * (i & 3))) & 0xffu);
  }
  if constexpr (NORM) {
#pragma unroll
    for (int i = 0; i < 8; i += 2) {  // packed pairs: x + (-mu) rounds as x - mu
      const float2 z =
          __fmul2_rn(__fadd2_rn(make_float2(f[i], f[i + 1]), make_float2(-mu, -mu)), make_float2(inv, inv));
      f[i] = z.x;
      f[i + 1] = z.y;
    }
  }
  if (pos + 8 > n) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (pos + i >= n) f[i] = ninf();
  }
  v0 = make_float4(f[0], f[1], f[2], f[3]);
  v1 = make_float4(f[4], f[5], f[6], f[7]);
}

// z-values of samples [pos, pos + 4) of the row at byte pointer `row` (any
// input type); -inf at and past nt.
__device__ __forceinline__ float4 load_z4d(const unsigned char* __restrict__ row, int64_t pos, int64_t nt,
                                           int dtype, bool vec, float mu, float inv) {
  float f[4];
  if (vec && pos + 4 <= nt) {
    if (dtype == kDtF32) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(row + 4 * pos));
      f[0] = v.x, f[1] = v.y, f[2] = v.z, f[3] = v.w;
    } else if (dtype == kDtU8) {
      const uint32_t v = __ldg(reinterpret_cast<const unsigned int*>(row + pos));
#pragma unroll
      for (int i = 0; i < 4; ++i) f[i] = __uint2float_rn((v >> (8 * i)) & 0xffu);
    } else {
      const uint2 v = __ldg(reinterpret_cast<const uint2*>(row + 2 * pos));
      const uint32_t w[2] = {v.x, v.y};
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        if (dtype == kDtF16) {
          f[2 * i] = f16_bits(w[i] & 0xffffu);
          f[2 * i + 1] = f16_bits(w[i] >> 16);
        } else {
          f[2 * i] = __uint_as_float(w[i] << 16);
          f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) f[i] = (f[i] - mu) * inv;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (pos + i < nt) {
        float v;
        if (dtype == kDtF32) v = __ldg(reinterpret_cast<const float*>(row) + pos + i);
        else if (dtype == kDtU8) v = __uint2float_rn(__ldg(row + pos + i));
        else if (dtype == kDtF16) v = f16_bits(__ldg(reinterpret_cast<const unsigned short*>(row) + pos + i));
        else v = __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(row) + pos + i) << 16);
        f[i] = (v - mu) * inv;
      } else {
        f[i] = ninf();
      }
    }
  }
  return make_float4(f[0], f[1], f[2], f[3]);
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

// vec: Y base 16-byte aligned, W base 8-byte aligned, ld % 4 == 0 (so Y rows
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

// ---------------------------------------------------------------- coded SNRs
// For grids of at most 2^B widths the width index can travel in the B low
// mantissa bits of an SNR (code = 2^B - 1 - index): the maximum of coded values
// is the maximum SNR to within 2^B - 1 ulp and, among values equal to that
// resolution, the smallest index wins (positive values); maxima and merges are
// then single max instructions.  A -inf candidate becomes a NaN, which max
// ignores; a maximum over NaNs only is the canonical (positive) NaN, which
// callers must treat as "no candidate" before using it as an ordered key.
//
// The code is set with one logic instruction: (v | low) & (~low | code), where
// low = 2^B - 1 sits in a register (opaque to the compiler, so that it is not
// folded back into the two-instruction (v & ~low) | code) and ~low | code is the
// instruction's immediate.
__device__ __forceinline__ int opaque_int(int v) {
  int r;
  asm("mov.b32 %0, %1;" : "=r"(r) : "r"(v));
  return r;
}
template <int B>
__device__ __forceinline__ float enc_w(float v, int code) {
  int r;
  asm("lop3.b32 %0, %1, %2, %3, 0xC8;"
      : "=r"(r)
      : "r"(__float_as_int(v)), "r"(~((1 << B) - 1) | code), "r"(opaque_int((1 << B) - 1)));
  return __int_as_float(r);
}
template <int B>
__device__ __forceinline__ int dec_w(float v) {
  return ((1 << B) - 1) - (__float_as_int(v) & ((1 << B) - 1));
}
template <int B>
__device__ __forceinline__ float dec_v(float v) {
  return __int_as_float(__float_as_int(v) & ~((1 << B) - 1));
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

// Coded evaluation of NP consecutive positions (see enc_w): out[r] is the
// maximum over the set of enc_w(SNR, code(rank)), with code(rank) = code0 -
// rank; PARTIAL: ranks at or above n_used (rank 0 always counts) are -inf.
//
// With several positions (NP >= 2) the sums are built from pair sums
// P[i] = w[i] + w[i+1] shared by the positions: the sum of an even number m of
// blocks extends the one of m - 2 by P[r + m - 2], an odd count adds one block
// to the even sum below it; odd counts outside the set are never formed.
// Coded candidate of rank RK into v[RK] (-inf when PARTIAL and RK >= n_used, RK > 0).
template <int B, bool PARTIAL, int RK, int NC>
__device__ __forceinline__ void enc_post(float x, int code0, int n_used, float (&v)[NC]) {
  const float c = enc_w<B>(x, code0 - RK);
  if constexpr (PARTIAL && RK > 0)
    v[RK] = RK < n_used ? c : ninf();
  else
    v[RK] = c;
}

//
// UNIT1: the scale of block count 1 is exactly 1 (white noise, width 1), so that
// candidate is the sum itself, with no multiplication.
template <int NP, int MMAX, class Pred, int B, bool PARTIAL, bool UNIT1 = false, class Scale>
__device__ __forceinline__ void eval_window_enc(const float* w, int n_used, Scale&& scale, int code0,
                                                float (&out)[NP]) {
  constexpr int NC = count_in<Pred, MMAX>();
  constexpr bool PAIRS = NP >= 2 && MMAX >= 2;
  constexpr int NPAIR = PAIRS ? NP + MMAX - 2 : 1;
  float P[NPAIR];
  if constexpr (PAIRS) static_for<0, NPAIR>([&](auto I) {
      constexpr int i = decltype(I)::value;
      P[i] = w[i] + w[i + 1];
    });
  if constexpr (PAIRS && (NP % 2) == 0) {
    // two positions (r, r + 1) at a time in packed f32x2 arithmetic: the same
    // roundings as the scalar form, half the add and scale instructions.  Their
    // operands are aligned pairs: (P[r + m - 2], P[r + m - 1]) and
    // (w[r + m - 1], w[r + m]) with r even and m even resp. odd.
    static_for<0, NP / 2>([&](auto R2) {
      constexpr int r = 2 * decltype(R2)::value;
      float v0[NC], v1[NC];
      float2 Se = make_float2(0.0f, 0.0f);
      static_for<1, MMAX + 1>([&](auto M) {
        constexpr int m = decltype(M)::value;
        float2 Sm = make_float2(0.0f, 0.0f);
        if constexpr ((m & 1) == 0) {
          Se = (m == 2) ? make_float2(P[r], P[r + 1]) : __fadd2_rn(Se, make_float2(P[r + m - 2], P[r + m - 1]));
          Sm = Se;
        } else if constexpr (Pred::in(m)) {
          Sm = (m == 1) ? make_float2(w[r], w[r + 1]) : __fadd2_rn(Se, make_float2(w[r + m - 1], w[r + m]));
        }
        if constexpr (Pred::in(m)) {
          const float2 x = (UNIT1 && m == 1) ? Sm : snr_of2(Sm, scale(M));
          enc_post<B, PARTIAL, Pred::rank(m)>(x.x, code0, n_used, v0);
          enc_post<B, PARTIAL, Pred::rank(m)>(x.y, code0, n_used, v1);
        }
      });
      out[r] = tree_max<NC>(v0);
      out[r + 1] = tree_max<NC>(v1);
    });
  } else {
    static_for<0, NP>([&](auto R) {
      constexpr int r = decltype(R)::value;
      float v[NC];
      float S = 0.0f, Se = 0.0f;  // running sum; pairs: the sum of the last even count
      static_for<1, MMAX + 1>([&](auto M) {
        constexpr int m = decltype(M)::value;
        float Sm;
        if constexpr (!PAIRS) {
          S += w[r + m - 1];
          Sm = S;
        } else if constexpr ((m & 1) == 0) {
          Se = (m == 2) ? P[r] : Se + P[r + m - 2];
          Sm = Se;
        } else if constexpr (Pred::in(m)) {
          Sm = (m == 1) ? w[r] : Se + w[r + m - 1];
        } else {
          Sm = 0.0f;  // not formed
        }
        if constexpr (Pred::in(m))
          enc_post<B, PARTIAL, Pred::rank(m)>((UNIT1 && m == 1) ? Sm : snr_of(Sm, scale(M)), code0, n_used, v);
      });
      out[r] = tree_max<NC>(v);
    });
  }
}

// Coded evaluation of one BoxDIT level (Alg. 1: block counts m = 1..K, every
// one a candidate) at NP consecutive positions: S_m = base[r] + w[r] + ... +
// w[r + m - 1] (added in block order, as the shifted decimation adds them), the
// SNR S_m * scale(m) coded with its rank m - 1 (code 31 - (m - 1), see enc_w),
// and out[r] = the coded maximum over m (PARTIAL: ranks >= n_used count as
// -inf); full[r] = S_K, the level's widest boxcar, the base of the next level.
// Two positions share each scale instruction (packed f32x2; the sums are added
// in packed form where the two addends are an aligned pair), and the maximum is
// kept running, so no candidate outlives its step.
template <int NP, int K, bool HAS_BASE, bool PARTIAL, class Scale>
__device__ __forceinline__ void eval_bd_enc(const float* w, const float* base, int n_used, Scale&& scale,
                                            float (&out)[NP], float (&full)[NP]) {
  static_assert(K <= 32 && K % 2 == 0, "5-bit codes, block counts in pairs");
  auto keep = [&](float c, auto M) {
    constexpr int m = decltype(M)::value;
    if constexpr (PARTIAL && m > 1)
      return (m - 1 < n_used) ? c : ninf();
    else
      return c;
  };
  if constexpr (NP % 2 == 0) {
    static_for<0, NP / 2>([&](auto R2) {
      constexpr int r = 2 * decltype(R2)::value;
      float2 S = HAS_BASE ? make_float2(base[r], base[r + 1]) : make_float2(0.0f, 0.0f);
      float a0 = ninf(), a1 = ninf(), c0 = ninf(), c1 = ninf();
      static_for<1, K + 1>([&](auto M) {
        constexpr int m = decltype(M)::value;
        if constexpr (m == 1 && !HAS_BASE) {
          S = make_float2(w[r], w[r + 1]);
        } else if constexpr (((r + m - 1) & 1) == 0) {
          S = __fadd2_rn(S, make_float2(w[r + m - 1], w[r + m]));
        } else {
          S.x += w[r + m - 1];
          S.y += w[r + m];
        }
        const float2 x = snr_of2(S, scale(M));
        const float e0 = keep(enc_w<5>(x.x, 32 - m), M), e1 = keep(enc_w<5>(x.y, 32 - m), M);
        if constexpr (m & 1) {
          c0 = e0;
          c1 = e1;
        } else {
          a0 = fmax3(a0, c0, e0);
          a1 = fmax3(a1, c1, e1);
        }
      });
      out[r] = a0;
      out[r + 1] = a1;
      full[r] = S.x;
      full[r + 1] = S.y;
    });
  } else {
    static_for<0, NP>([&](auto R) {
      constexpr int r = decltype(R)::value;
      float S = HAS_BASE ? base[r] : 0.0f;
      float a = ninf(), c = ninf();
      static_for<1, K + 1>([&](auto M) {
        constexpr int m = decltype(M)::value;
        S = (m == 1 && !HAS_BASE) ? w[r] : S + w[r + m - 1];
        const float e = keep(enc_w<5>(snr_of(S, scale(M)), 32 - m), M);
        if constexpr (m & 1)
          c = e;
        else
          a = fmax3(a, c, e);
      });
      out[r] = a;
      full[r] = S;
    });
  }
}

// Coded evaluation of one level of an arbitrary block-count set at NP
// consecutive positions, for sets whose largest count MMAX is too large for
// eval_window_enc's pair sums: S_m = w[r] + ... + w[r + m - 1] added in block
// order, and at every count m of the set the SNR S_m * scale(m) coded with its
// rank in the set (code 31 - rank, B = 5: at most 32 counts), kept as a running
// maximum; out[r] is that coded maximum (PARTIAL: ranks >= n_used, except rank
// 0, count as -inf).  Two positions share each scale instruction (packed f32x2).
template <int NP, int MMAX, class Pred, bool PARTIAL, class Scale>
__device__ __forceinline__ void eval_set_enc(const float* w, int n_used, Scale&& scale, float (&out)[NP]) {
  static_assert(count_in<Pred, MMAX>() <= 32, "5-bit codes");
  auto code = [&](float x, auto M) {
    constexpr int rk = Pred::rank(decltype(M)::value);
    const float c = enc_w<5>(x, 31 - rk);
    if constexpr (PARTIAL && rk > 0)
      return rk < n_used ? c : ninf();
    else
      return c;
  };
  if constexpr (NP % 2 == 0) {
    static_for<0, NP / 2>([&](auto R2) {
      constexpr int r = 2 * decltype(R2)::value;
      float2 S = make_float2(w[r], w[r + 1]);
      float a0 = ninf(), a1 = ninf();
      static_for<1, MMAX + 1>([&](auto M) {
        constexpr int m = decltype(M)::value;
        if constexpr (m > 1) {
          if constexpr (((r + m - 1) & 1) == 0) {
            S = __fadd2_rn(S, make_float2(w[r + m - 1], w[r + m]));
          } else {
            S.x += w[r + m - 1];
            S.y += w[r + m];
          }
        }
        if constexpr (Pred::in(m)) {
          const float2 x = snr_of2(S, scale(M));
          a0 = fmaxf(a0, code(x.x, M));
          a1 = fmaxf(a1, code(x.y, M));
        }
      });
      out[r] = a0;
      out[r + 1] = a1;
    });
  } else {
    static_for<0, NP>([&](auto R) {
      constexpr int r = decltype(R)::value;
      float S = w[r], a = ninf();
      static_for<1, MMAX + 1>([&](auto M) {
        constexpr int m = decltype(M)::value;
        if constexpr (m > 1) S += w[r + m - 1];
        if constexpr (Pred::in(m)) a = fmaxf(a, code(snr_of(S, scale(M)), M));
      });
      out[r] = a;
    });
  }
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

// Window of NW float4s from a split layout: float4 k at src + 4 (k / 2), plus
// ob (the odd array's offset) for odd k.
template <int NW>
__device__ __forceinline__ void load_window4_ab(const float* src, int ob, float (&w)[NW * 4]) {
  static_for<0, NW>([&](auto K) {
    constexpr int k = decltype(K)::value;
    const float4 t = *reinterpret_cast<const float4*>(src + 4 * (k / 2) + ((k & 1) ? ob : 0));
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

// store8 with the eight 16-bit widths already packed in pairs (pk[q]: width of
// start 2q in the low half, 2q + 1 in the high half).
__device__ __forceinline__ void store8_pk(float* __restrict__ yrow, uint16_t* __restrict__ wrow,
                                          int64_t s0, int64_t nt, bool vec, const float (&y)[8],
                                          const uint32_t (&pk)[4]) {
  if (vec && s0 + 8 <= nt) {
    __stcs(reinterpret_cast<float4*>(yrow + s0), make_float4(y[0], y[1], y[2], y[3]));
    __stcs(reinterpret_cast<float4*>(yrow + s0 + 4), make_float4(y[4], y[5], y[6], y[7]));
    if ((reinterpret_cast<uintptr_t>(wrow + s0) & 15) == 0) {
      __stcs(reinterpret_cast<uint4*>(wrow + s0), make_uint4(pk[0], pk[1], pk[2], pk[3]));
    } else {
      __stcs(reinterpret_cast<uint2*>(wrow + s0), make_uint2(pk[0], pk[1]));
      __stcs(reinterpret_cast<uint2*>(wrow + s0 + 4), make_uint2(pk[2], pk[3]));
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (s0 + k < nt) {
        yrow[s0 + k] = y[k];
        wrow[s0 + k] = (uint16_t)(pk[k >> 1] >> (16 * (k & 1)));
      }
  }
}

// The width indices of two coded SNRs (code = 2^B - 1 - index, B <= 8) packed as
// 16-bit halves: one byte permute gathers both low bytes, one logic instruction
// inverts and masks them (2^B - 1 - c == ~c & (2^B - 1)).
template <int B>
__device__ __forceinline__ uint32_t dec_w_pair(float lo, float hi) {
  static_assert(B <= 8, "the code must fit in the low byte");
  const uint32_t m = (1u << B) - 1u;
  return ~__byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x5410) & (m | (m << 16));
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
