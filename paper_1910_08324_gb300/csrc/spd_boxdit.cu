// spd_boxdit.cu -- BoxDIT BD-K search kernel (Sec. 3.1, Alg. 1).
//
// The grid, written as levels (spd_internal.h): level i is iteration i of
// Alg. 1 -- unit 2^i, starts s = n 2^i, widths c_i + m 2^i (m = 1..K) with
// c_i = K (2^i - 1).  Its candidates extend the level's base boxcar X_{c_i}[s]
// (Alg. 1's X^{i-1}, the widest boxcar of the previous iteration at s) by m
// blocks of 2^i samples that start c_i samples after s (the "shifted"
// decimation of Sec. 3.1).
//
// One CTA streams one segment of one DM row backwards in time, 2048-sample
// chunks at a time, with the same software pipeline as the IGRID kernel (one
// barrier per chunk): build chunk k+1 (normalise, pyramid, rings) -> barrier ->
// coarse work of chunk k+1 + fine work of chunk k.
//
//   fine levels 0..3: each thread owns 8 consecutive starts and evaluates them
//     at levels 0..3 (8, 4, 2, 1 positions) from register windows of shared-
//     memory block series.  Alg. 1's chain of base boxcars stays in registers:
//     the widest sum of level i at a start is the base of level i+1 there.
//   coarse levels 4..top: one thread per position.  Its base is not taken from
//     the previous level (that would chain threads); it is summed directly from
//     two ring buffers of the level: A_j (aligned 2^j-sample blocks) and, for
//     levels past log2(K), R_j (the first 2^j - K samples of an aligned block).
//     With n = s / 2^j,
//       j <= log2 K:  X_{c_j + m 2^j}[s] = sum_{t < c_j/2^j + m} A_j[n + t]
//       j >  log2 K:  X_{c_j + m 2^j}[s] = sum_{t < K - 1 + m} A_j[n + t] + R_j[n + K - 1 + m]
//     (c_j = (K - 1) 2^j + (2^j - K) when 2^j > K).  These are the same sums as
//     Alg. 1's, added in another order (fp32 rounding differs, exactness of the
//     grid does not).
// Coarse results reach the fine step of their chunk through a per-start atomic
// key, as in the IGRID kernel.  Samples past the end of a row are -inf; starts at
// or past the plan's n_starts are neither evaluated nor stored.
#include <climits>

#include "spd_common.cuh"

namespace spd {
namespace {

constexpr int kC = kChunk;
constexpr int kRing0 = 4;     // first ring level
constexpr int kChunkLog = 11;  // BoxDIT plans never go past level 11 (widths <= kMaxLend)
constexpr int kResN = 256;    // coarse-result slots of one buffer (one per coarse thread)
constexpr int kBcm = kC / 16;  // starts = 0 mod 16 in a chunk

template <int K>
struct BdS {
  static constexpr int KAP = (K == 8) ? 3 : (K == 16) ? 4 : 5;
  static_assert((1 << KAP) == K, "K must be 8, 16 or 32");
  static constexpr int MIR = 2 * K;  // mirrored ring entries: a coarse window spans 2K blocks
  // the level-i window of a position starts c_i / 2^i = K - K / 2^i entries after it
  static constexpr int OF1 = K / 2, OF2 = 3 * K / 4, OF3 = 7 * K / 8;
  static constexpr int NW0 = cdiv(7 + K, 4);  // float4s: 8 starts + K - 1 lookahead
  static constexpr int NW1 = cdiv(3 + K, 4);  // float4s: 4 positions
  static constexpr int NW2 = cdiv(1 + K, 2);  // float2s: 2 positions
  static constexpr int NW3 = K;               // scalars: 1 position
  static constexpr int TL0 = 4 * NW0 - 8;     // lookahead tails past the chunk
  static constexpr int TL1 = OF1 + 4 * NW1 - 4;
  static constexpr int TL2 = OF2 + 2 * NW2 - 2;
  static constexpr int TL3 = OF3 + NW3 - 1;
  static_assert(OF1 % 4 == 0 && OF2 % 2 == 0, "vector windows must stay aligned");
  static_assert(TL0 % 4 == 0 && TL1 % 4 == 0 && TL2 % 2 == 0, "tails are written as vectors");
  static constexpr int O1 = al4(kC + TL0);
  static constexpr int O2 = O1 + al4(kC / 2 + TL1);
  static constexpr int O3 = O2 + al4(kC / 4 + TL2);
  static constexpr int FB = O3 + al4(kC / 8 + TL3);  // one buffer of levels 0..3
  static constexpr int NBUF = 4;
  static constexpr int RINGS = NBUF * FB;
  __host__ __device__ static constexpr int f0(int b) { return b * FB; }
  __host__ __device__ static constexpr int f1(int b) { return b * FB + O1; }
  __host__ __device__ static constexpr int f2(int b) { return b * FB + O2; }
  __host__ __device__ static constexpr int f3(int b) { return b * FB + O3; }
};

// A ring holds every block a coarse window of the chunk being evaluated can
// reach plus the blocks of the chunk being built meanwhile.
template <int K>
__host__ __device__ constexpr int bd_ring_size(int j) {
  return next_pow2(cdiv(2 * kC, 1 << j) + 2 * K + 2);
}

// Offsets (floats) after the level buffers: rings (A_j, then R_j for j > log2 K,
// each with MIR mirrored entries), coarse results (two buffers), the
// coarse-merge keys (two buffers), the ring table and the coarse scale table.
template <int K>
struct BdDyn {
  int res_y, res_w, bcm, tab, stab, ab, total;
  // nab: widths of the table-noise constants (0 for white noise)
  __host__ __device__ BdDyn(int top, int nab) {
    using S = BdS<K>;
    int o = S::RINGS;
    for (int j = kRing0; j <= top; ++j) {
      const int n = bd_ring_size<K>(j) + S::MIR;
      o += al4(n) * (j > S::KAP ? 2 : 1);
    }
    res_y = o;
    o += 2 * kResN;
    res_w = o;
    o += kResN;  // 2 x kResN uint16
    bcm = o;
    o += 2 * kBcm;
    tab = o;
    o += 3 * kMaxLevels;
    stab = o;
    o += al4(kMaxLevels * (K + 1));
    ab = o;
    o += nab ? al4(2 * (nab + kAbPad)) : 0;
    total = o;
  }
};

// One coarse position: widths c_j + m 2^j, m = 1..K (ranks >= nu masked out).
// A points at the window's first aligned block (SKIP0: one block earlier, for
// the level whose base is K - 2 blocks), R at R_j[n]; sc[m - 1] is the scale of
// block count m (a float, or a float2 (a, b) for table noise).  Returns the
// maximum SNR coded with its rank m - 1 (see enc_w), kept running.
template <int K, bool HAS_R, bool SKIP0, class SC>
__device__ __forceinline__ float bd_coarse_eval(const float* A, const float* R, const SC* sc, int nu) {
  float S = SKIP0 ? 0.0f : A[0];
  static_for<1, K - 1>([&](auto T) { S += A[decltype(T)::value]; });
  float acc = ninf(), c = ninf();
  static_for<1, K + 1>([&](auto M) {
    constexpr int m = decltype(M)::value;
    S += A[K - 2 + m];
    const float X = HAS_R ? S + R[K - 1 + m] : S;
    const float e = (m == 1 || m - 1 < nu) ? enc_w<5>(snr_of(X, sc[m - 1]), 32 - m) : ninf();
    if constexpr (m & 1)
      c = e;
    else
      acc = fmax3(acc, c, e);
  });
  return acc;
}

// Table noise with K = 32 keeps 32 (a, b) pairs of level 0 live: one CTA per
// SM leaves room for them without spilling.
template <int K, bool COARSE, bool TABLE>
__device__ __forceinline__ void boxdit_unit(const SearchParams& p, const Unit& U, float* smem) {
  using S = BdS<K>;
  constexpr int KAP = S::KAP;
  constexpr int MIR = S::MIR;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t row = U.row, t0 = U.t0;
  const int top = p.top;
  const int T = U.T, H = p.halo;
  const bool vec = U.vec;
  const unsigned char* __restrict__ xseg = U.xrow + t0 * p.esize;  // byte address
  const int dt = p.dtype;
  const bool vx = U.vec_x;
  float* __restrict__ yseg = U.yrow + t0;
  uint16_t* __restrict__ wseg = U.wrow + t0;
  const int64_t nleft = U.nt - t0;
  const int nrel = (int)(nleft < (int64_t)(T + H) ? nleft : (int64_t)(T + H));
  const int64_t sleft = U.ns - t0;
  const int srel = (int)(sleft < (int64_t)T ? sleft : (int64_t)T);  // starts evaluated and stored
  const BdDyn<K> L(top, TABLE ? p.n_widths : 0);
  float2* AB = reinterpret_cast<float2*>(smem + L.ab);  // table noise: (a, b) per width index
  float mu, inv;
  row_noise<TABLE>(p, U.mu, U.sigma, row, AB, mu, inv);
  float* RESY = smem + L.res_y;
  uint16_t* RESW = reinterpret_cast<uint16_t*>(smem + L.res_w);
  int* BCM = reinterpret_cast<int*>(smem + L.bcm);
  int* RTAB = reinterpret_cast<int*>(smem + L.tab);  // [3j]: A ring, [3j+1]: R ring, [3j+2]: mask
  float* STAB = smem + L.stab;                        // [j (K+1) + m] = 1/sqrt(c_j + m 2^j) (white noise)

  for (int i = t; i < L.bcm; i += kThreads) smem[i] = ninf();
  for (int i = t; i < 2 * kBcm; i += kThreads) BCM[i] = INT_MIN;
  for (int i = t; i < kMaxLevels * (K + 1); i += kThreads) {
    const int j = i / (K + 1), m = i % (K + 1);
    STAB[i] = (j <= top && m >= 1) ? p.bscale[j][m] : 0.0f;
  }
  if (t == 0) {
    int o = S::RINGS;
    for (int j = 0; j < kMaxLevels; ++j) RTAB[3 * j] = RTAB[3 * j + 1] = RTAB[3 * j + 2] = 0;
    for (int j = kRing0; j <= top; ++j) {
      const int n = bd_ring_size<K>(j);
      RTAB[3 * j] = o;
      o += al4(n + MIR);
      RTAB[3 * j + 1] = RTAB[3 * j];
      if (j > KAP) {
        RTAB[3 * j + 1] = o;
        o += al4(n + MIR);
      }
      RTAB[3 * j + 2] = n - 1;
    }
  }
  __syncthreads();
  auto ring_put = [&](int base, int mask, int n, float v) {
    const int slot = n & mask;
    smem[base + slot] = v;
    smem[base + (slot < MIR ? slot + mask + 1 : slot)] = v;
  };
  int a0 = T + H - kC;
  if (a0 >= nrel) a0 = ((nrel - 1) / kC) * kC;
  const int nch = a0 / kC + 1;

  // ring levels 4..8 written by every lane of a block: ring offsets and chunk-0 indices
  int ra[5] = {0, 0, 0, 0, 0}, rr[5] = {0, 0, 0, 0, 0}, rm[5] = {0, 0, 0, 0, 0}, rn[5] = {0, 0, 0, 0, 0};
  // this thread's coarse position: level cj (0 = none)
  const int ctop = top < kChunkLog ? top : kChunkLog;
  int cj = 0, ca = 0, cr = 0, cmask = 0, cn = 0, cnu = 0, cfirst = 0, cbcm = 0, ccode = 0;
  if (COARSE) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const int j = kRing0 + i;
      ra[i] = RTAB[3 * j];
      rr[i] = RTAB[3 * j + 1];
      rm[i] = RTAB[3 * j + 2];
      rn[i] = (a0 >> j) + (t >> (j - 3));
    }
    if (t < kThreads - (1 << (kChunkLog - ctop))) {
      int j = kRing0, off = 0;
      while (t >= off + (kC >> j)) {
        off += kC >> j;
        ++j;
      }
      const int cq = t - off;
      cj = j;
      ca = RTAB[3 * j];
      cr = RTAB[3 * j + 1];
      cmask = RTAB[3 * j + 2];
      cn = (a0 >> j) + cq;
      cnu = (j == top) ? p.n_top : K;
      cfirst = p.lvl_first[j];
      cbcm = cq << (j - 4);
      ccode = 15 - (j - 4);
    }
  }
  // level-9..11 blocks of a chunk: lane L of the last warp builds block lb of level lj
  // from lw level-8 blocks (lanes 0..3: level 9, 4..5: level 10, 6: level 11)
  const int lj = lane < 4 ? 9 : (lane < 6 ? 10 : 11);
  const int lb = lane < 4 ? lane : (lane < 6 ? lane - 4 : 0);
  const int lw = 1 << (lj - 8);
  const bool lbuild = COARSE && warp == kThreads / 32 - 1 && lane < 7 && lj <= top;

  // ---- build chunk k: levels 0..3 into buffer k % 4 (+ tails), rings 4..8 ----
  auto build = [&](int k, const Raw8& raw) {
    const int buf = k % S::NBUF, nbuf = (k + 1) % S::NBUF;
    float4 v0, v1;
    cvt8(raw, a0 - k * kC + 8 * t, nrel, dt, mu, inv, v0, v1);
    float* F0 = smem + S::f0(buf);
    *reinterpret_cast<float4*>(F0 + 8 * t) = v0;
    *reinterpret_cast<float4*>(F0 + 8 * t + 4) = v1;
    if (8 * t < S::TL0) {
      float* T0 = smem + S::f0(nbuf) + kC + 8 * t;
      *reinterpret_cast<float4*>(T0) = v0;
      if (8 * t + 4 < S::TL0) *reinterpret_cast<float4*>(T0 + 4) = v1;
    }
    const float p0 = v0.x + v0.y, p1 = v0.z + v0.w, p2 = v1.x + v1.y, p3 = v1.z + v1.w;
    const float4 pp = make_float4(p0, p1, p2, p3);
    *reinterpret_cast<float4*>(smem + S::f1(buf) + 4 * t) = pp;
    if (4 * t < S::TL1) *reinterpret_cast<float4*>(smem + S::f1(nbuf) + kC / 2 + 4 * t) = pp;
    const float q0 = p0 + p1, q1 = p2 + p3;
    *reinterpret_cast<float2*>(smem + S::f2(buf) + 2 * t) = make_float2(q0, q1);
    if (2 * t < S::TL2) *reinterpret_cast<float2*>(smem + S::f2(nbuf) + kC / 4 + 2 * t) = make_float2(q0, q1);
    const float o8 = q0 + q1;
    smem[S::f3(buf) + t] = o8;
    if (t < S::TL3) smem[S::f3(nbuf) + kC / 8 + t] = o8;
    if (COARSE) {
      const int d = k * kC;
      float s = o8, r = 0.0f;  // A and R of this lane's block at the current level (R_kappa = 0)
      static_for<0, 5>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int j = kRing0 + i;
        constexpr int dl = 1 << i;  // lanes per half block
        if (i == 0 || top >= j) {
          const float so = __shfl_xor_sync(kFull, s, dl);
          if constexpr (j > KAP) {
            // R_j = A_{j-1}(lower half) + R_{j-1}(upper half)
            const bool lower = (lane & dl) == 0;
            const float g = __shfl_xor_sync(kFull, lower ? s : r, dl);
            r = lower ? s + g : g + r;
          }
          s = s + so;
          const int n = rn[i] - (d >> j);
          ring_put(ra[i], rm[i], n, s);
          if constexpr (j > KAP) ring_put(rr[i], rm[i], n, r);
        }
      });
    }
  };

  // ---- coarse work of chunk k ----------------------------------------------
  auto coarse = [&](int k) {
    const int ar = a0 - k * kC;
    if (warp == kThreads / 32 - 1 && top >= 9) {
      if (lbuild) {  // A_lj and R_lj of block lb from level-8 blocks of this chunk
        const int n8 = (ar >> 8) + lb * lw;
        const float* A8 = smem + ra[4];
        const float* R8 = smem + rr[4];
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < 7; ++i) {
          const float v = A8[(n8 + i) & rm[4]];
          acc += (i < lw - 1) ? v : 0.0f;
        }
        const int last = (n8 + lw - 1) & rm[4];
        const int n = (ar >> lj) + lb;
        ring_put(RTAB[3 * lj], RTAB[3 * lj + 2], n, acc + A8[last]);
        ring_put(RTAB[3 * lj + 1], RTAB[3 * lj + 2], n, acc + R8[last]);
      }
      __syncwarp();
    }
    if (ar >= srel || !cj) return;
    const int n = cn - ((k * kC) >> cj);
    float cv;
    auto run = [&](const auto* sc) {
      if (cj > KAP) {
        cv = bd_coarse_eval<K, true, false>(smem + ca + (n & cmask), smem + cr + (n & cmask), sc, cnu);
      } else if (K == 32 && cj == 4) {  // c_4 / 16 = K - 2 blocks: window starts one block early
        cv = bd_coarse_eval<K, false, true>(smem + ca + ((n - 1) & cmask), nullptr, sc, cnu);
      } else {
        cv = bd_coarse_eval<K, false, false>(smem + ca + (n & cmask), nullptr, sc, cnu);
      }
    };
    if constexpr (TABLE)
      run(static_cast<const float2*>(AB + cfirst));
    else
      run(static_cast<const float*>(STAB + cj * (K + 1) + 1));
    // a position with no valid candidate (every sum -inf) gives NaN: -inf instead
    const float bv = cv == cv ? dec_v<5>(cv) : ninf();
    RESY[(k & 1) * kResN + t] = bv;
    RESW[(k & 1) * kResN + t] = (uint16_t)(cfirst + dec_w<5>(cv));
    atomicMax(BCM + (k & 1) * kBcm + cbcm, (fkey(bv) & ~15) | ccode);
  };

  // ---- fine levels 0..3, merge and store of chunk k --------------------------
  float tmax = ninf();
  // candidate scale of block count m at fine level I (white: 1/sqrt(c_I + m 2^I);
  // table: the width's (a, b))
  auto scl = [&](auto I) {
    return [&](auto M) {
      constexpr int i = decltype(I)::value, m = decltype(M)::value;
      if constexpr (TABLE)
        return AB[p.lvl_first[i] + m - 1];
      else
        return p.bscale[i][m];
    };
  };
  const auto sc0 = scl(std::integral_constant<int, 0>{});
  const auto sc1 = scl(std::integral_constant<int, 1>{});
  const auto sc2 = scl(std::integral_constant<int, 2>{});
  const auto sc3 = scl(std::integral_constant<int, 3>{});
  auto fine = [&](int k) {
    const int ar = a0 - k * kC;
    if (ar >= srel) return;
    const int buf = k % S::NBUF;
    float y[8], f0[8];
    int w[8];
    // every level's maximum is coded with its rank (eval_bd_enc); a level is
    // decoded once per position and merged with the levels below by a strict '>'
    // (the smaller width wins a tie)
    auto merge_coded = [&](float& yv, int& wv, float c, int first) {
      merge1(yv, wv, dec_v<5>(c), first + dec_w<5>(c));
    };
    {
      float win[S::NW0 * 4], o[8];
      load_window4<S::NW0>(smem + S::f0(buf) + 8 * t, win);
      if (!COARSE && top == 0)
        eval_bd_enc<8, K, false, true>(win, nullptr, p.n_top, sc0, o, f0);
      else
        eval_bd_enc<8, K, false, false>(win, nullptr, p.n_top, sc0, o, f0);
#pragma unroll
      for (int r = 0; r < 8; ++r) {  // level 0 starts at width index 0
        y[r] = dec_v<5>(o[r]);
        w[r] = dec_w<5>(o[r]);
      }
    }
    float f1[4], f2[2];
    if (COARSE || top >= 1) {
      float win[S::NW1 * 4], o[4];
      const float b[4] = {f0[0], f0[2], f0[4], f0[6]};
      load_window4<S::NW1>(smem + S::f1(buf) + 4 * t + S::OF1, win);
      if (!COARSE && top == 1)
        eval_bd_enc<4, K, true, true>(win, b, p.n_top, sc1, o, f1);
      else
        eval_bd_enc<4, K, true, false>(win, b, p.n_top, sc1, o, f1);
      const int first = p.lvl_first[1];
#pragma unroll
      for (int r = 0; r < 4; ++r) merge_coded(y[2 * r], w[2 * r], o[r], first);
    }
    if (COARSE || top >= 2) {
      float win[S::NW2 * 2], o[2];
      const float b[2] = {f1[0], f1[2]};
      load_window2<S::NW2>(smem + S::f2(buf) + 2 * t + S::OF2, win);
      if (!COARSE && top == 2)
        eval_bd_enc<2, K, true, true>(win, b, p.n_top, sc2, o, f2);
      else
        eval_bd_enc<2, K, true, false>(win, b, p.n_top, sc2, o, f2);
      const int first = p.lvl_first[2];
      merge_coded(y[0], w[0], o[0], first);
      merge_coded(y[4], w[4], o[1], first);
    }
    if (COARSE || top >= 3) {
      float win[S::NW3], o[1], f3[1];
      const float b[1] = {f2[0]};
      load_window1<S::NW3>(smem + S::f3(buf) + t + S::OF3, win);
      if (!COARSE && top == 3)
        eval_bd_enc<1, K, true, true>(win, b, p.n_top, sc3, o, f3);
      else
        eval_bd_enc<1, K, true, false>(win, b, p.n_top, sc3, o, f3);
      merge_coded(y[0], w[0], o[0], p.lvl_first[3]);
    }
    if (COARSE) {  // best coarse level at start 8t (even t: 8t = 0 mod 16)
      int* kp = BCM + (k & 1) * kBcm + (t >> 1);
      const int key = *kp;
      *kp = INT_MIN;
      const int lvl = min(kRing0 + 15 - (key & 15), kChunkLog);  // no key: any level, unused
      const int slot = kThreads - (1 << (kChunkLog + 1 - lvl)) + (t >> (lvl - 3));
      const bool use = !(t & 1) && key != INT_MIN;
      const float yv = RESY[(k & 1) * kResN + (use ? slot : 0)];
      const int wv = RESW[(k & 1) * kResN + (use ? slot : 0)];
      const bool take = use && yv > y[0];
      y[0] = take ? yv : y[0];
      w[0] = take ? wv : w[0];
    }
    const int s0 = ar + 8 * t;
    if (s0 + 8 <= srel) {
#pragma unroll
      for (int r = 0; r < 8; ++r) tmax = fmaxf(tmax, y[r]);
    } else {
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (s0 + r < srel) tmax = fmaxf(tmax, y[r]);
    }
    store8(yseg, wseg, s0, srel, vec, y, w);
    if ((ar & (kCandTile - 1)) == 0) {
      tile_max_atomic(U.tm_row, t0 + ar, tmax);
      tmax = ninf();
    }
  };

  // ---- pipeline --------------------------------------------------------------
  Raw8 nx = load_raw8(xseg, a0 + 8 * t, nrel, dt, vx);
  {
    const Raw8 cx = nx;
    if (nch > 1) nx = load_raw8(xseg, a0 - kC + 8 * t, nrel, dt, vx);
    build(0, cx);
  }
  __syncthreads();
  if (COARSE) coarse(0);
  for (int k = 0; k < nch; ++k) {
    const bool more = k + 1 < nch;
    if (more) {
      const Raw8 cx = nx;
      if (k + 2 < nch) nx = load_raw8(xseg, a0 - (k + 2) * kC + 8 * t, nrel, dt, vx);
      build(k + 1, cx);
    }
    __syncthreads();
    if (COARSE && more) coarse(k + 1);
    fine(k);
  }
}

// One CTA per unit of a single-series search.
template <int K, bool COARSE, bool TABLE>
__global__ void __launch_bounds__(kThreads, (TABLE && K == 32) ? 1 : 2) boxdit_stream_kernel(const SearchParams p) {
  extern __shared__ __align__(16) float smem[];
  boxdit_unit<K, COARSE, TABLE>(p, plan_unit(p, blockIdx.x), smem);
}

// Batched search: persistent CTAs stride over the units of every range.
template <int K, bool COARSE>
__global__ void __launch_bounds__(kThreads, 2) boxdit_batch_kernel(const SearchParams p) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int flag;
  for (int64_t u = blockIdx.x; u < p.n_units; u += gridDim.x) {
    Unit U;
    if (!batch_unit(p, u, U, &flag)) continue;
    boxdit_unit<K, COARSE, false>(p, U, smem);
    __syncthreads();
  }
}

template <int K>
size_t bd_smem(int top, int nab) {
  return sizeof(float) * (size_t)BdDyn<K>(top, nab).total;
}

template <int K, bool TABLE>
cudaError_t launch_bd(const spd_plan& plan, const SearchParams& p, size_t smem, cudaStream_t s) {
  const int64_t nblk = plan.desc.ndm * plan.tiles_per_row;
  return plan.top >= kRing0 ? launch_one(boxdit_stream_kernel<K, true, TABLE>, smem, nblk, p, s)
                            : launch_one(boxdit_stream_kernel<K, false, TABLE>, smem, nblk, p, s);
}

}  // namespace

size_t boxdit_smem_bytes(const spd_plan& plan, bool table) {
  if (plan.bd_general) return boxdit_gen_smem_bytes(plan, table);
  const int nab = table ? (int)plan.widths.size() : 0;
  switch (plan.k) {
    case 8: return bd_smem<8>(plan.top, nab);
    case 16: return bd_smem<16>(plan.top, nab);
    case 32: return bd_smem<32>(plan.top, nab);
    default: return 0;
  }
}

namespace {
// Persistent launch: as many CTAs as fit on the device at once (at most one per unit).
template <class KernelT>
cudaError_t launch_persistent(KernelT kern, size_t smem, int64_t units, const SearchParams& p,
                              cudaStream_t s) {
  int per_sm = 0, sms = 0;
  const cudaError_t e = persistent_config(reinterpret_cast<const void*>(kern), smem, &per_sm, &sms);
  if (e != cudaSuccess) return e;
  if (p.ctas_per_sm > 0 && per_sm > p.ctas_per_sm) per_sm = p.ctas_per_sm;
  int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  if (grid > units) grid = units;
  kern<<<(unsigned)grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_boxdit_batch(const spd_plan& plan, const SearchParams& p, cudaStream_t s) {
  if (plan.bd_general) return launch_boxdit_gen_batch(plan, p, s);
  const size_t smem = boxdit_smem_bytes(plan, false);
  const bool coarse = plan.top >= kRing0;
  switch (plan.k) {
    case 8:
      return coarse ? launch_persistent(boxdit_batch_kernel<8, true>, smem, p.n_units, p, s)
                    : launch_persistent(boxdit_batch_kernel<8, false>, smem, p.n_units, p, s);
    case 16:
      return coarse ? launch_persistent(boxdit_batch_kernel<16, true>, smem, p.n_units, p, s)
                    : launch_persistent(boxdit_batch_kernel<16, false>, smem, p.n_units, p, s);
    case 32:
      return coarse ? launch_persistent(boxdit_batch_kernel<32, true>, smem, p.n_units, p, s)
                    : launch_persistent(boxdit_batch_kernel<32, false>, smem, p.n_units, p, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_boxdit(const spd_plan& plan, const SearchParams& p, cudaStream_t s) {
  if (plan.bd_general) return launch_boxdit_gen(plan, p, s);
  const bool table = p.table != 0;
  const size_t smem = boxdit_smem_bytes(plan, table);
  switch (plan.k) {
    case 8: return table ? launch_bd<8, true>(plan, p, smem, s) : launch_bd<8, false>(plan, p, smem, s);
    case 16: return table ? launch_bd<16, true>(plan, p, smem, s) : launch_bd<16, false>(plan, p, smem, s);
    case 32: return table ? launch_bd<32, true>(plan, p, smem, s) : launch_bd<32, false>(plan, p, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace spd
