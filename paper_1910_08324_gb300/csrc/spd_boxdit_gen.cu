// spd_boxdit_gen.cu -- BoxDIT with any even L^i_max, per iteration (Sec. 3.1,
// Alg. 1): the general kernel behind plans whose maximum widths are not one
// of 8, 16, 32 for every iteration (spd_boxdit.cu streams those).
//
// Iteration i (level i) has unit 2^i, starts s = n 2^i and the widths
// c_i + m 2^i, m = 1..k_i, with c_i = sum_{j<i} k_j 2^j (= L^{i-1}_MAX).  The
// kernel runs Alg. 1 as the paper states it, on one tile of T starts of one
// row (T = 4096 when the layout allows several CTAs per SM, else 2048;
// spd_plan_set_segment picks 2048, 4096 or 8192):
//   * the shifted decimated series x^i of the tile live in shared memory:
//     x^0 over the tile and its level-0 lookahead, x^1 summed in pairs
//     (x^1[u] = x^0[2u + k_0] + x^0[2u + k_0 + 1], the decimation of Sec. 3.1
//     with its shift of L^0_max / D: from x^0's window where it reaches, past it
//     straight from the input, 8 loads in flight per thread), and each x^{i+1}
//     from x^i in shared memory (x^{i+1}[u] = x^i[2u + k_i] + x^i[2u + k_i + 1]),
//     every series as long as the levels above still need it;
//   * level i evaluates its T / 2^i positions.  With 2, 4 or 8 or more per
//     thread, a thread takes tasks of 2, 4 or 8 consecutive positions and runs
//     them together on register windows of 8 or 4 block counts, each candidate
//     coded with its rank in the window (bdg_task); with fewer, one position
//     per thread, consecutive positions on consecutive lanes.  Either way the
//     sum starts from the base X^{i-1} at the position (kept by level i - 1)
//     and adds x^i[n], x^i[n + 1], ... in order, each partial sum times the
//     width's scale (a shared-memory table) being a candidate (strict '>', so
//     the smaller width wins a tie); the full sum of k_i blocks at an even
//     position is the next level's base;
//   * each level writes its best SNR and width index per position into an
//     array of its own in shared memory (level 0's over the tile's starts, the
//     others over x^0's buffer, dead by then), one barrier per level; the tile
//     store merges the levels at each start (increasing width order, strict
//     '>'), stores with vector stores, and folds the maximum into the
//     candidate-tile key.
// Plans above level kBdgSplit (4) run in two kernels.  The first takes levels
// 0-3 on the tiles above (three CTAs per SM) and also writes x^4, the level-3
// bases of its positions (X^3 at even positions) and a copy of its SNR and width
// at every 16th start to the workspace; the second takes levels 4.. on tiles of
// kBdgTile2 positions of x^4 (a level-4 position is 16 starts), starting from
// those bases and that copy, and rewrites a start only where a wider level won
// (strided stores touch partial sectors, so the fewer the better).  The levels
// above 3 then see tiles of 32768 starts, so their halo (the widest boxcar) is
// read 16 times less often and their positions fill the CTA.
// The series past the tile (the halo, up to the widest boxcar) are re-read by
// the neighbouring tiles' CTAs; the widest boxcar of a plan is at most 32768
// samples.  Samples past the end of the row are -inf, so a boxcar needing them
// never wins (the s + L <= nt rule); starts at or past the plan's n_starts are
// not stored.
#include <memory>

#include "spd_common.cuh"

namespace spd {

constexpr int kWinPad = 32;  // floats after each series buffer (see bdg_layout)

// Offset in the YC, WC regions of level i >= 1's P(i) results (P(i) = T / 2^i
// up to level lt = log2 T, then 1): the levels one after the other from level 1.
__host__ __device__ __forceinline__ int yc_off(int T, int lt, int i) {
  return i - 1 <= lt ? T - (T >> (i - 1)) : T - 1 + (i - 1 - lt);
}

// Window lengths and shared-memory offsets (floats) of a general BoxDIT plan
// with tiles of T starts (see the kernel's comment).
int bdg_layout(const spd_plan& plan, int T, bool table, int32_t* len, int32_t* off, int part, int h) {
  int lt = 0;
  while ((2 << lt) <= T) ++lt;  // log2 T
  auto P = [&](int i) { return i <= lt ? T >> i : 1; };
  const int lo = part == 2 ? h : 0;                 // first plan level of this kernel
  const int top = part == 1 ? h : plan.top - lo;    // its last (part 1: x^h, written out)
  auto K = [&](int i) { return plan.lvl_k[i + lo]; };
  for (int i = 0; i < kMaxLevels; ++i) len[i] = 0;
  len[top] = part == 1 ? P(top) : P(top) + plan.n_top - 1;
  for (int i = top - 1; i >= 0; --i) {
    const int a = P(i) + K(i) - 1, b = 2 * len[i + 1] + K(i);
    len[i] = a > b ? a : b;
  }
  // level 0 keeps only its own window: x^1 is summed straight from the input
  len[0] = T + (top == 0 ? plan.n_top : K(0)) - 1;
  int ma = 0, mb = 0;
  for (int i = 1; i <= top; ++i) {
    if (i & 1)
      ma = ma > len[i] + 1 ? ma : len[i] + 1;
    else
      mb = mb > len[i] + 1 ? mb : len[i] + 1;
  }
  // each series buffer is padded: a task's last register window may read up to
  // kGMC - 1 values past the series (never used)
  int o = 0;
  off[kBdgX0] = o;
  o += al4(len[0]) + kWinPad;
  off[kBdgXA] = o;
  o += al4(ma) + kWinPad;
  off[kBdgXB] = o;
  o += al4(mb) + kWinPad;
  off[kBdgBA] = o;
  o += al4(T / 2);
  off[kBdgBB] = o;
  o += al4(part == 2 ? T : T / 4);  // part 2: the bases of its level 0 (X^{h-1}) come in here
  off[kBdgY] = o;  // level 0's results
  o += T;
  off[kBdgW] = o;
  o += T / 2;
  const int nyc = yc_off(T, lt, (part == 1 ? h - 1 : top) + 1);  // levels 1.. (part 1: up to h - 1)
  if (nyc <= al4(len[0]) + kWinPad) {
    off[kBdgYC] = off[kBdgX0];  // x^0 is dead once level 0 is done
  } else {
    off[kBdgYC] = o;
    o += al4(nyc);
  }
  off[kBdgWC] = o;
  o += al4((nyc + 1) / 2);
  off[kBdgAB] = o;  // table noise: (a, b) per width; white noise: 1/sqrt(L) per width
  o += table ? al4(2 * ((int)plan.widths.size() + kAbPad)) : al4((int)plan.widths.size());
  return o;
}

namespace {

constexpr int kGMC = 8;        // block counts per register window at most (3-bit ranks)
constexpr int kLoadBatch = 8;  // input loads in flight per thread

// NP consecutive values at a 4 NP-byte aligned address (float4 or float2 loads)
template <int N, int NP>
__device__ __forceinline__ void load_run(const float* src, float (&w)[N]) {
  if constexpr (NP % 4 == 0) {
    static_assert(N % 4 == 0, "whole float4s");
    load_window4<N / 4>(src, w);
  } else {
    static_assert(N % 2 == 0, "whole float2s");
    load_window2<N / 2>(src, w);
  }
}

// One window of G (8 or 4) block counts m0.. of a task (see bdg_task); FULL:
// every count of the window is summed and a candidate (no per-count tests).
template <bool TABLE, int NP, bool FULL, int G>
__device__ __forceinline__ void bdg_window(const float* __restrict__ Xi, const float* __restrict__ SC, int n0,
                                           int m0, int first, int nu, int mend, float (&S)[NP], float (&bv)[NP],
                                           int (&bq)[NP]) {
  static_assert(G <= kGMC && G % 2 == 0, "ranks in 3 bits, taken in pairs");
  constexpr int NW = NP + G;  // NP + G - 1 values used
  float w[NW];
  load_run<NW, NP>(Xi + n0 + m0, w);
  float acc[NP], c[NP];  // c: the candidate of the previous (even) rank, for a three-input max
#pragma unroll
  for (int r = 0; r < NP; ++r) acc[r] = ninf();
  static_for<0, G>([&](auto J) {
    constexpr int j = decltype(J)::value;
    const int m = m0 + j;
    if (FULL || m < mend) {
      if constexpr ((j & 1) == 0) {  // aligned pairs of the window: packed f32x2 adds (the same roundings)
#pragma unroll
        for (int q = 0; q < NP / 2; ++q) {
          const float2 s2 = __fadd2_rn(make_float2(S[2 * q], S[2 * q + 1]), make_float2(w[2 * q + j], w[2 * q + j + 1]));
          S[2 * q] = s2.x;
          S[2 * q + 1] = s2.y;
        }
      } else {
#pragma unroll
        for (int r = 0; r < NP; ++r) S[r] += w[r + j];
      }
    }
    if (FULL || m < nu) {  // (nu <= mend)
      float x[NP];
      if constexpr (TABLE) {
        const float2 ab = reinterpret_cast<const float2*>(SC)[first + m];
#pragma unroll
        for (int r = 0; r < NP; ++r) x[r] = fmaf(S[r], ab.x, ab.y);
      } else {
        const float sc = SC[first + m];
#pragma unroll
        for (int q = 0; q < NP / 2; ++q) {  // two positions per scale instruction (packed f32x2)
          const float2 x2 = __fmul2_rn(make_float2(S[2 * q], S[2 * q + 1]), make_float2(sc, sc));
          x[2 * q] = x2.x;
          x[2 * q + 1] = x2.y;
        }
      }
#pragma unroll
      for (int r = 0; r < NP; ++r) {
        const float e = enc_w<3>(x[r], (kGMC - 1) - j);
        if constexpr ((j & 1) == 0)
          c[r] = e;
        else
          acc[r] = fmax3(acc[r], c[r], e);
      }
    } else {
#pragma unroll
      for (int r = 0; r < NP; ++r) {
        if constexpr ((j & 1) == 0)
          c[r] = ninf();
        else
          acc[r] = fmaxf(acc[r], c[r]);
      }
    }
  });
  static_assert(kGMC % 2 == 0, "ranks are taken in pairs");
#pragma unroll
  for (int r = 0; r < NP; ++r) {  // a NaN (no candidate in the window) never passes '>'
    const float v = dec_v<3>(acc[r]);
    const bool take = v > bv[r];
    bv[r] = take ? v : bv[r];
    bq[r] = take ? m0 + dec_w<3>(acc[r]) : bq[r];
  }
}

// Level i at the NP consecutive positions n0.. of a task (n0 a multiple of NP):
// running sums from the base (level 0 of the row: none), every partial sum
// times its width's scale a candidate.  The block counts go in windows of G = 8
// or 4 (bdg_window): a window's NP + G - 1 values come in with vector loads,
// each candidate carries its rank in the window in the 3 low mantissa bits
// (enc_w, smaller rank wins a tie) and the window's maximum is kept running
// with three-input max instructions; at the end of a window it is decoded and
// taken when strictly larger than the best of the earlier windows.  Windows of
// 8, then one of 4, take counts that are all candidates, without per-count
// tests; the rest go in windows of 4 with tests.  S[] ends as the sum of mend
// blocks (the next level's base); bv[], bq[] are the best SNR and its block
// count - 1.  SC: the widths' scales (white noise) or (a, b) pairs.
template <bool TABLE, bool BASE, int NP>
__device__ __forceinline__ void bdg_task(const float* __restrict__ Xi, const float* __restrict__ Bi,
                                         const float* __restrict__ SC, int n0, int first, int nu, int mend,
                                         float (&S)[NP], float (&bv)[NP], int (&bq)[NP]) {
  if constexpr (BASE) {
    load_run<NP, NP>(Bi + n0, S);
  } else {
#pragma unroll
    for (int r = 0; r < NP; ++r) S[r] = 0.0f;
  }
#pragma unroll
  for (int r = 0; r < NP; ++r) {
    bv[r] = ninf();
    bq[r] = 0;
  }
  // windows of 8 candidates, one of 4, then windows of 4 with tests
  int m0 = 0;
  for (; m0 + 8 <= nu; m0 += 8) bdg_window<TABLE, NP, true, 8>(Xi, SC, n0, m0, first, nu, mend, S, bv, bq);
  if (m0 + 4 <= nu) {
    bdg_window<TABLE, NP, true, 4>(Xi, SC, n0, m0, first, nu, mend, S, bv, bq);
    m0 += 4;
  }
  for (; m0 < mend; m0 += 4) bdg_window<TABLE, NP, false, 4>(Xi, SC, n0, m0, first, nu, mend, S, bv, bq);
}

// All tasks of NP positions of level i (every thread takes P / (NP kThreads)):
// the bases of level i + 1 (next) and the level's best SNR and width index at
// each of its P positions, into Yo, Wo (base: the sums start from the bases Bi;
// merge: Yo, Wo already hold results of smaller widths, replaced only where
// strictly exceeded).
template <bool TABLE, int NP>
__device__ __forceinline__ void bdg_level(int P, bool next, bool base, bool merge, const float* Xi, const float* Bi,
                                          float* Bn, const float* SC, int first, int nu, int mend, float* Yo,
                                          uint16_t* Wo) {
  for (int n0 = NP * (int)threadIdx.x; n0 < P; n0 += NP * kThreads) {
    float S[NP], bv[NP];
    int bq[NP];
    if (!base)
      bdg_task<TABLE, false, NP>(Xi, Bi, SC, n0, first, nu, mend, S, bv, bq);
    else
      bdg_task<TABLE, true, NP>(Xi, Bi, SC, n0, first, nu, mend, S, bv, bq);
#pragma unroll
    for (int r = 0; r < NP; ++r) bq[r] += first;
    if (merge) {  // keep the SNRs already there unless strictly exceeded (they have the smaller widths)
      float yo[NP];
      load_run<NP, NP>(Yo + n0, yo);
#pragma unroll
      for (int r = 0; r < NP; ++r) {
        const bool keep = !(bv[r] > yo[r]);
        bv[r] = keep ? yo[r] : bv[r];
        bq[r] = keep ? (int)Wo[n0 + r] : bq[r];
      }
    }
    uint32_t pk[NP / 2];
#pragma unroll
    for (int r = 0; r < NP / 2; ++r) pk[r] = (uint32_t)bq[2 * r] | ((uint32_t)bq[2 * r + 1] << 16);
    if constexpr (NP == 8) {
      if (next) *reinterpret_cast<float4*>(Bn + (n0 >> 1)) = make_float4(S[0], S[2], S[4], S[6]);
      *reinterpret_cast<float4*>(Yo + n0) = make_float4(bv[0], bv[1], bv[2], bv[3]);
      *reinterpret_cast<float4*>(Yo + n0 + 4) = make_float4(bv[4 % NP], bv[5 % NP], bv[6 % NP], bv[7 % NP]);
      *reinterpret_cast<uint4*>(Wo + n0) = make_uint4(pk[0], pk[1 % (NP / 2)], pk[2 % (NP / 2)], pk[3 % (NP / 2)]);
    } else if constexpr (NP == 4) {
      if (next) *reinterpret_cast<float2*>(Bn + (n0 >> 1)) = make_float2(S[0], S[2 % NP]);
      *reinterpret_cast<float4*>(Yo + n0) = make_float4(bv[0], bv[1], bv[2 % NP], bv[3 % NP]);
      *reinterpret_cast<uint2*>(Wo + n0) = make_uint2(pk[0], pk[1 % (NP / 2)]);
    } else {
      if (next) Bn[n0 >> 1] = S[0];
      *reinterpret_cast<float2*>(Yo + n0) = make_float2(bv[0], bv[1 % NP]);
      *reinterpret_cast<uint32_t*>(Wo + n0) = pk[0];
    }
  }
}

// x^1[u] for u < x1_split comes from x^0's window in shared memory (its pairs
// 2u + k_0, 2u + k_0 + 1 lie below T + k_0 - 1), the rest from the input; even,
// so the input part starts on a whole pair of pairs.
__device__ __forceinline__ int x1_split(int T, int n1) {
  const int u = T / 2 - 2;
  return u < n1 ? u : (n1 & ~1);
}

// One tile.  PART 0: every level of the plan on T starts of the input; PART 1:
// levels 0..h-1 on T starts, and x^h, the bases X^{h-1} and a copy of the
// results of the tile's T / 2^h level-h positions to the workspace; PART 2:
// levels h..top on T positions of x^h (t0 and T in level-h positions), stored
// at the starts where they beat the first part's copy.
template <bool TABLE, int PART>
__device__ __forceinline__ void bdg_unit(const SearchParams& p, const Unit& U, float* smem) {
  constexpr bool P1 = PART == 1, P2 = PART == 2;
  const int t = threadIdx.x;
  const int T = U.T;
  const int64_t t0 = U.t0;
  const int dt = p.dtype;
  const int h = p.gen_h;
  const int lo = P2 ? h : 0;  // the plan level of this tile's level 0
  // scales of the widths in shared memory: (a, b) pairs of table noise, or
  // 1/sqrt(L) of white noise
  float* SC = smem + p.gen_off[kBdgAB];
  float mu, inv;
  row_noise<TABLE>(p, U.mu, U.sigma, U.row, reinterpret_cast<float2*>(SC), mu, inv);
  if constexpr (!TABLE)
    for (int w = t; w < p.n_widths; w += kThreads) SC[w] = p.wscale[w];
  float* X0 = smem + p.gen_off[kBdgX0];
  float* XA = smem + p.gen_off[kBdgXA];
  float* XB = smem + p.gen_off[kBdgXB];
  float* BA = smem + p.gen_off[kBdgBA];
  float* BB = smem + p.gen_off[kBdgBB];
  // level 0's best SNR and width index at each of its T positions; levels 1..
  // in YC, WC, level i at offset yc_off(i)
  float* Y = smem + p.gen_off[kBdgY];
  uint16_t* W = reinterpret_cast<uint16_t*>(smem + p.gen_off[kBdgW]);
  float* YC = smem + p.gen_off[kBdgYC];
  uint16_t* WC = reinterpret_cast<uint16_t*>(smem + p.gen_off[kBdgWC]);
  int lt = 0;
  while ((2 << lt) <= T) ++lt;
  // levels with positions in this tile: a level of unit 2^i > T has one, at t0,
  // when 2^i divides t0 (and then so does every lower unit)
  int tt = P1 ? h - 1 : p.top - lo;
  while (tt > lt && (t0 & ((1LL << tt) - 1)) != 0) --tt;
  const float* xh = P2 ? p.gen_xh + U.row * p.gen_ldh : nullptr;
  const int64_t nxh = p.gen_ldh;  // positions of x^h per row (past them: -inf)

  // ---- x^0 over the tile's level-0 window, x^1 in pairs from the input ----
  {
    const int nq0 = (p.gen_len[0] + 3) / 4;  // quads of x^0
    const int k0 = p.lvl_k[lo], n1 = p.gen_len[1];
    const int q1 = tt >= 1 ? x1_split(T, n1) >> 1 : 0;                // first quad of x^1 from the input
    const int nq1 = tt >= 1 ? (n1 + 1) / 2 - q1 : 0;                   // ... and their number
    const bool v1 = U.vec_x && (k0 & 3) == 0;
    // one index space over both: quad j < nq0 of x^0, else quad q1 + j - nq0 of x^1's input;
    // kLoadBatch loads per thread are issued before any is used
    const int nq = nq0 + nq1;
    for (int j0 = t; j0 < nq; j0 += kLoadBatch * kThreads) {
      float4 v[kLoadBatch];
#pragma unroll
      for (int b = 0; b < kLoadBatch; ++b) {
        const int j = j0 + b * kThreads;
        const bool is0 = j < nq0;
        const int64_t pos = is0 ? t0 + 4 * j : t0 + k0 + 4 * (q1 + j - nq0);
        if constexpr (P2) {  // the series x^h of the first part (sums of normalised samples)
          // rows of nxh positions, nxh and t0 multiples of 4, k0 even
          const float4 ninf4 = make_float4(ninf(), ninf(), ninf(), ninf());
          if (is0) {
            v[b] = pos < nxh ? __ldg(reinterpret_cast<const float4*>(xh + pos)) : ninf4;
          } else if (j < nq) {
            const float2 a = pos < nxh ? __ldg(reinterpret_cast<const float2*>(xh + pos)) : make_float2(ninf(), ninf());
            const float2 c = pos + 2 < nxh ? __ldg(reinterpret_cast<const float2*>(xh + pos + 2))
                                           : make_float2(ninf(), ninf());
            v[b] = make_float4(a.x, a.y, c.x, c.y);
          } else {
            v[b] = make_float4(0, 0, 0, 0);
          }
        } else
          v[b] = j < nq ? load_z4d(U.xrow, pos, U.nt, dt, is0 ? U.vec_x : v1, mu, inv) : make_float4(0, 0, 0, 0);
      }
#pragma unroll
      for (int b = 0; b < kLoadBatch; ++b) {
        const int j = j0 + b * kThreads;
        if (j < nq0)
          *reinterpret_cast<float4*>(X0 + 4 * j) = v[b];
        else if (j < nq)
          *reinterpret_cast<float2*>(XA + 2 * (q1 + j - nq0)) = make_float2(v[b].x + v[b].y, v[b].z + v[b].w);
      }
    }
    if constexpr (P2) {  // the bases of level h, and the SNRs and widths the first part stored at its starts
      const float* bh = p.gen_bh + U.row * p.gen_ldh;
      for (int n = 4 * t; n < T; n += 4 * kThreads) {  // (nxh and t0 multiples of 4)
        const int64_t v = t0 + n;
        *reinterpret_cast<float4*>(BB + n) =
            v < nxh ? __ldg(reinterpret_cast<const float4*>(bh + v)) : make_float4(0, 0, 0, 0);
      }
      const float* yh = p.gen_yh + U.row * p.gen_ldh;  // (copies of the first part's, coalesced)
      const uint16_t* wh = p.gen_wh + U.row * p.gen_ldh;
      for (int n = t; n < T; n += kThreads) {
        const int64_t v = t0 + n;
        const bool in = (v << h) < U.ns;
        Y[n] = in ? yh[v] : ninf();
        W[n] = in ? wh[v] : (uint16_t)0;
      }
    }
  }
  __syncthreads();

  // ---- levels 0..tt: evaluate, decimate; one barrier per level ----
  for (int i = 0; i <= tt; ++i) {
    const int P = i <= lt ? T >> i : 1;
    const int k = p.lvl_k[i + lo];
    const int nu = (i + lo == p.top) ? p.n_top : k;  // block counts that are candidates
    const bool next = i < tt || P1;                  // a next level (part 1: level h) needs the bases
    const int mend = next ? k : nu;                  // blocks summed (the next level needs all k)
    const int first = p.lvl_first[i + lo];
    const bool base = i > 0 || P2;
    const float* Xi = (i == 0) ? X0 : ((i & 1) ? XA : XB);
    const float* Bi = (i & 1) ? BA : BB;
    float* Bn = (i & 1) ? BB : BA;
    const int yo = yc_off(T, lt, i);
    float* Yo = i == 0 ? Y : YC + yo;
    uint16_t* Wo = i == 0 ? W : WC + yo;
    const int per = P / kThreads;  // positions per thread (P and kThreads are powers of two)
    const bool merge = P2 && i == 0;  // merged into the stored SNRs of the first part
    if (per >= 8) {
      bdg_level<TABLE, 8>(P, next, base, merge, Xi, Bi, Bn, SC, first, nu, mend, Yo, Wo);
    } else if (per == 4) {
      bdg_level<TABLE, 4>(P, next, base, merge, Xi, Bi, Bn, SC, first, nu, mend, Yo, Wo);
    } else if (per == 2) {
      bdg_level<TABLE, 2>(P, next, base, merge, Xi, Bi, Bn, SC, first, nu, mend, Yo, Wo);
    } else for (int n = t; n < P; n += kThreads) {  // at most one position per thread
      float S = base ? Bi[n] : 0.0f;
      float best = ninf();
      int bq = 0;
      const float* xs = Xi + n;
      int m = 0;
#pragma unroll 4
      for (; m < nu; ++m) {
        S += xs[m];
        float v;
        if constexpr (TABLE) {
          const float2 ab = reinterpret_cast<const float2*>(SC)[first + m];
          v = fmaf(S, ab.x, ab.y);
        } else {
          v = S * SC[first + m];
        }
        if (v > best) {
          best = v;
          bq = m;
        }
      }
      for (; m < mend; ++m) S += xs[m];
      if (next && (n & 1) == 0) Bn[n >> 1] = S;
      if (!merge || best > Yo[n]) {
        Yo[n] = best;
        Wo[n] = (uint16_t)(first + bq);
      }
    }
    if (i == 0 && tt >= 1) {  // x^1[u] for u below the split, from x^0's window
      const int u1 = x1_split(T, p.gen_len[1]);
      for (int u = t; u < u1; u += kThreads) {
        const float2 v = *reinterpret_cast<const float2*>(X0 + 2 * u + k);  // k even: aligned pair
        XA[u] = v.x + v.y;
      }
    }
    if (i >= 1 && next) {  // x^{i+1} from x^i, shifted by k_i (Sec. 3.1's decimation)
      float* Xn = (i & 1) ? XB : XA;
      const int nn = p.gen_len[i + 1];
      for (int u = t; u < nn; u += kThreads) {
        const float2 v = *reinterpret_cast<const float2*>(Xi + 2 * u + k);  // k even: aligned pair
        Xn[u] = v.x + v.y;
      }
    }
    __syncthreads();
  }

  if constexpr (P1) {  // x^h and the bases of the tile's level-h positions, for the second part
    const float* Xh = ((h - 1) & 1) ? XB : XA;
    const float* Bh = ((h - 1) & 1) ? BB : BA;
    const int64_t v0 = t0 >> h;
    float* xo = p.gen_xh + U.row * p.gen_ldh + v0;
    float* bo = p.gen_bh + U.row * p.gen_ldh + v0;
    for (int u = t; u < (T >> h); u += kThreads) {
      xo[u] = Xh[u];
      bo[u] = Bh[u];
    }
  }

  // merge of the levels above level 0 at local position n of level 0 (levels in
  // increasing width order, strict '>': the smaller width keeps a tie)
  auto merge_up = [&](int n, int i1, float& y, int& w) {
    for (int i = i1; i <= tt && (n & ((1 << i) - 1)) == 0; ++i) {
      const int o = yc_off(T, lt, i) + (n >> i);
      const float v = YC[o];
      if (v > y) {
        y = v;
        w = WC[o];
      }
    }
  };

  if constexpr (P2) {  // ---- store the starts of levels h..: strided, key per warp step ----
    // only where a level above h - 1 won: a different (wider) width than the
    // first part stored there (strided stores fill partial sectors)
    const uint16_t* wh = p.gen_wh + U.row * p.gen_ldh;
    const int warp = t >> 5, lane = t & 31;
    for (int n0 = 32 * warp; n0 < T; n0 += kThreads) {
      const int n = n0 + lane;
      const int64_t st = (t0 + n) << h;
      float y = Y[n];
      int w = W[n];
      merge_up(n, 1, y, w);
      if (st < U.ns && w != (int)wh[t0 + n]) {
        U.yrow[st] = y;
        U.wrow[st] = (uint16_t)w;
      }
      if (((t0 + n0) << h) < U.ns)  // warp-uniform: the warp's starts lie in one candidate tile
        tile_max_atomic(U.tm_row, (t0 + n0) << h, st < U.ns ? y : ninf());
    }
    return;
  }

  // ---- merge and store the tile; its maximum goes to the candidate-tile key ----
  const int64_t sleft = U.ns - t0;
  const int srel = (int)(sleft < (int64_t)T ? sleft : (int64_t)T);
  float tmax = ninf();
  for (int q = t; 4 * q < srel; q += kThreads) {
    const float4 y4 = *reinterpret_cast<const float4*>(Y + 4 * q);
    const uint2 w4 = *reinterpret_cast<const uint2*>(W + 4 * q);
    float y[4] = {y4.x, y4.y, y4.z, y4.w};
    int w[4] = {(int)(w4.x & 0xffffu), (int)(w4.x >> 16), (int)(w4.y & 0xffffu), (int)(w4.y >> 16)};
    if (tt >= 1) {  // level 1 at the starts 4q and 4q + 2, then levels 2.. at 4q
      const float2 y1 = *reinterpret_cast<const float2*>(YC + 2 * q);  // (level 1 at offset 0)
      const uint32_t w1 = *reinterpret_cast<const uint32_t*>(WC + 2 * q);
      if (y1.x > y[0]) {
        y[0] = y1.x;
        w[0] = (int)(w1 & 0xffffu);
      }
      if (y1.y > y[2]) {
        y[2] = y1.y;
        w[2] = (int)(w1 >> 16);
      }
      merge_up(4 * q, 2, y[0], w[0]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (4 * q + r < srel) tmax = fmaxf(tmax, y[r]);
    store4(U.yrow, U.wrow, t0 + 4 * q, U.ns, U.vec, y, w);
    if (P1 && ((4 * q) & ((1 << h) - 1)) == 0) {  // a start of level h: a copy for the second part
      const int64_t v = (t0 + 4 * q) >> h;
      p.gen_yh[U.row * p.gen_ldh + v] = y[0];
      p.gen_wh[U.row * p.gen_ldh + v] = (uint16_t)w[0];
    }
  }
  if (t0 < U.ns) tile_max_atomic(U.tm_row, t0, tmax);  // (the first part covers the row up to nt)
}

template <bool TABLE, int PART>
__global__ void __launch_bounds__(kThreads, PART == 0 ? 2 : 3) boxdit_gen_kernel(const SearchParams p) {
  extern __shared__ __align__(16) float smem[];
  bdg_unit<TABLE, PART>(p, plan_unit(p, blockIdx.x), smem);
}

// Batched search: persistent CTAs stride over the units of every range.
__global__ void __launch_bounds__(kThreads, 2) boxdit_gen_batch_kernel(const SearchParams p) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int flag;
  for (int64_t u = blockIdx.x; u < p.n_units; u += gridDim.x) {
    Unit U;
    if (!batch_unit(p, u, U, &flag)) continue;
    bdg_unit<false, 0>(p, U, smem);
    __syncthreads();
  }
}

}  // namespace

bool bdg_two_part(const spd_plan& plan) {
  if (plan.family != kBoxdit || !plan.bd_general || plan.top <= kBdgSplit) return false;
  int32_t len[kMaxLevels], off[kBdgOffsets];
  return sizeof(float) * (size_t)bdg_layout(plan, plan.tile, true, len, off, 1, kBdgSplit) <= kBdgMaxSmem &&
         sizeof(float) * (size_t)bdg_layout(plan, kBdgTile2, true, len, off, 2, kBdgSplit) <= kBdgMaxSmem;
}

size_t boxdit_gen_smem_bytes(const spd_plan& plan, bool table) {
  int32_t len[kMaxLevels], off[kBdgOffsets];
  return sizeof(float) * (size_t)bdg_layout(plan, plan.tile, table, len, off);
}

namespace {

template <int PART>
cudaError_t launch_gen_part(const SearchParams& p, size_t smem, int64_t nblk, cudaStream_t s) {
  return p.table ? launch_one(boxdit_gen_kernel<true, PART>, smem, nblk, p, s)
                 : launch_one(boxdit_gen_kernel<false, PART>, smem, nblk, p, s);
}

}  // namespace

cudaError_t launch_boxdit_gen(const spd_plan& plan, const SearchParams& p, cudaStream_t s) {
  const bool table = p.table != 0;
  if (!p.gen_xh || !bdg_two_part(plan))  // every level in one kernel
    return launch_gen_part<0>(p, boxdit_gen_smem_bytes(plan, table), plan.desc.ndm * plan.tiles_per_row, s);
  // two kernels: levels below h on tiles covering the row (x^h is needed up to
  // its end), then levels h..top on tiles of kBdgTile2 level-h positions
  const int h = kBdgSplit;
  std::unique_ptr<SearchParams> q(new (std::nothrow) SearchParams(p));
  if (!q) return cudaErrorMemoryAllocation;
  q->gen_h = h;
  const size_t smem1 = sizeof(float) * (size_t)bdg_layout(plan, plan.tile, table, q->gen_len, q->gen_off, 1, h);
  const int64_t tiles1 = (plan.desc.nt + plan.tile - 1) / plan.tile;
  q->tiles_per_row = (int32_t)tiles1;
  cudaError_t e = launch_gen_part<1>(*q, smem1, plan.desc.ndm * tiles1, s);
  if (e != cudaSuccess) return e;
  *q = p;
  q->gen_h = h;
  q->tile = kBdgTile2;
  const size_t smem2 = sizeof(float) * (size_t)bdg_layout(plan, kBdgTile2, table, q->gen_len, q->gen_off, 2, h);
  const int64_t nh = (plan.n_starts + (1 << h) - 1) >> h;  // level-h positions with a start
  const int64_t tiles2 = (nh + kBdgTile2 - 1) / kBdgTile2;
  q->tiles_per_row = (int32_t)tiles2;
  return launch_gen_part<2>(*q, smem2, plan.desc.ndm * tiles2, s);
}

cudaError_t launch_boxdit_gen_batch(const spd_plan& plan, const SearchParams& p, cudaStream_t s) {
  const size_t smem = boxdit_gen_smem_bytes(plan, false);
  int per_sm = 0, sms = 0;
  const cudaError_t e =
      persistent_config(reinterpret_cast<const void*>(boxdit_gen_batch_kernel), smem, &per_sm, &sms);
  if (e != cudaSuccess) return e;
  if (p.ctas_per_sm > 0 && per_sm > p.ctas_per_sm) per_sm = p.ctas_per_sm;
  int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  if (grid > p.n_units) grid = p.n_units;
  boxdit_gen_batch_kernel<<<(unsigned)grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace spd
