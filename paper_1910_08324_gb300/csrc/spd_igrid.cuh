// spd_igrid.cuh -- IGRID / DIT search kernel templates (Sec. 3.2, Alg. 3,
// Eq. boxcarsize, Table 1), instantiated by spd_igrid.cu (grids with more than
// 32 widths, batched searches) and spd_igrid_coded.cu (coded grids: at most 32
// widths, the width index carried in the SNRs' low mantissa bits).
//
// The IGRID grid, written as levels (spd_internal.h): level 0 holds steps
// 0..p (separation 1); level j >= 1 is step p + j, with unit 2^j and block
// counts m = 2^p + q 2^(p-d).  The P layers of a step are the P start phases of
// one block series, so the paper's binary tree of layers is one aligned block
// pyramid here.
//
// One CTA streams one segment of one DM row, 2048-sample chunks at a time,
// *backwards in time*: when chunk [a, a + 2048) is processed, every block a
// window starting in it can reach (up to L_end later) has already been seen.
// Each sample is therefore loaded, normalised and summed exactly once; the
// segment's first L_end samples past its end are its only re-read (the halo).
// The chunk loop is software pipelined with one barrier per chunk.  Iteration
// k (chunks counted in processing order):
//   build   chunk k+1's 8 samples per thread (prefetched into registers one
//           iteration earlier) are normalised and reduced in registers and
//           warp shuffles into levels 0..3 (shared, three buffers, each with a
//           lookahead tail copied from the chunk processed before it) and into
//           ring buffers for the coarse levels 4.. (unit >= 16); the loads of
//           chunk k+2 are issued;
//   barrier
//   coarse  chunk k+1's coarse positions: quads of 4 consecutive positions of
//           levels 4..8 (one float4 ring window each) on the first 62 threads,
//           single positions of levels 9..11 on the last warp (after it has
//           built those levels' blocks); each result is posted to a per-start
//           key with a shared atomic maximum;
//   fine    each thread owns 8 consecutive starts of chunk k and evaluates
//           levels 0..3 from register windows (8 + 4 + 2 + 1 positions),
//           merges them with the start's coarse key (computed one iteration
//           earlier) and writes 8 SNRs (2 x float4) and 8 widths.
// Grids of at most 32 widths carry the width index in the SNRs' low mantissa
// bits, so every maximum and merge is one max instruction; two starts share
// each add and scale instruction (packed f32x2).  The coarse evaluation of one
// chunk overlaps the fine evaluation of the previous one instead of sitting
// between two barriers.  Samples past the end of the row are -inf, so a boxcar
// needing them never wins (the s + L <= nt rule); starts at or past the plan's
// n_starts are neither evaluated nor stored.
#pragma once

#include <climits>

#include "spd_common.cuh"

namespace spd {
namespace {

constexpr int kC = kChunk;            // starts per chunk
constexpr int kSpt = kC / kThreads;   // starts per thread
static_assert(kSpt == 8, "the per-thread level layout assumes 8 starts per thread");
constexpr int kRing0 = 4;             // first coarse (ring) level
constexpr int kChunkLog = 11;         // log2(kC): levels above it span several chunks
static_assert((1 << kChunkLog) == kC, "chunk must be 2^11");
constexpr int kResHi = 256;           // RES slots of levels > kChunkLog start here
constexpr int kTailWarp = 2;          // the warp that copies the lookahead tails

template <int D, int PL>
struct IgS {
  using SM = IgM<D, PL>;
  using S0 = Ig0<D, PL>;
  static constexpr int MMAX = SM::MMAX;
  static constexpr int NW0 = cdiv(7 + MMAX, 4);  // float4 window of level 0 (starts 8t..8t+7)
  static constexpr int NW1 = cdiv(3 + MMAX, 4);  // float4 window of level 1 (4 positions)
  static constexpr int NW2 = cdiv(1 + MMAX, 2);  // float2 window of level 2 (2 positions)
  static constexpr int NW3 = MMAX;               // scalar window of level 3 (1 position)
  static constexpr int TL0 = 4 * NW0 - 8;        // lookahead tails (values past the chunk)
  // level 0 is stored as two arrays of 4-sample quads, even quads (A) and odd
  // quads (B), so that a thread's 16-byte accesses are 16 bytes apart (no bank
  // conflicts); window float4 k of thread t is A[t + k/2] (k even) or B[t + k/2]
  static constexpr int TLA = 4 * cdiv(NW0, 2) - 4, TLB = 4 * (NW0 / 2) - 4;
  static constexpr int TL1 = 4 * NW1 - 4;
  static constexpr int TL2 = 2 * NW2 - 2;
  static constexpr int TL3 = NW3 - 1;
  static constexpr int TLALL = TLA + TLB + TL1 + TL2 + TL3;  // tail values per chunk
  static constexpr int NWQ = cdiv(3 + MMAX, 4);  // float4 window of a coarse quad (4 positions)
  static constexpr int MIR = 4 * NWQ;            // mirrored ring entries: no window ever wraps
  // Grids with at most 32 widths (every plan of these (D, P) up to the widest
  // boxcar allowed) carry the width index in the SNR's low bits (enc_w).
  static constexpr bool ENC = D <= 1 && PL <= 2;
  static constexpr int EB = 5, EMAX = (1 << EB) - 1;
  static constexpr int NC0 = count_in<S0, MMAX>();  // level-0 widths; level j >= 1 starts at NC0 + (j-1) 2^D
};

// Shared-memory layout: three buffers of levels 0..3 (compile-time strides),
// then the rings of levels 4..top, the per-chunk coarse results and a small
// table of ring offsets/masks.
template <int D, int PL>
struct IgFix {
  using S = IgS<D, PL>;
  static constexpr int OB = al4(kC / 2 + S::TLA);  // B after A
  static constexpr int O1 = OB + al4(kC / 2 + S::TLB);
  static constexpr int O2 = O1 + al4(kC / 2 + S::TL1);
  static constexpr int O3 = O2 + al4(kC / 4 + S::TL2);
  static constexpr int FB = O3 + al4(kC / 8 + S::TL3);  // one buffer of levels 0..3
  __host__ __device__ static constexpr int f0(int b) { return b * FB; }  // A; B at f0 + OB
  __host__ __device__ static constexpr int f1(int b) { return b * FB + O1; }
  __host__ __device__ static constexpr int f2(int b) { return b * FB + O2; }
  __host__ __device__ static constexpr int f3(int b) { return b * FB + O3; }
  static constexpr int NBUF = 3;
  static constexpr int RINGS = NBUF * FB;
};

// A ring holds every block a window of the chunk being evaluated can reach
// (the chunk and mmax blocks past it), plus the blocks of the chunk being built
// meanwhile.
__host__ __device__ inline int ring_size(int j, int mmax) {
  return next_pow2(cdiv(2 * kC, 1 << j) + mmax + 2);
}

// offsets (floats) of the rings' end, the coarse results (two buffers of
// values and widths), the coarse-merge keys (two buffers) and the ring table.
// Each ring stores mmax extra entries that mirror its first ones, so that a
// window of mmax consecutive blocks never wraps.
constexpr int kResN = kResHi + kMaxLevels;  // slots of one coarse-result buffer
constexpr int kBcm = kC / 16;               // starts = 0 mod 16 in a chunk


struct IgDyn {
  int res_y, res_w, bcm, tab, ab, total;
  // nab: widths of the table-noise constants (0 for white noise); enc: coded
  // SNRs (no result slots)
  __host__ __device__ IgDyn(int rings, int top, int mmax, int nab, bool enc) {
    int o = rings;
    for (int j = kRing0; j <= top; ++j) o += al4(ring_size(j, mmax) + 4 * cdiv(3 + mmax, 4));
    res_y = o;
    o += enc ? 0 : 2 * kResN;
    res_w = o;
    o += enc ? 0 : kResN;
    bcm = o;
    o += 2 * kBcm;
    tab = o;
    o += 2 * kMaxLevels;
    ab = o;
    o += nab ? al4(2 * (nab + kAbPad)) : 0;
    total = o;
  }
};

// Tail value i of a chunk (levels 0A, 0B, 1, 2, 3 in turn): its offset src in
// the buffer of the previous chunk (that chunk's head) and dst in the chunk's
// own buffer (past the chunk's values).
template <class S, class FX>
__device__ __forceinline__ void tail_offsets(int i, int& src, int& dst) {
  if (i < S::TLA) {
    src = i;
    dst = kC / 2 + i;
  } else if ((i -= S::TLA) < S::TLB) {
    src = FX::OB + i;
    dst = FX::OB + kC / 2 + i;
  } else if ((i -= S::TLB) < S::TL1) {
    src = FX::O1 + i;
    dst = FX::O1 + kC / 2 + i;
  } else if ((i -= S::TL1) < S::TL2) {
    src = FX::O2 + i;
    dst = FX::O2 + kC / 4 + i;
  } else {
    i -= S::TL2;
    src = FX::O3 + i;
    dst = FX::O3 + kC / 8 + i;
  }
}

template <int D, int PL, bool COARSE, bool TABLE, int DT = -1>
__device__ __forceinline__ void igrid_unit(const SearchParams& p, const Unit& U, float* smem) {
  using S = IgS<D, PL>;
  using FX = IgFix<D, PL>;
  using SM = typename S::SM;
  using S0 = typename S::S0;
  constexpr int MMAX = S::MMAX;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t row = U.row, t0 = U.t0;
  const int top = p.top;
  const int T = U.T, H = p.halo;
  const bool vec = U.vec;
  // everything below is relative to the segment start t0 (32-bit offsets)
  const unsigned char* __restrict__ xseg = U.xrow + t0 * p.esize;  // byte address
  const int dt = DT >= 0 ? DT : p.dtype;  // DT >= 0: the input type is fixed at compile time
  const bool vx = U.vec_x;
  float* __restrict__ yseg = U.yrow + t0;
  uint16_t* __restrict__ wseg = U.wrow + t0;
  const int64_t nleft = U.nt - t0;
  const int nrel = (int)(nleft < (int64_t)(T + H) ? nleft : (int64_t)(T + H));  // samples that exist
  const int64_t sleft = U.ns - t0;
  const int srel = (int)(sleft < (int64_t)T ? sleft : (int64_t)T);  // starts evaluated and stored
  constexpr bool ENC = S::ENC;
  const IgDyn L(FX::RINGS, top, MMAX, TABLE ? p.n_widths : 0, ENC);
  float2* AB = reinterpret_cast<float2*>(smem + L.ab);  // table noise: (a, b) per width index
  float mu, inv;
  row_noise<TABLE>(p, U.mu, U.sigma, row, AB, mu, inv);
  // candidate scale of block count m (white noise: 1/sqrt(m), times the level's
  // 2^(-j/2) after the maximum; table noise: the width's (a, b), first = the
  // level's first width index)
  auto scl = [&](const float2* ab, auto Pred) {
    return [&, ab](auto M) {
      constexpr int m = decltype(M)::value;
      if constexpr (TABLE)
        return ab[decltype(Pred)::rank(m)];
      else
        return p.rs[m];
    };
  };
  auto lvl_f = [&](int j) { return TABLE ? 1.0f : p.lvl_scale[j]; };
  // fine level J: white noise scales by bscale[J][m] = 1/sqrt(m 2^J) directly
  auto scl_fine = [&](auto J, auto Pred) {
    return [&](auto M) {
      constexpr int j = decltype(J)::value, m = decltype(M)::value;
      if constexpr (TABLE)
        return AB[p.lvl_first[j] + decltype(Pred)::rank(m)];
      else
        return p.bscale[j][m];
    };
  };
  float* RESY = smem + L.res_y;
  uint16_t* RESW = reinterpret_cast<uint16_t*>(smem + L.res_w);
  int* BCM = reinterpret_cast<int*>(smem + L.bcm);   // [2][kBcm] keys of the best coarse level
  int* RTAB = reinterpret_cast<int*>(smem + L.tab);  // [2j]: ring offset, [2j+1]: mask

  // -inf everywhere a chunk past the end of the row would have written
  for (int i = t; i < L.bcm; i += kThreads) smem[i] = ninf();
  for (int i = t; i < 2 * kBcm; i += kThreads) BCM[i] = INT_MIN;
  if (t == 0) {
    int o = FX::RINGS;
    for (int j = 0; j < kMaxLevels; ++j) {
      RTAB[2 * j] = 0;
      RTAB[2 * j + 1] = 0;
    }
    for (int j = kRing0; j <= top; ++j) {
      const int n = ring_size(j, MMAX);
      RTAB[2 * j] = o;
      RTAB[2 * j + 1] = n - 1;
      o += al4(n + S::MIR);
    }
  }
  __syncthreads();
  // ring write: slot and, for the first MIR slots, its mirror (a select, no branch)
  auto ring_put = [&](int base, int mask, int n, float v) {
    const int slot = n & mask;
    smem[base + slot] = v;
    smem[base + (slot < S::MIR ? slot + mask + 1 : slot)] = v;
  };
  // chunks at relative starts ar(k) = a0 - k*kC, k = 0..nch-1 (backwards in time)
  int a0 = T + H - kC;
  if (a0 >= nrel) a0 = ((nrel - 1) / kC) * kC;  // chunks at or past nt are all -inf
  const int nch = a0 / kC + 1;

  // Ring writes of levels 4..8: the 31 blocks a warp completes per chunk (16 of
  // level 4, 8 of 5, 4 of 6, 2 of 7, 1 of 8) are written by one lane each:
  // lane l writes block wb of level wj.  The lane that writes a block is one
  // that holds its sum after the warp's
  // butterfly: block b of level 4 on lane 2b + 1, of level 5 on 4b, of level 6
  // on 8b + 2, of level 7 on 16b + 6, level 8's on lane 14 (lane 30 has none),
  // so no lane fetches another lane's sum.
  const int wj = (lane & 1) ? 4 : (lane & 3) == 0 ? 5 : (lane & 7) == 2 ? 6 : (lane & 15) == 6 ? 7 : 8;
  const int wb = lane >> (wj - 3);
  const bool wput = COARSE && lane != 30 && wj <= top;
  int wn = 0;
  // Coarse evaluation: quads of 4 consecutive positions (float4 ring windows) for
  // levels 4..8 on the 62 first threads (32, 16, 8, 4, 2 quads); single positions
  // of levels 9, 10, 11 on lanes 0..6 of the last warp (after it has built those
  // levels; one code path for all seven), levels above 11 on its lane 7.
  const int ctop = top < kChunkLog ? top : kChunkLog;
  // (the coarse quads and singles of grids with more than 32 widths re-read
  // their ring offsets, masks and level constants per chunk from the ring table
  // and the kernel parameters; the ring writes and the coded grids' coarse
  // positions hold theirs in registers)
  int qj = 0, qn = 0, qq = 0;
  int sj = 0, sn = 0, sq = 0;
  // Coded grids: one coarse position per thread and chunk.  The chunk has
  // 2048 / 2^j positions of level j (255 for levels 4..11), so thread t takes
  // position cq of level cj: t < 128 level 4, the next 64 level 5, ..., t = 254
  // level 11; thread 255 takes the levels above 11 (one position every few
  // chunks).  Every warp then does the same small amount of coarse work.
  int cj = 0, cq = 0;
  if constexpr (COARSE && ENC) {
    int j = kRing0, u = t, n = kC >> kRing0;
    while (n > 1 && u >= n) {
      u -= n;
      n >>= 1;
      ++j;
    }
    if (u < n && j <= ctop) {
      cj = j;
      cq = u;
    }
  }
  // the ring of this thread's coarse level: offset and mask (the table is set)
  const int wbase = wput ? RTAB[2 * wj] : 0, wmask = wput ? RTAB[2 * wj + 1] : 0;  // this lane's ring writes
  const int cbase = (COARSE && ENC && cj) ? RTAB[2 * cj] : 0;
  const int cmask = (COARSE && ENC && cj) ? RTAB[2 * cj + 1] : 0;
  if (COARSE && wput) wn = ((a0 + 256 * warp) >> wj) + wb;  // block index at chunk 0 (relative to the segment)
  if (COARSE && !ENC) {
    int j = 0, u = -1;
    if (t < 62) {
      j = kRing0;
      u = t;
      while (u >= (512 >> j)) {
        u -= 512 >> j;
        ++j;
      }
    }
    if (u >= 0 && j <= ctop) {
      qj = j;
      qq = 4 * u;
      qn = (a0 >> j) + qq;  // first block of the quad at chunk 0
    }
    if (warp == kThreads / 32 - 1 && lane < 7) {
      const int j1 = lane < 4 ? 9 : (lane < 6 ? 10 : 11);
      if (j1 <= ctop) {
        sj = j1;
        sq = lane < 4 ? lane : (lane < 6 ? lane - 4 : 0);
        sn = (a0 >> j1) + sq;
      }
    }
  }
  // level-9..11 blocks of a chunk: lanes 0..7 of the last warp hold the chunk's
  // eight level-8 blocks and a butterfly over them gives the sums; block b of
  // level 9 is put by lane 2b + 1, of level 10 by lane 4b, level 11's by lane 2
  const int lj = (lane & 1) ? 9 : (lane & 3) == 0 ? 10 : 11;
  const int lb = lane >> (lj - 8);
  const bool lbuild = COARSE && warp == kThreads / 32 - 1 && lane < 8 && lane != 6 && lj <= top;

  // ---- building chunk k: levels 0..3 into buffer k % 3 (+ tails), rings 4..8 ----
  // The lookahead tail of chunk k is the head of chunk k-1 (built one iteration
  // earlier, before the last barrier), copied from its buffer.  Writing it into
  // the next buffer from registers instead would race with a slow warp still
  // evaluating the chunk that buffer held three chunks ago.
  // (buf: k mod 3, the buffer set of chunk k, kept by the pipeline loop)
  auto build = [&](int k, int buf, const Raw8& raw) {
    const int ar = a0 - k * kC;
    if (k > 0 && warp == kTailWarp) {  // lookahead tails, one value per lane of one warp
      const int pb = buf == 0 ? FX::NBUF - 1 : buf - 1;
      for (int i = lane; i < S::TLALL; i += 32) {
        int src, dst;
        tail_offsets<S, FX>(i, src, dst);
        smem[buf * FX::FB + dst] = smem[pb * FX::FB + src];
      }
    }
    float4 v0, v1;
    cvt8(raw, ar + 8 * t, nrel, dt, mu, inv, v0, v1);
    float* F0 = smem + FX::f0(buf);
    *reinterpret_cast<float4*>(F0 + 4 * t) = v0;
    *reinterpret_cast<float4*>(F0 + FX::OB + 4 * t) = v1;
    const float p0 = v0.x + v0.y, p1 = v0.z + v0.w, p2 = v1.x + v1.y, p3 = v1.z + v1.w;
    const float4 pp = make_float4(p0, p1, p2, p3);
    *reinterpret_cast<float4*>(smem + FX::f1(buf) + 4 * t) = pp;
    const float q0 = p0 + p1, q1 = p2 + p3;
    *reinterpret_cast<float2*>(smem + FX::f2(buf) + 2 * t) = make_float2(q0, q1);
    const float o8 = q0 + q1;
    smem[FX::f3(buf) + t] = o8;
    if (COARSE) {
      // block sums of levels 4..8 (every lane of a block holds its sum), then one
      // lane per block fetches it and writes the ring
      const float s4 = o8 + __shfl_xor_sync(kFull, o8, 1);
      const float s5 = s4 + __shfl_xor_sync(kFull, s4, 2);
      const float s6 = s5 + __shfl_xor_sync(kFull, s5, 4);
      const float s7 = s6 + __shfl_xor_sync(kFull, s6, 8);
      const float s8 = s7 + __shfl_xor_sync(kFull, s7, 16);
      const float v = wj == 4 ? s4 : wj == 5 ? s5 : wj == 6 ? s6 : wj == 7 ? s7 : s8;
      if (wput) ring_put(wbase, wmask, wn - ((k * kC) >> wj), v);
    }
  };

  // ---- coarse work of chunk k (after the barrier that follows its build) ----
  // Each result also goes into a per-start key (order-preserving float key with
  // the level in its 4 low bits) through a shared atomic maximum, so that the
  // fine step finds the best coarse level of a start with one read.
  auto coarse = [&](int k) {
    const int ar = a0 - k * kC;
    if (warp == kThreads / 32 - 1 && top >= 9) {  // blocks of levels 9.. need every warp's level 8
      {
        const float v8 = lane < 8 ? smem[RTAB[2 * 8] + (((ar >> 8) + lane) & RTAB[2 * 8 + 1])] : 0.0f;
        const float s9 = v8 + __shfl_xor_sync(kFull, v8, 1);
        const float s10 = s9 + __shfl_xor_sync(kFull, s9, 2);
        const float s11 = s10 + __shfl_xor_sync(kFull, s10, 4);
        if (lbuild) ring_put(RTAB[2 * lj], RTAB[2 * lj + 1], (ar >> lj) + lb, lj == 9 ? s9 : lj == 10 ? s10 : s11);
      }
      for (int j = kChunkLog + 1; j <= top; ++j) {  // blocks longer than a chunk (rare)
        __syncwarp();
        if (lane == 0 && (((t0 + ar) & ((1LL << j) - 1)) == 0)) {
          const int n = ar >> j;
          const float* R = smem + RTAB[2 * (j - 1)];
          const int m = RTAB[2 * (j - 1) + 1];
          ring_put(RTAB[2 * j], RTAB[2 * j + 1], n, R[(2 * n) & m] + R[(2 * n + 1) & m]);
        }
      }
      __syncwarp();
    }
    if (ar >= srel) return;  // halo chunk (or past the evaluated starts): nothing to evaluate
    float* RY = RESY + (k & 1) * kResN;  // unused with coded SNRs
    uint16_t* RW = RESW + (k & 1) * kResN;
    int* KB = BCM + (k & 1) * kBcm;
    if constexpr (ENC) {
      if (cj) {  // this thread's position: a window of MMAX blocks
        const int first = p.lvl_first[cj];
        const float* R = smem + cbase + (((ar >> cj) + cq) & cmask);  // mirrored ring: no wrap
        float win[MMAX];
        load_window1<MMAX>(R, win);
        auto scq = [&](auto M) {
          constexpr int m = decltype(M)::value;
          if constexpr (TABLE)
            return AB[first + SM::rank(m)];
          else
            return p.bscale[cj][m];
        };
        float out[1];
        eval_window_enc<1, MMAX, SM, S::EB, true>(win, (cj == top) ? p.n_top : SM::MM, scq, S::EMAX - first, out);
        // a position without a valid candidate (all -inf, coded as NaNs) yields the
        // canonical NaN, whose key would beat every SNR: it posts nothing
        atomicMax(KB + (cq << (cj - 4)), out[0] == out[0] ? fkey(out[0]) : INT_MIN);
      }
      if (t == kThreads - 1)
        for (int jj = kChunkLog + 1; jj <= top; ++jj)
          if (((t0 + ar) & ((1LL << jj) - 1)) == 0) {
            float bv;
            int bq;
            eval_one_masked<MMAX, SM>(smem + RTAB[2 * jj] + ((ar >> jj) & RTAB[2 * jj + 1]),
                                      (jj == top) ? p.n_top : SM::MM, scl(AB + p.lvl_first[jj], SM{}), bv, bq);
            const float y = enc_w<S::EB>(bv * lvl_f(jj), S::EMAX - p.lvl_first[jj] - bq);
            if (y == y) atomicMax(KB, fkey(y));
          }
      return;
    }
    // result of position q of level j: slot (the position's index among the
    // chunk's coarse positions), start key for the fine step's merge
    auto put = [&](int j, int q, float y, int wi) {
      const int slot = (j <= kChunkLog) ? kThreads - (1 << (kChunkLog + 1 - j)) + q : kResHi + j - kChunkLog - 1;
      RY[slot] = y;
      RW[slot] = (uint16_t)wi;
      atomicMax(KB + (q << (j - 4)), (fkey(y) & ~15) | (15 - (j - 4)));
    };
    if (qj) {  // four consecutive positions from one float4 window
      float win[S::NWQ * 4];
      const int first = p.lvl_first[qj];
      const float f = lvl_f(qj);
      const int nu = (qj == top) ? p.n_top : SM::MM;
      load_window4<S::NWQ>(smem + RTAB[2 * qj] + ((qn - ((k * kC) >> qj)) & RTAB[2 * qj + 1]), win);
      if constexpr (ENC) {
        float out[4];
        auto scq = [&](auto M) {
          constexpr int m = decltype(M)::value;
          if constexpr (TABLE)
            return AB[first + SM::rank(m)];
          else
            return p.rs[m] * f;
        };
        eval_window_enc<4, MMAX, SM, S::EB, true>(win, nu, scq, S::EMAX - first, out);
        // a position without a valid candidate (all -inf, coded as NaNs) yields the
        // canonical NaN, whose key would beat every SNR: it posts nothing
#pragma unroll
        for (int r = 0; r < 4; ++r)
          atomicMax(KB + ((qq + r) << (qj - 4)), out[r] == out[r] ? fkey(out[r]) : INT_MIN);
      } else {
        float o[4];
        eval_set_enc<4, MMAX, SM, true>(win, nu, scl(AB + first, SM{}), o);
#pragma unroll
        for (int r = 0; r < 4; ++r) put(qj, qq + r, o[r] == o[r] ? dec_v<5>(o[r]) * f : ninf(), first + dec_w<5>(o[r]));
      }
    }
    if (sj) {
      float bv;
      int bq;
      const int first = p.lvl_first[sj];
      eval_one_masked<MMAX, SM>(smem + RTAB[2 * sj] + ((sn - ((k * kC) >> sj)) & RTAB[2 * sj + 1]),
                                (sj == top) ? p.n_top : SM::MM, scl(AB + first, SM{}), bv, bq);
      if constexpr (ENC) {
        const float y = enc_w<S::EB>(bv * lvl_f(sj), S::EMAX - first - bq);
        atomicMax(KB + (sq << (sj - 4)), y == y ? fkey(y) : INT_MIN);
      }
      else
        put(sj, sq, bv * lvl_f(sj), first + bq);
    }
    if (warp == kThreads / 32 - 1 && lane == 7)
      for (int jj = kChunkLog + 1; jj <= top; ++jj)
        if (((t0 + ar) & ((1LL << jj) - 1)) == 0) {
          float bv;
          int bq;
          eval_one_masked<MMAX, SM>(smem + RTAB[2 * jj] + ((ar >> jj) & RTAB[2 * jj + 1]),
                                    (jj == top) ? p.n_top : SM::MM, scl(AB + p.lvl_first[jj], SM{}), bv, bq);
          if constexpr (ENC) {
            const float y = enc_w<S::EB>(bv * lvl_f(jj), S::EMAX - p.lvl_first[jj] - bq);
            if (y == y) atomicMax(KB, fkey(y));
          }
          else
            put(jj, 0, bv * lvl_f(jj), p.lvl_first[jj] + bq);
        }
  };

  // ---- fine levels, merge and store of chunk k -----------------------------
  float tmax = ninf();
  auto fine = [&](int k, int buf) {
    const int ar = a0 - k * kC;
    if (ar >= srel) return;
    float y[8];
    int w[8];
    uint32_t pk[4];  // coded grids: the widths, packed in pairs
    if constexpr (ENC) {
      // coded SNRs: every maximum and merge is a max instruction; level j >= 1
      // starts at width index NC0 + (j-1) MM (compile-time)
      {
        float win[S::NW0 * 4];
        load_window4_ab<S::NW0>(smem + FX::f0(buf) + 4 * t, FX::OB, win);
        const auto sc0 = scl(AB, S0{});
        // (white noise: width 1, block count 1 of level 0, has scale 1)
        if (!COARSE && top == 0)
          eval_window_enc<8, MMAX, S0, S::EB, true, !TABLE>(win, p.n_top, sc0, S::EMAX, y);
        else
          eval_window_enc<8, MMAX, S0, S::EB, false, !TABLE>(win, p.n_top, sc0, S::EMAX, y);
      }
      if (COARSE || top >= 1) {
        float win1[S::NW1 * 4], o[4];
        load_window4<S::NW1>(smem + FX::f1(buf) + 4 * t, win1);
        const auto scj = scl_fine(std::integral_constant<int, 1>{}, SM{});
        constexpr int c0 = S::EMAX - S::NC0;
        if (!COARSE && top == 1)
          eval_window_enc<4, MMAX, SM, S::EB, true>(win1, p.n_top, scj, c0, o);
        else
          eval_window_enc<4, MMAX, SM, S::EB, false>(win1, p.n_top, scj, c0, o);
#pragma unroll
        for (int r = 0; r < 4; ++r) y[2 * r] = fmaxf(y[2 * r], o[r]);
      }
      if (COARSE || top >= 2) {
        float win2[S::NW2 * 2], o[2];
        load_window2<S::NW2>(smem + FX::f2(buf) + 2 * t, win2);
        const auto scj = scl_fine(std::integral_constant<int, 2>{}, SM{});
        constexpr int c0 = S::EMAX - S::NC0 - SM::MM;
        if (!COARSE && top == 2)
          eval_window_enc<2, MMAX, SM, S::EB, true>(win2, p.n_top, scj, c0, o);
        else
          eval_window_enc<2, MMAX, SM, S::EB, false>(win2, p.n_top, scj, c0, o);
        y[0] = fmaxf(y[0], o[0]);
        y[4] = fmaxf(y[4], o[1]);
      }
      if (COARSE || top >= 3) {
        float win3[S::NW3], o[1];
        load_window1<S::NW3>(smem + FX::f3(buf) + t, win3);
        const auto scj = scl_fine(std::integral_constant<int, 3>{}, SM{});
        constexpr int c0 = S::EMAX - S::NC0 - 2 * SM::MM;
        if (!COARSE && top == 3)
          eval_window_enc<1, MMAX, SM, S::EB, true>(win3, p.n_top, scj, c0, o);
        else
          eval_window_enc<1, MMAX, SM, S::EB, false>(win3, p.n_top, scj, c0, o);
        y[0] = fmaxf(y[0], o[0]);
      }
      if (COARSE) {  // best coarse result at start 8t (even t): one key, NaN when none
        int* kp = BCM + (k & 1) * kBcm + (t >> 1);
        const int key = *kp;
        *kp = INT_MIN;  // ready for chunk k + 2 (both lanes of a pair write the same value)
        y[0] = fmaxf(y[0], (t & 1) ? ninf() : fkey_inv(key));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) pk[q] = dec_w_pair<S::EB>(y[2 * q], y[2 * q + 1]);
#pragma unroll
      for (int r = 0; r < 8; ++r) y[r] = dec_v<S::EB>(y[r]);
    } else {
      // more than 32 widths: every level's maximum is coded with its rank within
      // the level (eval_set_enc), decoded once per position and merged with the
      // levels below by a strict '>' (the smaller width wins a tie)
      auto merge_coded = [&](float& yv, int& wv, float c, int first) {
        merge1(yv, wv, dec_v<5>(c), first + dec_w<5>(c));
      };
      {
        float win[S::NW0 * 4], o[8];
        load_window4_ab<S::NW0>(smem + FX::f0(buf) + 4 * t, FX::OB, win);
        const auto sc0 = scl(AB, S0{});
        if (!COARSE && top == 0)
          eval_set_enc<8, MMAX, S0, true>(win, p.n_top, sc0, o);
        else
          eval_set_enc<8, MMAX, S0, false>(win, p.n_top, sc0, o);
#pragma unroll
        for (int r = 0; r < 8; ++r) {  // level 0 starts at width index 0
          y[r] = dec_v<5>(o[r]);
          w[r] = dec_w<5>(o[r]);
        }
      }
      if (COARSE || top >= 1) {
        float win[S::NW1 * 4], o[4];
        load_window4<S::NW1>(smem + FX::f1(buf) + 4 * t, win);
        const auto scj = scl_fine(std::integral_constant<int, 1>{}, SM{});
        if (!COARSE && top == 1)
          eval_set_enc<4, MMAX, SM, true>(win, p.n_top, scj, o);
        else
          eval_set_enc<4, MMAX, SM, false>(win, p.n_top, scj, o);
        const int first = p.lvl_first[1];
#pragma unroll
        for (int r = 0; r < 4; ++r) merge_coded(y[2 * r], w[2 * r], o[r], first);
      }
      if (COARSE || top >= 2) {
        float win[S::NW2 * 2], o[2];
        load_window2<S::NW2>(smem + FX::f2(buf) + 2 * t, win);
        const auto scj = scl_fine(std::integral_constant<int, 2>{}, SM{});
        if (!COARSE && top == 2)
          eval_set_enc<2, MMAX, SM, true>(win, p.n_top, scj, o);
        else
          eval_set_enc<2, MMAX, SM, false>(win, p.n_top, scj, o);
        const int first = p.lvl_first[2];
        merge_coded(y[0], w[0], o[0], first);
        merge_coded(y[4], w[4], o[1], first);
      }
      if (COARSE || top >= 3) {
        float win[S::NW3], o[1];
        load_window1<S::NW3>(smem + FX::f3(buf) + t, win);
        const auto scj = scl_fine(std::integral_constant<int, 3>{}, SM{});
        if (!COARSE && top == 3)
          eval_set_enc<1, MMAX, SM, true>(win, p.n_top, scj, o);
        else
          eval_set_enc<1, MMAX, SM, false>(win, p.n_top, scj, o);
        merge_coded(y[0], w[0], o[0], p.lvl_first[3]);
      }
      if (COARSE) {  // best coarse level at start 8t (even t: 8t = 0 mod 16), without branching
        int* kp = BCM + (k & 1) * kBcm + (t >> 1);
        const int key = *kp;
        *kp = INT_MIN;  // ready for chunk k + 2 (both lanes of a pair write the same value)
        const int lvl = kRing0 + 15 - (key & 15);
        const int slot = (lvl <= kChunkLog) ? 256 - (1 << (kChunkLog + 1 - lvl)) + (t >> (lvl - 3))
                                            : kResHi + lvl - kChunkLog - 1;
        const bool use = !(t & 1) && key != INT_MIN;
        const float yv = RESY[(k & 1) * kResN + (use ? slot : 0)];
        const int wv = RESW[(k & 1) * kResN + (use ? slot : 0)];
        const bool take = use && yv > y[0];
        y[0] = take ? yv : y[0];
        w[0] = take ? wv : w[0];
      }
    }
    const int s0 = ar + 8 * t;
    if (s0 + 8 <= srel) {
      tmax = fmax3(fmax3(tmax, y[0], y[1]), fmax3(y[2], y[3], y[4]), fmax3(y[5], y[6], y[7]));
    } else {
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (s0 + r < srel) tmax = fmaxf(tmax, y[r]);
    }
    if constexpr (ENC)
      store8_pk(yseg, wseg, s0, srel, vec, y, pk);
    else
      store8(yseg, wseg, s0, srel, vec, y, w);
    if ((ar & (kCandTile - 1)) == 0) {  // last chunk of a candidate tile (we walk backwards)
      tile_max_atomic(U.tm_row, t0 + ar, tmax);
      tmax = ninf();
    }
  };

  // ---- pipeline --------------------------------------------------------------
  // the samples of the next chunk but one are loaded (prefetched into registers)
  // while the current chunks are worked on
  Raw8 nx = load_raw8(xseg, a0 + 8 * t, nrel, dt, vx);
  {
    const Raw8 cx = nx;
    if (nch > 1) nx = load_raw8(xseg, a0 - kC + 8 * t, nrel, dt, vx);
    build(0, 0, cx);
  }
  __syncthreads();
  if (COARSE) coarse(0);
  int b0 = 0, b1 = 1;  // buffer sets of chunks k and k + 1
  for (int k = 0; k < nch; ++k) {
    const bool more = k + 1 < nch;
    if (more) {
      const Raw8 cx = nx;
      if (k + 2 < nch) nx = load_raw8(xseg, a0 - (k + 2) * kC + 8 * t, nrel, dt, vx);
      build(k + 1, b1, cx);
    }
    __syncthreads();
    if (COARSE && more) coarse(k + 1);
    fine(k, b0);
    b0 = b1;
    b1 = b1 == FX::NBUF - 1 ? 0 : b1 + 1;
  }
}

// CTAs per SM the registers are sized for (measured per grid on 4 096 x 1 048 576
// rows: IG(2) 15.8 / 15.2 / 14.8 ms at 2 / 3 / 4 CTAs, IG(3) 25.2 / 24.0 / 24.4 ms)
template <int D, int PL>
constexpr int ig_min_ctas() {
  return (IgS<D, PL>::MMAX <= 6 || (D == 2 && PL == 3)) ? 4 : 3;
}

// One CTA per unit of a single-series search (DT: input type fixed at compile
// time, or -1: read from the parameters).
template <int D, int PL, bool COARSE, bool TABLE, int DT>
__global__ void __launch_bounds__(kThreads, (ig_min_ctas<D, PL>())) igrid_stream_kernel(const SearchParams p) {
  extern __shared__ __align__(16) float smem[];
  igrid_unit<D, PL, COARSE, TABLE, DT>(p, plan_unit(p, blockIdx.x), smem);
}

// Batched search: persistent CTAs stride over the units of every range.
template <int D, int PL, bool COARSE>
__global__ void __launch_bounds__(kThreads, (IgS<D, PL>::MMAX <= 6 ? 4 : 2)) igrid_batch_kernel(const SearchParams p) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int flag;
  for (int64_t u = blockIdx.x; u < p.n_units; u += gridDim.x) {
    Unit U;
    if (!batch_unit(p, u, U, &flag)) continue;
    igrid_unit<D, PL, COARSE, false>(p, U, smem);
    __syncthreads();
  }
}


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

template <int D, int PL, bool TABLE, int DT>
cudaError_t launch_ig(const spd_plan& plan, const SearchParams& p, size_t smem, cudaStream_t s) {
  const int64_t nblk = plan.desc.ndm * plan.tiles_per_row;
  return plan.top >= kRing0 ? launch_one(igrid_stream_kernel<D, PL, true, TABLE, DT>, smem, nblk, p, s)
                            : launch_one(igrid_stream_kernel<D, PL, false, TABLE, DT>, smem, nblk, p, s);
}

template <int D, int PL>
size_t ig_smem_bytes(const spd_plan& plan, bool table) {
  const int nab = table ? (int)plan.widths.size() : 0;
  return sizeof(float) * (size_t)IgDyn(IgFix<D, PL>::RINGS, plan.top, IgS<D, PL>::MMAX, nab, IgS<D, PL>::ENC).total;
}

}  // namespace
}  // namespace spd
