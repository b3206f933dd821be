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
//   * one CTA per row; each of its 8 warps streams its own contiguous share of
//     the row in steps of 256 samples (8 per lane), the samples of 16-byte
//     aligned rows arriving by bulk copies (cp.async.bulk) into a per-warp ring
//     of shared-memory stages of two steps each (one copy and one mbarrier wait
//     per two steps; a waiting warp sleeps in the wait instead of spinning on
//     the issue slots); no barrier of the CTA
//     until the final reduction;
//   * levels 0..3 from each lane's samples, 4..8 from the warp's shuffle tree,
//     9..11 from a tree over the level-8 sums of the 8 steps of a 2048-sample
//     chunk, 12.. accumulated over chunks; one lane keeps each block;
//   * a value of level k is kept when |v - mu_k| <= thr sigma_k of the previous
//     pass (the first pass keeps every value);
//   * each lane sums the kept values shifted by the previous mean (w = v - c_k,
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

// ---- staged copies: cp.async.bulk into per-warp shared rings, completion on mbarriers
constexpr int kSub = 256;                       // samples of one warp step (8 per lane)
constexpr int kWarpRing = 4096;                 // bytes of one warp's ring (4 f32 / 8 f16 / 16 u8 steps)
constexpr int kMaxStages = kWarpRing / kSub;    // stages of u8 steps
constexpr int kWarps = kThreads / 32;
constexpr long long kMsdWaitNs = 2000000000LL;  // limit of one wait for a step's samples (they arrive in microseconds)

__device__ __forceinline__ uint32_t smem_addr(const void* q) { return (uint32_t)__cvta_generic_to_shared(q); }

__device__ __forceinline__ void bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

// One thread: announce `bytes` on `bar` and copy them from global `src` to shared `dst`
// (both 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Wait until the phase of parity `par` of `bar` has completed; false when that
// takes longer than kMsdWaitNs.
constexpr uint32_t kSuspendNs = 20000;  // a waiting warp sleeps (no issue slots) until the copy lands, at most this long
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t par) {
  const uint32_t a = smem_addr(bar);
  uint32_t ok;
  uint64_t t0 = 0;
  for (int it = 0;; ++it) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(par), "r"(kSuspendNs)
        : "memory");
    if (ok) return true;
    uint64_t now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (it == 0) t0 = now;
    else if ((long long)(now - t0) > kMsdWaitNs) return false;
  }
}

// The 8 raw samples of lane l from a staged step (the layout of load_raw8).
__device__ __forceinline__ Raw8 read_stage(const unsigned char* s, int l, int dtype) {
  Raw8 r;
  if (dtype == kDtF32) {
    const uint4* q = reinterpret_cast<const uint4*>(s + 32 * l);
    r.a = q[0];
    r.b = q[1];
  } else if (dtype == kDtU8) {
    const uint2 v = *reinterpret_cast<const uint2*>(s + 8 * l);
    r.a = make_uint4(v.x, v.y, 0u, 0u);
    r.b = make_uint4(0u, 0u, 0u, 0u);
  } else {
    r.a = *reinterpret_cast<const uint4*>(s + 16 * l);
    r.b = make_uint4(0u, 0u, 0u, 0u);
  }
  return r;
}

// One pass over a row (one CTA of 8 warps).  Each warp streams its own
// contiguous share of the row, whole groups of max(2048, 2^(nlev-1)) samples,
// so that no block of any level straddles two warps, in steps of 256 samples (8
// per lane) and needs no barrier until the final reduction.  BULK (16-byte
// aligned rows): the whole steps of a warp arrive through its shared ring, lane 0
// refilling a stage once the warp has used it; otherwise each lane loads its
// samples one step ahead into registers.
//   * levels 0..3: each lane's 8 samples;
//   * levels 4..8: after the warp's shuffle tree lane l (l > 0) holds the block of
//     level 4 + ctz(l) that no other lane keeps (level 4: odd lanes, 5: lanes 2
//     mod 4, 6: 4 mod 8, 7: 8 and 24, 8: 16);
//   * levels 9..11: lane i (i < 8) holds the level-8 sum of step i of the
//     current 2048-sample chunk; the same tree over lanes 0..7 leaves level
//     9 + ctz(l) in lane l = 1..7;
//   * levels 12..15: lane k - 4 (lanes 8..11) accumulates chunk sums into blocks
//     of 2^(k-11) chunks.
// So each lane keeps at most one value of one level per step and one per chunk.
// A row whose staged copy did not arrive gets NaN statistics.
template <bool BULK, int DT>
__global__ void __launch_bounds__(kThreads, 3) msd_pass_kernel(const MsdParams p, int pass) {
  constexpr int ES = DT == kDtF32 ? 4 : (DT == kDtU8 ? 1 : 2);  // bytes per sample
  __shared__ alignas(128) unsigned char ring[BULK ? kWarps * kWarpRing : 16];
  __shared__ alignas(8) uint64_t full[kWarps][kMaxStages];
  __shared__ float cshift[kMsdMaxLevels], clim[kMsdMaxLevels];
  __shared__ float s8[kThreads / 32];
  __shared__ double red[kThreads / 32][kMsdMaxLevels][2];
  __shared__ long long redn[kThreads / 32][kMsdMaxLevels];
  __shared__ int done, failed;
  __shared__ float kahan[16 * kThreads];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t row = blockIdx.x;
  const int nlev = p.nlev;
  MsdLevel* st = reinterpret_cast<MsdLevel*>(p.state) + row * kMsdMaxLevels;
  const unsigned char* __restrict__ xrow = static_cast<const unsigned char*>(p.x) + row * p.ld * ES;
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
    // pilot shift: the mean of the row's first 2048 samples, times 2^k
    const int n0 = nt < kC ? (int)nt : kC;
    float v0, v1;
    {
      float4 a, b;
      cvt8<false>(load_raw8(xrow, 8 * t, n0, DT, vx), 8 * t, n0, DT, 0.0f, 1.0f, a, b);
      float f[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      v0 = 0.0f;
#pragma unroll
      for (int i = 0; i < 8; ++i) v0 += (8 * t + i < n0) ? f[i] : 0.0f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v0 += __shfl_xor_sync(kFull, v0, o);
    if (lane == 0) s8[warp] = v0;
    __syncthreads();
    v1 = 0.0f;
    for (int w = 0; w < kThreads / 32; ++w) v1 += s8[w];
    const float c0 = v1 / (float)n0;
    if (t < nlev) {
      cshift[t] = c0 * (float)(1 << t);
      clim[t] = FLT_MAX;
    }
  }
  if (t == 0) failed = 0;

  // this warp's steps [u0, u1): whole groups of gs steps
  const int64_t nsub = (nt + kSub - 1) / kSub, nfs = nt / kSub;  // steps; whole steps
  const int gs = (1 << (nlev - 1)) > kC ? (1 << (nlev - 1)) / kSub : kC / kSub;
  const int64_t ng = (nsub + gs - 1) / gs;
  const int64_t u0 = (ng * warp / kWarps) * gs;
  const int64_t u1 = min((ng * (warp + 1) / kWarps) * gs, nsub);
  constexpr int sbytes = kSub * ES;
  constexpr int lgs = ES == 4 ? 2 : (ES == 2 ? 3 : 4);  // steps in the ring: kWarpRing / sbytes
  constexpr int lgp = lgs - 1;                          // stages of two steps each, one copy per stage
  const int64_t ub = BULK ? min(u1, nfs) : u0;  // steps [u0, ub) arrive staged
  unsigned char* wring = ring + (BULK ? warp * kWarpRing : 0);
  if (BULK) {
    if (lane == 0) {
      for (int i = 0; i < (1 << lgp); ++i) bar_init(&full[warp][i]);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      for (int i = 0; i < (1 << lgp); ++i) {
        const int64_t us = u0 + 2 * i;
        if (us < ub)
          bulk_load(wring + 2 * i * sbytes, xrow + us * sbytes, (uint32_t)((us + 2 <= ub ? 2 : 1) * sbytes),
                    &full[warp][i]);
      }
    }
  }
  __syncthreads();

  // levels this lane keeps; an unused level gets limit -1 (nothing passes |w| <= -1)
  float sh[4], lim[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    sh[k] = k < nlev ? cshift[k] : 0.0f;
    lim[k] = k < nlev ? clim[k] : -1.0f;
  }
  const int jl = lane ? __ffs(lane) - 1 : 5;  // set A: level 4 + jl (lane 0: none)
  const int ka = 4 + jl;
  const float sha = (jl < 5 && ka < nlev) ? cshift[ka] : 0.0f;
  const float lima = (jl < 5 && ka < nlev) ? clim[ka] : -1.0f;
  // set B: lanes 1..7 level 9 + ctz(lane), block lane >> (ctz + 1); lanes 8..11 level lane + 4
  const int kb = (lane >= 1 && lane < 8) ? 9 + jl : ((lane >= 8 && lane < 12) ? lane + 4 : 0);
  const float shb = (kb && kb < nlev) ? cshift[kb] : 0.0f;
  const float limb = (kb && kb < nlev) ? clim[kb] : -1.0f;
  const int endb = (lane >= 1 && lane < 8) ? ((lane >> (jl + 1)) + 1) << kb : kC;  // block end in its chunk

  // levels 0..3: compensated sums over chunks (shared memory, one column per
  // thread: they change once per chunk), and sums over the steps of the
  // current chunk (registers)
  float* kc = kahan + t;  // [4 sums][4 levels][kThreads]
#pragma unroll
  for (int i = 0; i < 16; ++i) kc[i * kThreads] = 0.0f;
  float pw[4], pw2[4];
  float2 qw = make_float2(0.0f, 0.0f), qw2 = qw;  // levels 0, 1, 2 in packed pairs (first pass)
  float2 q1 = qw, q12 = qw, q2 = qw, q22 = qw;
  int cn[4], nfast = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) pw[k] = pw2[k] = 0.0f, cn[k] = 0;
  // First pass (no limits yet): a whole step whose 256 samples are finite keeps
  // every value of levels 0..8, so its sums need no compare and no select and
  // run in packed pairs; other steps (and later passes) take the general form.
  const bool keep_all = pass == 0 && nlev > 8;
  const bool has_a = jl < 5;
  float sa = 0.0f, sa2 = 0.0f, sb = 0.0f, sb2 = 0.0f, blk = 0.0f, q = 0.0f;
  int na = 0, nb = 0, bad = 0;

  auto step = [&](auto WHOLE, const Raw8& cx, int64_t u) {
    constexpr bool whole = decltype(WHOLE)::value;
    const int rem = whole ? kSub : (int)(nt - u * kSub);  // samples of the step
    const int o = 8 * lane;
    float f[8];
    {
      float4 a, b;
      cvt8<false>(cx, o, rem, DT, 0.0f, 1.0f, a, b);
      f[0] = a.x, f[1] = a.y, f[2] = a.z, f[3] = a.w, f[4] = b.x, f[5] = b.y, f[6] = b.z, f[7] = b.w;
      if (!whole) {
#pragma unroll
        for (int i = 0; i < 8; ++i) f[i] = (o + i < rem) ? f[i] : 0.0f;  // sums stay finite
      }
    }
    float p1[4], p2[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) p1[i] = f[2 * i] + f[2 * i + 1];
#pragma unroll
    for (int i = 0; i < 2; ++i) p2[i] = p1[2 * i] + p1[2 * i + 1];
    const float s3 = p2[0] + p2[1];
    float s = s3, v = 0.0f;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      s += __shfl_xor_sync(kFull, s, 1 << j);
      if (jl == j) v = s;
    }
    // s: the warp's 256-sample sum (the same in every lane); finite only when every sample is
    if (whole && keep_all && fabsf(s) <= FLT_MAX) {
#pragma unroll
      for (int i = 0; i < 8; i += 2) {  // level 0: two values per instruction
        const float2 w = __fadd2_rn(make_float2(f[i], f[i + 1]), make_float2(-sh[0], -sh[0]));
        qw = __fadd2_rn(qw, w);
        qw2 = __ffma2_rn(w, w, qw2);
      }
#pragma unroll
      for (int i = 0; i < 4; i += 2) {
        const float2 w = __fadd2_rn(make_float2(p1[i], p1[i + 1]), make_float2(-sh[1], -sh[1]));
        q1 = __fadd2_rn(q1, w);
        q12 = __ffma2_rn(w, w, q12);
      }
      {
        const float2 w = __fadd2_rn(make_float2(p2[0], p2[1]), make_float2(-sh[2], -sh[2]));
        q2 = __fadd2_rn(q2, w);
        q22 = __ffma2_rn(w, w, q22);
      }
      const float w3 = s3 - sh[3];
      pw[3] += w3;
      pw2[3] = fmaf(w3, w3, pw2[3]);
      ++nfast;  // 8, 4, 2, 1 values of levels 0..3
      const float wa = has_a ? v - sha : 0.0f;
      sa += wa;
      sa2 = fmaf(wa, wa, sa2);
      na += has_a ? 1 : 0;
      return s;
    }
    // a block counts when it ends inside the row
    auto keep = [&](int k, float v, int end) {
      const float w = v - sh[k];
      const bool in = (whole || end <= rem) && fabsf(w) <= lim[k];
      const float wm = in ? w : 0.0f;
      pw[k] += wm;
      pw2[k] = fmaf(wm, wm, pw2[k]);
      cn[k] += in ? 1 : 0;
    };
#pragma unroll
    for (int i = 0; i < 8; ++i) keep(0, f[i], o + i + 1);
#pragma unroll
    for (int i = 0; i < 4; ++i) keep(1, p1[i], o + 2 * i + 2);
#pragma unroll
    for (int i = 0; i < 2; ++i) keep(2, p2[i], o + 4 * i + 4);
    keep(3, s3, o + 8);
    const float w = v - sha;
    const int end = 8 * (lane & ~((2 << jl) - 1)) + (16 << jl);
    const bool in = (whole || end <= rem) && fabsf(w) <= lima;
    const float wa = in ? w : 0.0f;
    sa += wa;
    sa2 = fmaf(wa, wa, sa2);
    na += in ? 1 : 0;
    return s;  // the step's sum (level 8)
  };

  Raw8 nx;
  if (!BULK && u0 < u1) {
    const int64_t left = nt - u0 * kSub;
    nx = load_raw8(xrow + u0 * sbytes, 8 * lane, left < kSub ? (int)left : kSub, DT, vx);
  }
  uint32_t kk = 0;  // steps done by this warp (mod 2^32: ring stage, phase parity, step within its chunk)
  for (int64_t u = u0; u < u1; ++u, ++kk) {
    Raw8 cx;
    const uint32_t pk = kk >> 1;  // the stage (pair of steps) of this step
    const int stg = (int)(pk & ((1u << lgp) - 1));
    if (BULK && u < ub) {
      if ((kk & 1u) == 0) bad |= bar_wait(&full[warp][stg], (pk >> lgp) & 1u) ? 0 : 1;
      cx = read_stage(wring + (2 * stg + (int)(kk & 1u)) * sbytes, lane, DT);
    } else if (BULK) {
      cx = load_raw8(xrow + u * sbytes, 8 * lane, (int)(nt - u * kSub), DT, vx);
    } else {
      cx = nx;
      if (u + 1 < u1) {
        const int64_t left = nt - (u + 1) * kSub;
        nx = load_raw8(xrow + (u + 1) * sbytes, 8 * lane, left < kSub ? (int)left : kSub, DT, vx);
      }
    }
    const float s = u < nfs ? step(std::true_type{}, cx, u) : step(std::false_type{}, cx, u);
    if (lane == (int)(kk & 7u)) q = s;
    if (BULK && u < ub) {
      if ((kk & 1u) == 0 && __any_sync(kFull, bad)) {  // a stage did not arrive: wait (bounded) for the copies in flight
        if (lane == 0)
          for (uint32_t r = 0; r < (1u << lgp); ++r)
            if (u0 + 2 * (int64_t)(pk + r) < ub)
              bar_wait(&full[warp][(pk + r) & ((1u << lgp) - 1)], ((pk + r) >> lgp) & 1u);
        if (lane == 0) failed = 1;
        break;
      }
      if ((kk & 1u) == 1 || u + 1 == ub) {  // both steps of the stage used (or the last one): refill it
        __syncwarp();
        const int64_t us = u - (int64_t)(kk & 1u) + 2 * (1 << lgp);
        if (lane == 0 && us < ub)
          bulk_load(wring + 2 * stg * sbytes, xrow + us * sbytes, (uint32_t)((us + 2 <= ub ? 2 : 1) * sbytes),
                    &full[warp][stg]);
      }
    }
    if ((kk & 7u) == 7u || u + 1 == u1) {  // end of a 2048-sample chunk (or of the warp's share)
      const int64_t ch = u >> 3;
      float z = lane < 8 ? q : 0.0f, vb = 0.0f;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        z += __shfl_xor_sync(kFull, z, 1 << j);
        if (jl == j) vb = z;
      }
      const float v11 = __shfl_sync(kFull, z, 0);
      bool valid = ch * kC + endb <= nt;
      if (lane >= 8 && lane < 12) {
        blk += v11;
        vb = blk;
        const bool complete = ((ch + 1) & ((1 << (kb - 11)) - 1)) == 0;
        valid = complete && valid;
        if (complete) blk = 0.0f;
      }
      const float wb = vb - shb;
      const bool inb = valid && fabsf(wb) <= limb;
      sb += inb ? wb : 0.0f;
      sb2 += inb ? wb * wb : 0.0f;
      nb += inb ? 1 : 0;
      q = 0.0f;
      pw[0] += qw.x + qw.y;
      pw2[0] += qw2.x + qw2.y;
      pw[1] += q1.x + q1.y;
      pw2[1] += q12.x + q12.y;
      pw[2] += q2.x + q2.y;
      pw2[2] += q22.x + q22.y;
      qw = qw2 = q1 = q12 = q2 = q22 = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float s1 = kc[k * kThreads], c1 = kc[(8 + k) * kThreads];
        float s2 = kc[(4 + k) * kThreads], c2 = kc[(12 + k) * kThreads];
        kahan_add(s1, c1, pw[k]);
        kahan_add(s2, c2, pw2[k]);
        kc[k * kThreads] = s1, kc[(8 + k) * kThreads] = c1;
        kc[(4 + k) * kThreads] = s2, kc[(12 + k) * kThreads] = c2;
        pw[k] = pw2[k] = 0.0f;
      }
    }
  }
  __syncthreads();
  if (failed) {
    if (t < kMsdMaxLevels) {
      MsdLevel L;
      L.mu = L.sd = __longlong_as_double(0x7ff8000000000000LL);
      L.n = -2;
      L.conv = 1;
      L.pad = 0;
      st[t] = L;
    }
    return;
  }

  // FP64 reduction over the CTA, then the new statistics of every level
#pragma unroll
  for (int k = 0; k < kMsdMaxLevels; ++k) {
    double a, b;
    long long n;
    if (k < 4) {
      a = (double)kc[k * kThreads] - (double)kc[(8 + k) * kThreads];
      b = (double)kc[(4 + k) * kThreads] - (double)kc[(12 + k) * kThreads];
      n = cn[k] + ((long long)nfast << (3 - k));
    } else if (k < 9) {
      a = ka == k ? sa : 0.0, b = ka == k ? sa2 : 0.0, n = ka == k ? na : 0;
    } else {
      a = kb == k ? sb : 0.0, b = kb == k ? sb2 : 0.0, n = kb == k ? nb : 0;
    }
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
  const bool failed = st[0].n == -2;  // a chunk of the row did not arrive
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
    p.out_mu[row * p.n_widths + w] = failed ? __int_as_float(0x7fc00000) : (float)((double)L * m);
    p.out_sigma[row * p.n_widths + w] = failed ? __int_as_float(0x7fc00000) : (float)(sqrt((double)L) * r);
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
    const unsigned g = (unsigned)plan.desc.ndm;
    switch (p.dtype * 2 + (p.vec_x ? 1 : 0)) {
      case kDtF32 * 2 + 1: msd_pass_kernel<true, kDtF32><<<g, kThreads, 0, s>>>(p, pass); break;
      case kDtF32 * 2: msd_pass_kernel<false, kDtF32><<<g, kThreads, 0, s>>>(p, pass); break;
      case kDtF16 * 2 + 1: msd_pass_kernel<true, kDtF16><<<g, kThreads, 0, s>>>(p, pass); break;
      case kDtF16 * 2: msd_pass_kernel<false, kDtF16><<<g, kThreads, 0, s>>>(p, pass); break;
      case kDtBF16 * 2 + 1: msd_pass_kernel<true, kDtBF16><<<g, kThreads, 0, s>>>(p, pass); break;
      case kDtBF16 * 2: msd_pass_kernel<false, kDtBF16><<<g, kThreads, 0, s>>>(p, pass); break;
      case kDtU8 * 2 + 1: msd_pass_kernel<true, kDtU8><<<g, kThreads, 0, s>>>(p, pass); break;
      default: msd_pass_kernel<false, kDtU8><<<g, kThreads, 0, s>>>(p, pass); break;
    }
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  msd_table_kernel<<<(unsigned)plan.desc.ndm, kThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace spd
