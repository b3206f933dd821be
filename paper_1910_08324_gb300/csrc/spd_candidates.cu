// spd_candidates.cu -- threshold + peak-finding candidate selection (sm_103a).
//
// The paper selects candidates from the search output "using a peak-finding
// algorithm" (Sec. 4.5) without defining it.  Rule implemented here: start s of
// a row is a candidate iff Y[s] >= thr, Y[s] > Y[s'] for s - R <= s' < s and
// Y[s] >= Y[s'] for s < s' <= s + R (inside the row); the leftmost sample of a
// plateau wins and R = 0 is a plain threshold.
//
// Deterministic compaction in (row, start) order.  Candidate tiles (16384
// starts of one row) are taken 32 at a time by one warp ("groups"):
//   count  -- a warp reads its group's 32 tile maxima (recorded by the search
//             kernel) with one load, skips the tiles below the threshold without
//             reading them, and counts the candidates of the others; it writes
//             the 32 per-tile counts and their sum;
//   scan   -- one CTA turns the group sums into int64 group offsets (coalesced
//             passes of 1024 groups with a running carry) and writes the total
//             to *d_count;
//   write  -- a warp scans its group's 32 counts and re-tests the starts of the
//             tiles that have candidates, writing their records at offset +
//             prefix (a ballot per 32 consecutive starts keeps the order); only
//             the first cap records are kept.
// A warp reads a tile 512 starts at a time (16 independent loads per lane)
// and runs the peak test only where the threshold is met.
// Count and write run as a grid of persistent CTAs (a few per SM) that stride
// over the groups, eight groups (one per warp) at a time.  A CTA with few tiles
// that have candidates scans each of them with all its warps at once, one
// segment per warp (cta_together); otherwise each warp scans its own group's.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "spd_common.cuh"

// Scratch of spd_candidates_static: per-tile counts (int32), then per-group sums
// (int32) and offsets (int64), for at most kStaticCandTiles candidate tiles
// (1.1 MiB).  Every device that loads the library holds this array until the
// process exits; all calls on a device share it.
static __device__ __align__(256) unsigned char
    g_static_cand_scratch[spd::kStaticCandTiles * sizeof(int32_t) +
                          (spd::kStaticCandTiles / spd::kCandGroup) * (sizeof(int32_t) + sizeof(int64_t))];

namespace spd {
namespace {

constexpr int kCandThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kCandCtasPerSm = 8;  // persistent CTAs per SM of the count and write passes
static_assert(kCandGroup == 32, "a group is one tile per lane");
static_assert(sizeof(spd_candidate) == 24 && offsetof(spd_candidate, row) == 0 &&
                  offsetof(spd_candidate, width_idx) == 4 && offsetof(spd_candidate, start) == 8 &&
                  offsetof(spd_candidate, snr) == 16 && offsetof(spd_candidate, width) == 20,
              "records are written as three 8-byte words");

__device__ __forceinline__ float key_to_float(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// neighbours are read only inside [lo, hi) (the row, or for a mapped row the
// part of it that lies inside the original series)
__device__ __forceinline__ bool is_cand(const float* __restrict__ y, int64_t s, int64_t lo, int64_t hi,
                                        float thr, int R) {
  const float v = y[s];
  if (!(v >= thr)) return false;
  for (int q = 1; q <= R; ++q) {
    if (s - q >= lo && !(v > y[s - q])) return false;
    if (s + q < hi && !(v >= y[s + q])) return false;
  }
  return true;
}

__device__ __forceinline__ bool in_window(const CandParams& p, int64_t s) { return s >= p.s_lo && s < p.s_hi; }

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// (row, first start, end) of candidate tile `tile`
struct TileSpan {
  const float* y;
  const uint16_t* w;
  int64_t row, t0, end;
  int64_t lo, hi;  // the starts whose SNRs the peak test may read
  __device__ TileSpan(const CandParams& p, int64_t tile) {
    row = tile / p.tiles_per_row;
    t0 = (tile % p.tiles_per_row) * (int64_t)p.tile;
    end = (t0 + p.tile < p.nt) ? t0 + p.tile : p.nt;
    y = p.snr + row * p.ld;
    w = p.widx + row * p.ld;
    lo = 0;
    hi = p.nt;
    if (p.row_ids) {  // start s of this row is start s + off of the original one
      const int64_t off = (p.row_ids[row] % p.map_bpr) * p.map_block - p.s_lo;
      lo = -off > 0 ? -off : 0;
      hi = p.map_nt - off < p.nt ? p.map_nt - off : p.nt;
    }
  }
};

// The warp's SNRs at starts b + u*32 + lane, u < kUnroll (all loads issued
// before any is used); -inf at and past lim (<= the tile's end).
constexpr int kUnroll = 16;
__device__ __forceinline__ void load_block(const TileSpan& ts, int64_t b, int64_t lim, int lane,
                                           float (&v)[kUnroll]) {
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const int64_t s = b + u * 32 + lane;
    v[u] = (s < lim) ? __ldcs(ts.y + s) : __int_as_float(0xff800000u);
  }
}

// A tile with candidates is scanned by all kCtaWarps warps of a CTA at once, one
// segment each (a whole number of 32 * kUnroll-start blocks).
constexpr int kCtaWarps = kCandThreads / 32;
__device__ __forceinline__ int64_t seg_len(const CandParams& p) {
  const int64_t per = (p.tile + kCtaWarps - 1) / kCtaWarps;
  return (per + 32 * kUnroll - 1) / (32 * kUnroll) * (32 * kUnroll);
}

// Whether a CTA scans its live tiles together (each tile by all warps, one after
// the other) or each warp its own group's: together when that ends sooner.  A
// tile scanned together costs about twice its share of one warp's time (two
// barriers, the write pass counting its segment again, idle warps past a short
// row's end), so together wins when the busiest warp holds more than 2 /
// kCtaWarps of the live tiles (a few live tiles: together; most tiles live, as in
// a search of flagged blocks: each warp its own).
__device__ __forceinline__ bool cta_together(const unsigned (&hot)[kCtaWarps]) {
  int n = 0, mx = 0;
#pragma unroll
  for (int w = 0; w < kCtaWarps; ++w) {
    const int c = __popc(hot[w]);
    n += c;
    mx = c > mx ? c : mx;
  }
  return 2 * n < kCtaWarps * mx;
}

// Candidates among the starts [b0, b1) of a tile (one warp; the warp's total).
__device__ __forceinline__ int count_span(const CandParams& p, const TileSpan& ts, int64_t b0, int64_t b1,
                                         int lane) {
  int c = 0;
  for (int64_t b = b0; b < b1; b += 32 * kUnroll) {
    float v[kUnroll];
    load_block(ts, b, b1, lane, v);
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
      if (v[u] >= p.thr && in_window(p, b + u * 32 + lane))
        c += is_cand(ts.y, b + u * 32 + lane, ts.lo, ts.hi, p.thr, p.radius) ? 1 : 0;
  }
  return warp_sum(c);
}

// A CTA takes kCtaWarps consecutive groups at a time: each warp reads its
// group's 32 tile maxima, then the CTA counts the tiles at or above the
// threshold one after the other, all warps on each (one segment per warp).
__global__ void __launch_bounds__(kCandThreads) cand_count_kernel(const CandParams p, int64_t ntiles,
                                                                  int64_t ngroups) {
  __shared__ unsigned hot[kCtaWarps];
  __shared__ int segc[kCtaWarps];
  __shared__ int gs[kCtaWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = seg_len(p);
  for (int64_t g0 = (int64_t)blockIdx.x * kCtaWarps; g0 < ngroups; g0 += (int64_t)gridDim.x * kCtaWarps) {
    const int64_t g = g0 + warp;
    const int64_t tile = g * kCandGroup + lane;
    const bool in = g < ngroups && tile < ntiles;
    bool live = in;
    if (live && p.tile_max) live = key_to_float(reinterpret_cast<const int*>(p.tile_max)[tile]) >= p.thr;
    const unsigned m = __ballot_sync(kFull, live);
    if (lane == 0) {
      hot[warp] = m;
      gs[warp] = 0;
    }
    if (in && !live) p.counts[tile] = 0;
    __syncthreads();
    if (!cta_together(hot)) {  // each warp its own group's tiles, whole
      unsigned todo = m;
      int gsum = 0;
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const TileSpan ts(p, g * kCandGroup + src);
        const int c = count_span(p, ts, ts.t0, ts.end, lane);
        if (lane == 0) p.counts[g * kCandGroup + src] = c;
        gsum += c;
      }
      if (g < ngroups && lane == 0) p.gsum[g] = gsum;
      __syncthreads();  // hot is reused by the next groups
      continue;
    }
    for (int w2 = 0; w2 < kCtaWarps; ++w2) {
      unsigned todo = hot[w2];  // (the same for every thread)
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int64_t tl = (g0 + w2) * kCandGroup + src;
        const TileSpan ts(p, tl);
        const int64_t b0 = ts.t0 + warp * seg;
        const int64_t b1 = (b0 + seg < ts.end) ? b0 + seg : ts.end;
        const int c = (b0 < b1) ? count_span(p, ts, b0, b1, lane) : 0;
        if (lane == 0) segc[warp] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
          int tot = 0;
#pragma unroll
          for (int i = 0; i < kCtaWarps; ++i) tot += segc[i];
          p.counts[tl] = tot;
          gs[w2] += tot;
        }
        __syncthreads();
      }
    }
    if (g < ngroups && lane == 0) p.gsum[g] = gs[warp];
    __syncthreads();  // hot and gs are reused by the next groups
  }
}

__global__ void __launch_bounds__(kScanThreads) cand_scan_kernel(const CandParams p, int64_t ngroups) {
  __shared__ int64_t wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t carry = 0;
  for (int64_t base = 0; base < ngroups; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = (i < ngroups) ? p.gsum[i] : 0;
    int64_t x = v;  // inclusive warp scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += u;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(kFull, w, o);
        if (lane >= o) w += u;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    if (i < ngroups) p.goff[i] = carry + (warp ? wsum[warp - 1] : 0) + x - v;
    carry += wsum[kScanThreads / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *p.d_count = carry;
}

// Records of the candidates among the starts [b0, b1) of a tile (one warp),
// from offset base on, in start order (a ballot per 32 consecutive starts).
__device__ __forceinline__ void write_span(const CandParams& p, const TileSpan& ts, int64_t b0, int64_t b1,
                                           int lane, int64_t base) {
  const unsigned below = (1u << lane) - 1u;
  for (int64_t b = b0; b < b1 && base < p.cap; b += 32 * kUnroll) {
    float v[kUnroll];
    load_block(ts, b, b1, lane, v);
    static_for<0, kUnroll>([&](auto U) {
      constexpr int u = decltype(U)::value;
      const int64_t s = b + u * 32 + lane;
      const bool f = v[u] >= p.thr && in_window(p, s) && is_cand(ts.y, s, ts.lo, ts.hi, p.thr, p.radius);
      const unsigned bal = __ballot_sync(kFull, f);
      if (f) {
        const int64_t pos = base + __popc(bal & below);
        if (pos < p.cap) {  // the 24-byte record as three 8-byte stores
          const int wi = (int)ts.w[s];
          const int wd = p.width_mode ? p.width_tab[wi] : wi + 1;
          int64_t orow = ts.row, ostart = s;
          if (p.row_ids) {  // a searched block back to its row and start
            const int64_t blk = p.row_ids[ts.row];
            orow = blk / p.map_bpr;
            ostart = (blk % p.map_bpr) * p.map_block + (s - p.s_lo);
          }
          int2* o = reinterpret_cast<int2*>(p.out + pos);
          o[0] = make_int2((int)orow, wi);
          *reinterpret_cast<long long*>(o + 1) = (long long)ostart;
          o[2] = make_int2(__float_as_int(v[u]), wd);
        }
      }
      base += __popc(bal);
    });
  }
}

// The same groups per CTA as the count pass; each tile with candidates is
// written by all warps at once: each counts its segment again, takes its
// offset from the counts of the segments before it, and writes its records.
__global__ void __launch_bounds__(kCandThreads, 1) cand_write_kernel(const CandParams p, int64_t ntiles,
                                                                  int64_t ngroups) {
  __shared__ unsigned hot[kCtaWarps];
  __shared__ long long toff[kCtaWarps][kCandGroup];
  __shared__ int segc[kCtaWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = seg_len(p);
  for (int64_t g0 = (int64_t)blockIdx.x * kCtaWarps; g0 < ngroups; g0 += (int64_t)gridDim.x * kCtaWarps) {
    const int64_t g = g0 + warp;
    const int64_t tile = g * kCandGroup + lane;
    const int c = (g < ngroups && tile < ntiles) ? p.counts[tile] : 0;
    int x = c;  // inclusive warp scan of the tile counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += u;
    }
    toff[warp][lane] = (g < ngroups ? p.goff[g] : 0) + (x - c);
    const unsigned m = __ballot_sync(kFull, c > 0);
    if (lane == 0) hot[warp] = m;
    __syncthreads();
    if (!cta_together(hot)) {  // each warp its own group's tiles, whole
      unsigned todo = m;
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int64_t base = toff[warp][src];
        if (base >= p.cap) break;  // later tiles of the group start even later
        const TileSpan ts(p, g * kCandGroup + src);
        write_span(p, ts, ts.t0, ts.end, lane, base);
      }
      __syncthreads();  // hot and toff are reused by the next groups
      continue;
    }
    for (int w2 = 0; w2 < kCtaWarps; ++w2) {
      unsigned todo = hot[w2];  // (the same for every thread)
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int64_t base = toff[w2][src];
        if (base >= p.cap) break;  // later tiles of the group start even later
        const int64_t tl = (g0 + w2) * kCandGroup + src;
        const TileSpan ts(p, tl);
        const int64_t b0 = ts.t0 + warp * seg;
        const int64_t b1 = (b0 + seg < ts.end) ? b0 + seg : ts.end;
        const int cs = (b0 < b1) ? count_span(p, ts, b0, b1, lane) : 0;
        if (lane == 0) segc[warp] = cs;
        __syncthreads();
        int64_t sb = base;
        for (int i = 0; i < warp; ++i) sb += segc[i];
        if (b0 < b1 && cs > 0 && sb < p.cap) write_span(p, ts, b0, b1, lane, sb);
        __syncthreads();  // segc is reused by the next tile
      }
    }
    __syncthreads();  // hot and toff are reused by the next groups
  }
}

}  // namespace

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};  // device address of the scratch, per device
int g_sm_count[kMaxDevices] = {};       // multiprocessors of each device
}  // namespace

// The host-side name g_static_cand_scratch is not a device address: the address
// is looked up with the device current.  Outside a stream capture it is looked
// up on every call (so a context that was torn down and created again gets the
// new address); during a capture the address of the last call outside one is
// used, so the first call on a device must come before any capture.
cudaError_t static_cand_scratch(cudaStream_t s, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* a = nullptr;
    e = cudaGetSymbolAddress(&a, g_static_cand_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = a;
  }
  if (!g_static_addr[dev]) return cudaErrorStreamCaptureUnsupported;
  *out = g_static_addr[dev];
  return cudaSuccess;
}

// Multiprocessor count of the current device, queried on its first use and kept
// (the query is not a stream operation, so capture does not prevent it).
cudaError_t device_sm_count(int* n) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_sm_count[dev]) {
    e = cudaDeviceGetAttribute(&g_sm_count[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  *n = g_sm_count[dev];
  return cudaSuccess;
}

cudaError_t launch_candidates_static(const spd_plan& plan, CandParams& p, cudaStream_t s) {
  void* base = nullptr;
  const cudaError_t e = static_cand_scratch(s, &base);
  if (e != cudaSuccess) return e;
  char* b = static_cast<char*>(base);
  p.counts = reinterpret_cast<int32_t*>(b);
  p.gsum = reinterpret_cast<int32_t*>(b + kStaticCandTiles * sizeof(int32_t));
  p.goff = reinterpret_cast<int64_t*>(b + kStaticCandTiles * sizeof(int32_t) +
                                      (kStaticCandTiles / kCandGroup) * sizeof(int32_t));
  p.tile_max = nullptr;  // no tile maxima without a workspace: every tile is scanned
  return launch_candidates(plan, p, s);
}

cudaError_t launch_candidates(const spd_plan& plan, CandParams& p, cudaStream_t s) {
  const int64_t ntiles = plan.desc.ndm * plan.cand_tiles_per_row;
  const int64_t ngroups = (ntiles + kCandGroup - 1) / kCandGroup;
  int sms = 0;
  cudaError_t e = device_sm_count(&sms);
  if (e != cudaSuccess) return e;
  int64_t ctas = (ngroups + kCandThreads / 32 - 1) / (kCandThreads / 32);
  if (ctas > (int64_t)sms * kCandCtasPerSm) ctas = (int64_t)sms * kCandCtasPerSm;
  cand_count_kernel<<<(unsigned)ctas, kCandThreads, 0, s>>>(p, ntiles, ngroups);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cand_scan_kernel<<<1, kScanThreads, 0, s>>>(p, ngroups);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cand_write_kernel<<<(unsigned)ctas, kCandThreads, 0, s>>>(p, ntiles, ngroups);
  return cudaGetLastError();
}

}  // namespace spd
