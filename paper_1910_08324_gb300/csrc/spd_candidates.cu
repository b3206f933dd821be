// spd_candidates.cu -- threshold + peak-finding candidate selection (sm_103a).
//
// The paper selects candidates from the search output "using a peak-finding
// algorithm" (Sec. 4.5) without defining it.  Rule implemented here: start s of
// a row is a candidate iff Y[s] >= thr, Y[s] > Y[s'] for s - R <= s' < s and
// Y[s] >= Y[s'] for s < s' <= s + R (inside the row); the leftmost sample of a
// plateau wins and R = 0 is a plain threshold.
//
// Deterministic compaction in (row, start) order, three launches:
//   count  -- one CTA per tile counts its candidates (tiles whose maximum SNR,
//             recorded by the search kernel, is below the threshold are
//             skipped without reading them);
//   scan   -- one CTA turns the per-tile counts into int64 offsets and writes
//             the total to *d_count;
//   write  -- tiles with candidates re-test their starts 256 at a time and
//             write their records at offset + block-prefix, keeping the first
//             cap records overall.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "spd_internal.h"

// Scratch of spd_candidates_static: per-tile counts (int32) followed by per-tile
// offsets (int64) for at most kStaticCandTiles candidate tiles (3 MiB).  Every
// device that loads the library holds this array until the process exits; all
// calls on a device share it.
static __device__ __align__(256) unsigned char
    g_static_cand_scratch[spd::kStaticCandTiles * (sizeof(int32_t) + sizeof(int64_t))];

namespace spd {
namespace {

constexpr int kCandThreads = 256;
constexpr int kScanThreads = 1024;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float key_to_float(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

__device__ __forceinline__ bool is_cand(const float* __restrict__ y, int64_t s, int64_t nt,
                                        float thr, int R) {
  const float v = y[s];
  if (!(v >= thr)) return false;
  for (int q = 1; q <= R; ++q) {
    if (s - q >= 0 && !(v > y[s - q])) return false;
    if (s + q < nt && !(v >= y[s + q])) return false;
  }
  return true;
}

__global__ void __launch_bounds__(kCandThreads) cand_count_kernel(const CandParams p) {
  __shared__ int red[kCandThreads / 32];
  const int64_t t = blockIdx.x;
  const int64_t row = t / p.tiles_per_row;
  const int64_t t0 = (t % p.tiles_per_row) * (int64_t)p.tile;
  if (p.tile_max && !(key_to_float(reinterpret_cast<const int*>(p.tile_max)[t]) >= p.thr)) {
    if (threadIdx.x == 0) p.counts[t] = 0;
    return;
  }
  const float* y = p.snr + row * p.ld;
  const int64_t end = (t0 + p.tile < p.nt) ? t0 + p.tile : p.nt;
  int c = 0;
  for (int64_t s = t0 + threadIdx.x; s < end; s += kCandThreads) c += is_cand(y, s, p.nt, p.thr, p.radius) ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int k = 0; k < kCandThreads / 32; ++k) tot += red[k];
    p.counts[t] = tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) cand_scan_kernel(const CandParams p, int64_t ntiles) {
  __shared__ int64_t part[kScanThreads];
  const int64_t per = (ntiles + kScanThreads - 1) / kScanThreads;
  const int64_t a = threadIdx.x * per;
  const int64_t b = (a + per < ntiles) ? a + per : ntiles;
  int64_t s = 0;
  for (int64_t i = a; i < b; ++i) s += p.counts[i];
  part[threadIdx.x] = s;
  __syncthreads();
  // inclusive Hillis-Steele scan of the 1024 partial sums (tiny; once per call)
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const int64_t v = (threadIdx.x >= o) ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = (threadIdx.x > 0) ? part[threadIdx.x - 1] : 0;
  for (int64_t i = a; i < b; ++i) {
    p.offsets[i] = run;
    run += p.counts[i];
  }
  if (threadIdx.x == kScanThreads - 1) *p.d_count = part[kScanThreads - 1];
}

__global__ void __launch_bounds__(kCandThreads) cand_write_kernel(const CandParams p) {
  __shared__ int wsum[kCandThreads / 32];
  const int64_t t = blockIdx.x;
  if (p.counts[t] == 0) return;
  const int64_t row = t / p.tiles_per_row;
  const int64_t t0 = (t % p.tiles_per_row) * (int64_t)p.tile;
  const float* y = p.snr + row * p.ld;
  const uint16_t* w = p.widx + row * p.ld;
  const int64_t end = (t0 + p.tile < p.nt) ? t0 + p.tile : p.nt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t base = p.offsets[t];
  for (int64_t s0 = t0; s0 < end; s0 += kCandThreads) {
    const int64_t s = s0 + threadIdx.x;
    const bool f = (s < end) && is_cand(y, s, p.nt, p.thr, p.radius);
    const unsigned bal = __ballot_sync(kFull, f);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0, tot = 0;
    for (int k = 0; k < kCandThreads / 32; ++k) {
      before += (k < warp) ? wsum[k] : 0;
      tot += wsum[k];
    }
    if (f) {
      const int64_t pos = base + before + __popc(bal & ((1u << lane) - 1u));
      if (pos < p.cap) {
        spd_candidate c;
        c.row = (int32_t)row;
        c.width_idx = (int32_t)w[s];
        c.start = s;
        c.snr = y[s];
        c.width = p.width_mode ? p.width_tab[c.width_idx] : c.width_idx + 1;
        p.out[pos] = c;
      }
    }
    base += tot;
    __syncthreads();
  }
}

}  // namespace

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};  // device address of the scratch, per device
}  // namespace

// The host-side name g_static_cand_scratch is not a device address: the address
// is looked up once per device (with that device current) and cached.
cudaError_t static_cand_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* a = nullptr;
    e = cudaGetSymbolAddress(&a, g_static_cand_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = a;
  }
  *out = g_static_addr[dev];
  return cudaSuccess;
}

cudaError_t launch_candidates_static(const spd_plan& plan, CandParams& p, cudaStream_t s) {
  void* base = nullptr;
  const cudaError_t e = static_cand_scratch(&base);
  if (e != cudaSuccess) return e;
  p.counts = static_cast<int32_t*>(base);
  p.offsets = reinterpret_cast<int64_t*>(static_cast<char*>(base) + kStaticCandTiles * sizeof(int32_t));
  p.tile_max = nullptr;  // no tile maxima without a workspace: every tile is scanned
  return launch_candidates(plan, p, s);
}

cudaError_t launch_candidates(const spd_plan& plan, CandParams& p, cudaStream_t s) {
  const int64_t ntiles = plan.desc.ndm * plan.cand_tiles_per_row;
  cand_count_kernel<<<(unsigned)ntiles, kCandThreads, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cand_scan_kernel<<<1, kScanThreads, 0, s>>>(p, ntiles);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cand_write_kernel<<<(unsigned)ntiles, kCandThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace spd
