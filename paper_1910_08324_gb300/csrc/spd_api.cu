// spd_api.cu -- the C ABI of libspd.so: plan construction (width grids of the
// paper's algorithms), argument validation and kernel launches.  See
// include/spd.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <new>

#include "spd_internal.h"

namespace {

using spd::kBoxdit;
using spd::kExhaustive;
using spd::kIgrid;

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2i(int v) {
  int i = 0;
  while ((2 << i) <= v) ++i;
  return i;
}

// Appends the widths of one level; stops (returns true) once a width >= s_end
// has been appended, recording the top level and how many of its widths count.
bool add_level(spd_plan* p, int level, const int* widths, int n, int sep) {
  p->lvl_first.push_back((int32_t)p->widths.size());
  for (int q = 0; q < n; ++q) {
    p->widths.push_back(widths[q]);
    p->seps.push_back(sep);
    if (widths[q] >= p->desc.s_end) {
      p->top = level;
      p->n_top = q + 1;
      return true;
    }
  }
  return false;
}

// BoxDIT (Alg. 1, D = 2): iteration i has separation 2^i and the widths
// L^{i-1}_MAX + 2^i m, m = 1..k_i, with L^{i-1}_MAX = sum_{j<i} k_j 2^j.  k_i is
// k[i] (the last entry repeats for later iterations; Sec. 3.1 lets L^i_max
// change from iteration to iteration).  n_iter > 0: exactly n_iter full
// iterations; otherwise up to the first width >= s_end.  A plan whose k_i are
// all 8, all 16 or all 32 is streamed by the BD-K kernels (spd_boxdit.cu),
// every other one by the general kernel (spd_boxdit_gen.cu).
spd_status build_boxdit(spd_plan* p, const int32_t* k, int nk, int n_iter) {
  std::vector<int> w;
  int64_t c = 0;
  bool uniform = true;
  for (int i = 0; i < spd::kMaxLevels; ++i) {
    const int ki = k[i < nk ? i : nk - 1];
    uniform = uniform && ki == k[0];
    w.clear();
    for (int m = 1; m <= ki; ++m) {
      const int64_t v = c + ((int64_t)m << i);
      if (v > (1LL << 30)) return SPD_ERR_INVALID_ARG;
      w.push_back((int)v);
    }
    p->lvl_base.push_back((int32_t)c);
    p->lvl_k.push_back(ki);
    bool last;
    if (n_iter > 0) {
      p->lvl_first.push_back((int32_t)p->widths.size());
      for (int q = 0; q < ki; ++q) {
        p->widths.push_back(w[q]);
        p->seps.push_back(1 << i);
      }
      last = i == n_iter - 1;
      if (last) {
        p->top = i;
        p->n_top = ki;
      }
    } else {
      last = add_level(p, i, w.data(), ki, 1 << i);
    }
    if (last) {
      p->bd_general = !(uniform && (k[0] == 8 || k[0] == 16 || k[0] == 32));
      p->k = p->bd_general ? 0 : k[0];
      return SPD_OK;
    }
    c += (int64_t)ki << i;
  }
  return SPD_ERR_INVALID_ARG;
}

bool boxdit_k_ok(int k) { return k >= 2 && k <= spd::kMaxBoxditK && k % 2 == 0; }

// IGRID IG(d) with P = 2^p layers (Sec. 3.2).  Steps 0..p all have boxcar
// separation 2^i / P <= 1, so they form level 0 together: step i contributes
// 2^i + q max(1, 2^(i-d)) for q < 2^min(i, d).  Step p + j (j >= 1) has
// separation 2^j and the widths 2^j (2^p + q 2^(p-d)), q < 2^d.
spd_status build_igrid(spd_plan* p) {
  const int d = p->d, pl = p->pl;
  int w[64];
  int n = 0;
  for (int i = 0; i <= pl; ++i) {
    const int cnt = 1 << (i < d ? i : d);
    const int inc = (i >= d) ? (1 << (i - d)) : 1;
    for (int q = 0; q < cnt; ++q) w[n++] = (1 << i) + q * inc;
  }
  p->lvl_base.push_back(0);
  if (add_level(p, 0, w, n, 1)) return SPD_OK;
  const int mbase = 1 << pl, mstep = 1 << (pl - d), mm = 1 << d;
  for (int j = 1; j < spd::kMaxLevels; ++j) {
    for (int q = 0; q < mm; ++q) {
      const int64_t v = (int64_t)(mbase + q * mstep) << j;
      if (v > (1LL << 30)) return SPD_ERR_INVALID_ARG;
      w[q] = (int)v;
    }
    p->lvl_base.push_back(0);
    if (add_level(p, j, w, mm, 1 << j)) return SPD_OK;
  }
  return SPD_ERR_INVALID_ARG;
}

spd_status check_cuda(cudaError_t e) { return e == cudaSuccess ? SPD_OK : SPD_ERR_CUDA; }

// Streaming kernels: a CTA searches a segment of `segment` starts of a row (a
// multiple of the candidate tile), or the whole row rounded up to candidate
// tiles when that is shorter.
constexpr int kDefaultSegment = 131072;
int segment_tile(int64_t nt, int segment) {
  int64_t T = ((nt + spd::kCandTile - 1) / spd::kCandTile) * spd::kCandTile;
  if (T > segment) T = segment;
  return (int)T;
}
// Default segment of a plan: the longest of 524288, 262144 and 131072 starts that
// still gives at least kTargetCtas CTAs (four waves of 4 CTAs on 152 SMs), so long
// rows re-read less halo per start and few rows still fill the GPU.  (Measured on
// 4096 x 1M rows, IG(1): 131072 -> 10.46 ms, 262144 -> 10.21, 524288 -> 10.13.)
constexpr int64_t kTargetCtas = 2432;
int default_segment(int64_t ndm, int64_t nt) {
  for (int seg = 524288; seg > kDefaultSegment; seg >>= 1)
    if (ndm * ((nt + seg - 1) / seg) >= kTargetCtas) return seg;
  return kDefaultSegment;
}
bool segment_ok(const spd_plan& p, int64_t segment) {
  const int64_t align = (int64_t)1 << (p.top > 14 ? p.top : 14);  // levels above 11 need aligned segments
  return segment >= spd::kCandTile && segment <= ((int64_t)1 << 24) && segment % align == 0;
}

int dtype_size(int dtype) {
  switch (dtype) {
    case SPD_F32: return 4;
    case SPD_F16:
    case SPD_BF16: return 2;
    default: return 1;
  }
}

// Workspace: tile maxima (written by the search, read by the candidate step),
// per-tile candidate counts, per-group sums and offsets, and the level
// statistics of spd_noise_stats.
// General BoxDIT plans above level kBdgSplit also keep the series x^h, the
// bases X^{h-1} and the first kernel's results at level h's starts of every row
// between their two kernels.
struct WsLayout {
  size_t tile_max, counts, gsum, goff, msd, gen, total;
  int64_t gen_ldh;
  explicit WsLayout(const spd_plan& p) {
    const size_t nt = (size_t)(p.desc.ndm * p.cand_tiles_per_row);
    const size_t ng = (nt + spd::kCandGroup - 1) / spd::kCandGroup;
    tile_max = 0;
    counts = align_up(tile_max + nt * sizeof(float));
    gsum = align_up(counts + nt * sizeof(int32_t));
    goff = align_up(gsum + ng * sizeof(int32_t));
    msd = align_up(goff + ng * sizeof(int64_t));
    gen = align_up(msd + spd::msd_state_bytes(p.desc.ndm));
    gen_ldh = spd::bdg_two_part(p) ? spd::bdg_ldh(p.desc.nt, p.tile) : 0;
    // x^h, the bases, and the first kernel's SNRs and widths at level h's starts
    total = align_up(gen + (3 * sizeof(float) + sizeof(uint16_t)) * (size_t)(p.desc.ndm * gen_ldh));
  }
};

spd_status validate_ws(const spd_plan* plan, void* d_ws, size_t ws_bytes) {
  const WsLayout wl(*plan);
  if (ws_bytes < wl.total) return SPD_ERR_WORKSPACE_TOO_SMALL;
  if (!d_ws || ((uintptr_t)d_ws % kAlign) != 0) return SPD_ERR_INVALID_ARG;
  return SPD_OK;
}

// Grid constants of the search kernels (levels, widths, scale tables).
void fill_grid(spd::SearchParams& p, const spd_plan& plan) {
  p.dtype = plan.desc.dtype;
  p.esize = dtype_size(plan.desc.dtype);
  p.halo = plan.halo;
  p.top = plan.top;
  p.n_top = plan.n_top;
  p.lmax = plan.lend;
  for (size_t j = 0; j < plan.lvl_first.size() && j < (size_t)spd::kMaxLevels; ++j) {
    p.lvl_first[j] = plan.lvl_first[j];
    p.lvl_scale[j] = (float)std::pow(2.0, -0.5 * (double)j);
  }
  for (int m = 1; m < 64; ++m) p.rs[m] = (float)(1.0 / std::sqrt((double)m));
  p.n_widths = (int32_t)plan.widths.size();
  p.unit_widths = (plan.family == kExhaustive && !plan.explicit_grid) ? 1 : 0;
  if (!p.unit_widths)
    for (size_t i = 0; i < plan.widths.size() && i < (size_t)spd::kMaxGridWidths; ++i) p.wtab[i] = plan.widths[i];
  p.grid = plan.explicit_grid ? 1 : 0;
  if (plan.explicit_grid)
    for (size_t i = 0; i < plan.seps.size() && i < (size_t)spd::kMaxGridWidths; ++i) p.wsep[i] = plan.seps[i];
  if (plan.family == kBoxdit && plan.bd_general) {
    for (int j = 0; j <= plan.top; ++j) p.lvl_k[j] = plan.lvl_k[j];
    spd::bdg_layout(plan, plan.tile, true, p.gen_len, p.gen_off);
    p.gen_h = spd::kBdgSplit;
    for (size_t i = 0; i < plan.widths.size() && i < (size_t)spd::kMaxGridWidths; ++i)
      p.wscale[i] = (float)(1.0 / std::sqrt((double)plan.widths[i]));
  } else if (plan.family == kBoxdit) {
    for (int j = 0; j <= plan.top; ++j)
      for (int m = 1; m <= plan.k; ++m)
        p.bscale[j][m] = (float)(1.0 / std::sqrt((double)plan.lvl_base[j] + (double)m * (double)(1 << j)));
  } else if (plan.family == kIgrid) {  // 1/sqrt(m 2^j) in one constant (block count m of level j)
    for (int j = 0; j <= plan.top && j < spd::kMaxLevels; ++j)
      for (int m = 1; m <= 32; ++m) p.bscale[j][m] = (float)(1.0 / std::sqrt((double)m * (double)(1 << j)));
  }
}

spd_status do_execute(const spd_plan* plan, const void* d_x, const spd_noise* noise, float* d_snr,
                      uint16_t* d_width_idx, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
  if (!plan || !d_x || !noise || !d_snr || !d_width_idx) return SPD_ERR_INVALID_ARG;
  if (noise->mode != 0 && noise->mode != 1) return SPD_ERR_INVALID_ARG;
  if (!noise->mu || !noise->sigma || ((uintptr_t)noise->mu % 4) || ((uintptr_t)noise->sigma % 4))
    return SPD_ERR_INVALID_ARG;
  const int esize = dtype_size(plan->desc.dtype);
  if (((uintptr_t)d_x % esize) || ((uintptr_t)d_snr % 4) || ((uintptr_t)d_width_idx % 2))
    return SPD_ERR_INVALID_ARG;
  const spd_status ws = validate_ws(plan, d_ws, ws_bytes);
  if (ws != SPD_OK) return ws;
  const WsLayout wl(*plan);
  spd::SearchParams* sp = new (std::nothrow) spd::SearchParams();
  if (!sp) return SPD_ERR_HOST_ALLOC;
  spd::SearchParams& p = *sp;
  p.x = d_x;
  p.vec_x = ((uintptr_t)d_x % 16 == 0 && (plan->desc.ld * esize) % 16 == 0) ? 1 : 0;
  p.snr = d_snr;
  p.widx = d_width_idx;
  p.tile_max = reinterpret_cast<float*>(static_cast<char*>(d_ws) + wl.tile_max);
  p.mu = noise->mu;
  p.sigma = noise->sigma;
  p.ndm = plan->desc.ndm;
  p.nt = plan->desc.nt;
  p.n_starts = plan->n_starts;
  p.ld = plan->desc.ld;
  p.tile = plan->tile;
  p.tiles_per_row = (int32_t)plan->tiles_per_row;
  p.cand_tiles_per_row = (int32_t)plan->cand_tiles_per_row;
  p.vec = ((uintptr_t)d_snr % 16 == 0 && (uintptr_t)d_width_idx % 8 == 0 && plan->desc.ld % 4 == 0)
              ? 1
              : 0;
  fill_grid(p, *plan);
  if (wl.gen_ldh > 0) {
    p.gen_xh = reinterpret_cast<float*>(static_cast<char*>(d_ws) + wl.gen);
    p.gen_bh = p.gen_xh + plan->desc.ndm * wl.gen_ldh;
    p.gen_yh = p.gen_bh + plan->desc.ndm * wl.gen_ldh;
    p.gen_wh = reinterpret_cast<uint16_t*>(p.gen_yh + plan->desc.ndm * wl.gen_ldh);
    p.gen_ldh = wl.gen_ldh;
  }
  p.table = noise->mode == 1 ? 1 : 0;
  // tile maxima start at a key below every float (0x80808080)
  cudaError_t e = cudaMemsetAsync(p.tile_max, 0x80,
                                  sizeof(float) * (size_t)(plan->desc.ndm * plan->cand_tiles_per_row),
                                  stream);
  if (e == cudaSuccess) e = spd::launch_search(*plan, p, stream);
  delete sp;
  return check_cuda(e);
}

spd_status check_cand_args(const spd_plan* plan, const float* d_snr, const uint16_t* d_width_idx,
                           float threshold, int32_t peak_radius, spd_candidate* d_out, int64_t cap,
                           int64_t* d_count) {
  if (!plan || !d_snr || !d_width_idx || !d_count) return SPD_ERR_INVALID_ARG;
  if (cap < 0 || (cap > 0 && !d_out)) return SPD_ERR_INVALID_ARG;
  if (peak_radius < 0 || peak_radius > spd::kMaxPeakRadius) return SPD_ERR_INVALID_ARG;
  if (std::isnan(threshold)) return SPD_ERR_INVALID_ARG;
  if (((uintptr_t)d_count % 8) || ((uintptr_t)d_out % 8)) return SPD_ERR_INVALID_ARG;
  return SPD_OK;
}

// Fills everything but the scratch pointers (counts, gsum, goff, tile_max).
void fill_cand_params(spd::CandParams& p, const spd_plan* plan, const float* d_snr,
                      const uint16_t* d_width_idx, float threshold, int32_t peak_radius,
                      spd_candidate* d_out, int64_t cap, int64_t* d_count) {
  p.snr = d_snr;
  p.widx = d_width_idx;
  p.out = d_out;
  p.d_count = d_count;
  p.ndm = plan->desc.ndm;
  p.nt = plan->n_starts;  // the candidate step's extent: the evaluated starts
  p.ld = plan->desc.ld;
  p.cap = cap;
  p.tile = spd::kCandTile;
  p.tiles_per_row = (int32_t)plan->cand_tiles_per_row;
  p.radius = peak_radius;
  p.thr = threshold;
  p.width_mode = (plan->family == kExhaustive && !plan->explicit_grid) ? 0 : 1;
  if (p.width_mode)
    for (size_t i = 0; i < plan->widths.size() && i < 512; ++i) p.width_tab[i] = plan->widths[i];
  p.s_lo = 0;
  p.s_hi = p.nt;
  p.row_ids = nullptr;
  p.map_bpr = 1;
  p.map_nt = 0;
  p.map_block = 0;
}

// Candidate window and block map of a proposal search (CandParams).
struct BlockMap {
  int64_t s_lo, s_hi;
  const int64_t* ids;
  int64_t bpr, nt;
  int32_t block;
};

spd_status do_candidates(const spd_plan* plan, const float* d_snr, const uint16_t* d_width_idx,
                         float threshold, int32_t peak_radius, spd_candidate* d_out, int64_t cap,
                         int64_t* d_count, void* d_ws, size_t ws_bytes, bool use_tile_max,
                         cudaStream_t stream, const BlockMap* map = nullptr) {
  spd_status st = check_cand_args(plan, d_snr, d_width_idx, threshold, peak_radius, d_out, cap, d_count);
  if (st != SPD_OK) return st;
  st = validate_ws(plan, d_ws, ws_bytes);
  if (st != SPD_OK) return st;
  const WsLayout wl(*plan);
  spd::CandParams* cp = new (std::nothrow) spd::CandParams();
  if (!cp) return SPD_ERR_HOST_ALLOC;
  spd::CandParams& p = *cp;
  fill_cand_params(p, plan, d_snr, d_width_idx, threshold, peak_radius, d_out, cap, d_count);
  char* base = static_cast<char*>(d_ws);
  p.tile_max = use_tile_max ? reinterpret_cast<const float*>(base + wl.tile_max) : nullptr;
  p.counts = reinterpret_cast<int32_t*>(base + wl.counts);
  p.gsum = reinterpret_cast<int32_t*>(base + wl.gsum);
  p.goff = reinterpret_cast<int64_t*>(base + wl.goff);
  if (map) {
    p.s_lo = map->s_lo;
    p.s_hi = map->s_hi;
    p.row_ids = map->ids;
    p.map_bpr = map->bpr;
    p.map_nt = map->nt;
    p.map_block = map->block;
  }
  const cudaError_t e = spd::launch_candidates(*plan, p, stream);
  delete cp;
  return check_cuda(e);
}

}  // namespace

// A batch: ranges of one grid (spd_batch_create).
struct spd_batch {
  spd_plan grid;  // the shared grid (desc.ndm 1, desc.nt the longest range)
  int32_t n;
  int64_t ndm[spd::kMaxRanges], nt[spd::kMaxRanges], ld[spd::kMaxRanges];
  int32_t segment;
  int64_t wait_ns;
  int32_t ctas_per_sm = 0;  // persistent CTAs per SM of spd_batch_execute (0: as many as fit)
};

namespace {

struct BatchLayout {  // workspace of a batch
  size_t status, tile_max[spd::kMaxRanges], counts, gsum, goff, total;
  explicit BatchLayout(const spd_batch& b) {
    size_t o = 0;
    status = o;
    o = align_up(o + sizeof(int32_t));
    size_t maxt = 0;
    for (int r = 0; r < b.n; ++r) {
      const size_t nt = (size_t)(b.ndm[r] * ((b.nt[r] + spd::kCandTile - 1) / spd::kCandTile));
      tile_max[r] = o;
      o = align_up(o + nt * sizeof(float));
      maxt = nt > maxt ? nt : maxt;
    }
    const size_t ng = (maxt + spd::kCandGroup - 1) / spd::kCandGroup;
    counts = o;
    gsum = align_up(counts + maxt * sizeof(int32_t));
    goff = align_up(gsum + ng * sizeof(int32_t));
    total = align_up(goff + ng * sizeof(int64_t));
  }
};

// The single-series view of range r (for the candidate step).
spd_plan range_plan(const spd_batch& b, int r) {
  spd_plan p = b.grid;
  p.desc.ndm = b.ndm[r];
  p.desc.nt = b.nt[r];
  p.desc.ld = b.ld[r];
  p.tile = b.grid.bd_general ? b.grid.tile : segment_tile(b.nt[r], b.segment);
  p.n_starts = b.nt[r];
  p.tiles_per_row = (b.nt[r] + p.tile - 1) / p.tile;
  p.cand_tiles_per_row = (b.nt[r] + spd::kCandTile - 1) / spd::kCandTile;
  return p;
}

}  // namespace

namespace spd {
cudaError_t persistent_config(const void* kernel, size_t smem, int* per_sm, int* sms, int threads) {
  struct Entry {
    const void* k;
    int dev;
    size_t smem;
    int threads, per_sm, sms;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& c : cache)
      if (c.k == kernel && c.dev == dev && c.smem == smem && c.threads == threads) {
        *per_sm = c.per_sm;
        *sms = c.sms;
        return cudaSuccess;
      }
  }
  Entry c{kernel, dev, smem, threads, 0, 0};
  if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  if ((e = cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.per_sm, kernel, threads, smem)) != cudaSuccess)
    return e;
  std::lock_guard<std::mutex> lock(mu);
  cache.push_back(c);
  *per_sm = c.per_sm;
  *sms = c.sms;
  return cudaSuccess;
}
}  // namespace spd

namespace {
// Geometry common to every plan (widest width, tiles, halo, limits); takes
// ownership of p.
spd_status finish_plan(spd_plan* p, spd_plan** out) {
  const spd_plan_desc& d = p->desc;
  p->lend = p->widths.back();
  if (p->lend > spd::kMaxLend || p->widths.size() > 65535 ||
      (p->family != kExhaustive && p->widths.size() > (size_t)spd::kMaxGridWidths) ||
      p->top >= spd::kMaxLevels) {
    delete p;
    return SPD_ERR_INVALID_ARG;
  }
  if (p->family == kExhaustive) {
    p->tile = spd::kChunk;
    p->halo = 0;
  } else {
    // BoxDIT and IGRID: one CTA streams a segment of 131072 to 524288 starts (a
    // multiple of the candidate tile; default_segment); the halo is the widest
    // boxcar, rounded to whole chunks
    if (p->family == kBoxdit && !p->bd_general && p->top > 11) {  // unreachable below kMaxLend
      delete p;
      return SPD_ERR_UNSUPPORTED;
    }
    // IGRID with depth <= 1 and <= 4 layers carries width indices in 5 SNR bits
    // (at most 31 widths below kMaxLend)
    if (p->family == kIgrid && p->d <= 1 && p->pl <= 2 && p->widths.size() > 32) {
      delete p;
      return SPD_ERR_UNSUPPORTED;
    }
    p->tile = segment_tile(d.nt, default_segment(d.ndm, d.nt));
    p->halo = ((p->lend + spd::kChunk - 1) / spd::kChunk) * spd::kChunk;
    if (p->bd_general) {
      // tiles of 4096 starts when two CTAs still fit on an SM, else 2048 (plans
      // above level kBdgSplit: the first of their two kernels)
      int32_t len[spd::kMaxLevels], off[spd::kBdgOffsets];
      p->tile = 4096;
      if (spd::bdg_two_part(*p)) {
        if (sizeof(float) * (size_t)spd::bdg_layout(*p, 4096, true, len, off, 1, spd::kBdgSplit) > 113 * 1024)
          p->tile = 2048;
      } else if (sizeof(float) * (size_t)spd::bdg_layout(*p, 4096, true, len, off) > 113 * 1024) {
        p->tile = 2048;
      }
      p->halo = p->lend;
    }
  }
  p->n_starts = d.nt;
  p->tiles_per_row = (d.nt + p->tile - 1) / p->tile;
  p->cand_tiles_per_row = (d.nt + spd::kCandTile - 1) / spd::kCandTile;
  if (p->desc.ndm * p->tiles_per_row > ((int64_t)1 << 31) - 1 ||
      spd::search_smem_bytes(*p, true) > 227 * 1024) {
    delete p;
    return SPD_ERR_UNSUPPORTED;
  }
  *out = p;
  return SPD_OK;
}
}  // namespace

// A proposal search (spd_propose_search): the network flags 4096-sample blocks
// of the series; the flagged blocks, each with `left` samples before it and the
// widest boxcar after it, are copied into compact rows of `width` samples
// (stride ld_c) and searched with `plan` (rows: up to max_blocks).
struct spd_proposal {
  spd_plan plan;       // the grid over compact rows (desc.ndm = max_blocks)
  spd_plan_desc src;   // the series (ndm, nt, ld, dtype)
  int32_t radius, left, width;
  int64_t ld_c, max_blocks, bpr;
};

namespace {
constexpr int kPropBlock = 4096;  // input samples per block
constexpr int kPropDec = 16;      // the network reads blocks decimated x16

struct PropLayout {  // workspace of a proposal search
  size_t dec, logits, ids, cnt, mu0, sg0, xc, yc, wc, muc, sgc, ws, ws_bytes, total;
  explicit PropLayout(const spd_proposal& q) {
    const int64_t ndm = q.src.ndm, nblk = ndm * q.bpr, mb = q.max_blocks;
    const size_t nw = q.plan.widths.size();
    const size_t rows = (size_t)mb * (size_t)q.ld_c;
    size_t o = 0;
    dec = o;
    o = align_up(o + (size_t)ndm * (size_t)(q.src.nt / kPropDec) * sizeof(float));
    logits = o;
    o = align_up(o + (size_t)nblk * sizeof(float));
    ids = o;
    o = align_up(o + (size_t)nblk * sizeof(int64_t));
    cnt = o;
    o = align_up(o + sizeof(int64_t));
    mu0 = o;
    o = align_up(o + (size_t)ndm * sizeof(float));
    sg0 = o;
    o = align_up(o + (size_t)ndm * sizeof(float));
    xc = o;
    o = align_up(o + rows * (size_t)dtype_size(q.src.dtype));
    yc = o;
    o = align_up(o + rows * sizeof(float));
    wc = o;
    o = align_up(o + rows * sizeof(uint16_t));
    muc = o;
    o = align_up(o + (size_t)mb * nw * sizeof(float));
    sgc = o;
    o = align_up(o + (size_t)mb * nw * sizeof(float));
    ws = o;
    ws_bytes = WsLayout(q.plan).total;
    total = align_up(o + ws_bytes);
  }
};
}  // namespace

extern "C" {

const char* spd_status_string(spd_status s) {
  switch (s) {
    case SPD_OK: return "ok";
    case SPD_ERR_INVALID_ARG: return "invalid argument";
    case SPD_ERR_UNSUPPORTED: return "unsupported in this build";
    case SPD_ERR_CUDA: return "CUDA error";
    case SPD_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case SPD_ERR_BUFFER_TOO_SMALL: return "buffer too small";
    case SPD_ERR_TIMEOUT: return "device wait timed out";
    case SPD_ERR_HOST_ALLOC: return "host allocation failed";
  }
  return "unknown status";
}

const char* spd_version(void) { return "0.1"; }

spd_status spd_plan_create(const spd_plan_desc* desc, spd_plan** out) {
  if (!out) return SPD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc) return SPD_ERR_INVALID_ARG;
  const spd_plan_desc& d = *desc;
  if (d.ndm < 1 || d.nt < 1 || d.ld < d.nt || d.s_end < 1) return SPD_ERR_INVALID_ARG;
  if (d.ndm > (int64_t)1 << 24 || d.nt > (int64_t)1 << 40) return SPD_ERR_INVALID_ARG;
  if (d.dtype < SPD_F32 || d.dtype > SPD_U8) return SPD_ERR_INVALID_ARG;
  if (d.algo < SPD_ALGO_EXHAUSTIVE || d.algo > SPD_ALGO_IGRID) return SPD_ERR_INVALID_ARG;
  spd_plan* p = new (std::nothrow) spd_plan();
  if (!p) return SPD_ERR_HOST_ALLOC;
  p->desc = d;
  spd_status st = SPD_OK;
  try {
    if (d.algo == SPD_ALGO_EXHAUSTIVE) {
      if (d.s_end > spd::kMaxExhaustive) {
        st = SPD_ERR_INVALID_ARG;
      } else {
        p->family = kExhaustive;
        for (int w = 1; w <= d.s_end; ++w) {
          p->widths.push_back(w);
          p->seps.push_back(1);
        }
        p->lvl_first.push_back(0);
        p->lvl_base.push_back(0);
        p->top = 0;
        p->n_top = d.s_end;
      }
    } else if (d.algo == SPD_ALGO_BOXDIT) {
      if (!boxdit_k_ok(d.boxdit_lmax)) {
        st = SPD_ERR_INVALID_ARG;
      } else {
        p->family = kBoxdit;
        st = build_boxdit(p, &d.boxdit_lmax, 1, 0);
      }
    } else {
      const int dd = d.igrid_depth, P = d.igrid_layers;
      if (dd < 0 || dd > 3 || !is_pow2(P) || P < (1 << dd) || P > (2 << dd)) {
        st = SPD_ERR_INVALID_ARG;
      } else {
        p->family = kIgrid;
        p->d = dd;
        p->pl = ilog2i(P);
        st = build_igrid(p);
      }
    }
  } catch (const std::bad_alloc&) {
    st = SPD_ERR_HOST_ALLOC;
  }
  if (st != SPD_OK) {
    delete p;
    return st;
  }
  return finish_plan(p, out);
}

spd_status spd_plan_create_boxdit(const spd_plan_desc* desc, const int32_t* lmax, int32_t n_lmax,
                                  int32_t n_iter, spd_plan** out) {
  if (!out) return SPD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || !lmax || n_lmax < 1 || n_lmax > spd::kMaxLevels || n_iter < 0 || n_iter > spd::kMaxLevels)
    return SPD_ERR_INVALID_ARG;
  const spd_plan_desc& d = *desc;
  if (d.ndm < 1 || d.nt < 1 || d.ld < d.nt || (n_iter == 0 && d.s_end < 1)) return SPD_ERR_INVALID_ARG;
  if (d.ndm > (int64_t)1 << 24 || d.nt > (int64_t)1 << 40) return SPD_ERR_INVALID_ARG;
  if (d.dtype < SPD_F32 || d.dtype > SPD_U8) return SPD_ERR_INVALID_ARG;
  for (int32_t i = 0; i < n_lmax; ++i)
    if (!boxdit_k_ok(lmax[i])) return SPD_ERR_INVALID_ARG;
  spd_plan* p = new (std::nothrow) spd_plan();
  if (!p) return SPD_ERR_HOST_ALLOC;
  p->desc = d;
  p->desc.algo = SPD_ALGO_BOXDIT;
  p->desc.boxdit_lmax = lmax[0];
  if (n_iter > 0) p->desc.s_end = 1;  // not used: the iteration count decides the grid
  spd_status st = SPD_OK;
  try {
    p->family = kBoxdit;
    st = build_boxdit(p, lmax, n_lmax, n_iter);
  } catch (const std::bad_alloc&) {
    st = SPD_ERR_HOST_ALLOC;
  }
  if (st != SPD_OK) {
    delete p;
    return st;
  }
  if (n_iter > 0) p->desc.s_end = p->widths.back();
  return finish_plan(p, out);
}

spd_status spd_plan_create_grid(const spd_plan_desc* desc, const int32_t* widths, const int32_t* seps,
                                int32_t n_widths, spd_plan** out) {
  if (!out) return SPD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || !widths || !seps || n_widths < 1 || n_widths > spd::kMaxGridWidths) return SPD_ERR_INVALID_ARG;
  const spd_plan_desc& d = *desc;
  if (d.ndm < 1 || d.nt < 1 || d.ld < d.nt || d.ndm > (int64_t)1 << 24 || d.nt > (int64_t)1 << 40)
    return SPD_ERR_INVALID_ARG;
  if (d.dtype < SPD_F32 || d.dtype > SPD_U8) return SPD_ERR_INVALID_ARG;
  if (widths[0] != 1 || seps[0] != 1) return SPD_ERR_INVALID_ARG;  // width 1 at every start
  for (int32_t i = 0; i < n_widths; ++i) {
    if (widths[i] < 1 || widths[i] > spd::kMaxExhaustive || (i > 0 && widths[i] <= widths[i - 1]))
      return SPD_ERR_INVALID_ARG;
    if (seps[i] < 1 || seps[i] > spd::kMaxExhaustive || !is_pow2(seps[i])) return SPD_ERR_INVALID_ARG;
  }
  spd_plan* p = new (std::nothrow) spd_plan();
  if (!p) return SPD_ERR_HOST_ALLOC;
  p->desc = d;
  p->desc.algo = SPD_ALGO_EXHAUSTIVE;
  p->desc.s_end = widths[n_widths - 1];
  try {
    p->family = kExhaustive;
    p->explicit_grid = true;
    p->widths.assign(widths, widths + n_widths);
    p->seps.assign(seps, seps + n_widths);
    p->lvl_first.push_back(0);
    p->lvl_base.push_back(0);
  } catch (const std::bad_alloc&) {
    delete p;
    return SPD_ERR_HOST_ALLOC;
  }
  p->top = 0;
  p->n_top = n_widths;
  return finish_plan(p, out);
}

spd_status spd_plan_destroy(spd_plan* plan) {
  delete plan;
  return SPD_OK;
}

spd_status spd_plan_widths(const spd_plan* plan, int32_t* widths, int32_t* seps, int32_t cap,
                           int32_t* n) {
  if (!plan || !n) return SPD_ERR_INVALID_ARG;
  const int32_t cnt = (int32_t)plan->widths.size();
  *n = cnt;
  if (!widths && !seps) return SPD_OK;
  if (cap < cnt) return SPD_ERR_BUFFER_TOO_SMALL;
  for (int32_t i = 0; i < cnt; ++i) {
    if (widths) widths[i] = plan->widths[i];
    if (seps) seps[i] = plan->seps[i];
  }
  return SPD_OK;
}

spd_status spd_workspace_size(const spd_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return SPD_ERR_INVALID_ARG;
  *bytes = WsLayout(*plan).total;
  return SPD_OK;
}

spd_status spd_execute(const spd_plan* plan, const void* d_x, const spd_noise* noise, float* d_snr,
                       uint16_t* d_width_idx, void* d_ws, size_t ws_bytes, spd_stream_t stream) {
  return do_execute(plan, d_x, noise, d_snr, d_width_idx, d_ws, ws_bytes,
                    reinterpret_cast<cudaStream_t>(stream));
}

spd_status spd_candidates(const spd_plan* plan, const float* d_snr, const uint16_t* d_width_idx,
                          float threshold, int32_t peak_radius, spd_candidate* d_out, int64_t cap,
                          int64_t* d_count, void* d_ws, size_t ws_bytes, int32_t use_tile_max,
                          spd_stream_t stream) {
  return do_candidates(plan, d_snr, d_width_idx, threshold, peak_radius, d_out, cap, d_count, d_ws,
                       ws_bytes, use_tile_max != 0, reinterpret_cast<cudaStream_t>(stream));
}

spd_status spd_candidates_static(const spd_plan* plan, const float* d_snr,
                                 const uint16_t* d_width_idx, float threshold, int32_t peak_radius,
                                 spd_candidate* d_out, int64_t cap, int64_t* d_count,
                                 spd_stream_t stream) {
  spd_status st = check_cand_args(plan, d_snr, d_width_idx, threshold, peak_radius, d_out, cap, d_count);
  if (st != SPD_OK) return st;
  if (plan->desc.ndm * plan->cand_tiles_per_row > spd::kStaticCandTiles) return SPD_ERR_UNSUPPORTED;
  spd::CandParams* cp = new (std::nothrow) spd::CandParams();
  if (!cp) return SPD_ERR_HOST_ALLOC;
  fill_cand_params(*cp, plan, d_snr, d_width_idx, threshold, peak_radius, d_out, cap, d_count);
  const cudaError_t e = spd::launch_candidates_static(*plan, *cp, reinterpret_cast<cudaStream_t>(stream));
  delete cp;
  return check_cuda(e);
}

spd_status spd_search(const spd_plan* plan, const void* d_x, const spd_noise* noise, float* d_snr,
                      uint16_t* d_width_idx, float threshold, int32_t peak_radius,
                      spd_candidate* d_out, int64_t cap, int64_t* d_count, void* d_ws,
                      size_t ws_bytes, spd_stream_t stream) {
  // validate the candidate arguments before queueing the search
  if (!d_count || cap < 0 || (cap > 0 && !d_out) || peak_radius < 0 ||
      peak_radius > spd::kMaxPeakRadius || std::isnan(threshold))
    return SPD_ERR_INVALID_ARG;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const spd_status st = do_execute(plan, d_x, noise, d_snr, d_width_idx, d_ws, ws_bytes, s);
  if (st != SPD_OK) return st;
  return do_candidates(plan, d_snr, d_width_idx, threshold, peak_radius, d_out, cap, d_count, d_ws,
                       ws_bytes, true, s);
}

spd_status spd_noise_stats(const spd_plan* plan, const void* d_x, float outlier_sigma,
                           int32_t max_passes, float* d_mu, float* d_sigma, void* d_ws,
                           size_t ws_bytes, spd_stream_t stream) {
  if (!plan || !d_x || !d_mu || !d_sigma) return SPD_ERR_INVALID_ARG;
  if (max_passes < 1 || max_passes > 64 || std::isnan(outlier_sigma) || std::isinf(outlier_sigma))
    return SPD_ERR_INVALID_ARG;
  const int esize = dtype_size(plan->desc.dtype);
  if (((uintptr_t)d_x % esize) || ((uintptr_t)d_mu % 4) || ((uintptr_t)d_sigma % 4))
    return SPD_ERR_INVALID_ARG;
  spd_status st = validate_ws(plan, d_ws, ws_bytes);
  if (st != SPD_OK) return st;
  spd::MsdParams* mp = new (std::nothrow) spd::MsdParams();
  if (!mp) return SPD_ERR_HOST_ALLOC;
  spd::MsdParams& p = *mp;
  p.x = d_x;
  p.ndm = plan->desc.ndm;
  p.nt = plan->desc.nt;
  p.ld = plan->desc.ld;
  p.dtype = plan->desc.dtype;
  p.esize = esize;
  p.vec_x = ((uintptr_t)d_x % 16 == 0 && (plan->desc.ld * esize) % 16 == 0) ? 1 : 0;
  int nlev = 1;
  while (nlev < spd::kMsdMaxLevels && (1 << (nlev - 1)) < plan->lend) ++nlev;
  p.nlev = nlev;
  p.thr = outlier_sigma;
  p.state = static_cast<char*>(d_ws) + WsLayout(*plan).msd;
  p.out_mu = d_mu;
  p.out_sigma = d_sigma;
  p.n_widths = (int32_t)plan->widths.size();
  p.unit_widths = (plan->family == kExhaustive && !plan->explicit_grid) ? 1 : 0;
  if (!p.unit_widths)
    for (size_t i = 0; i < plan->widths.size() && i < (size_t)spd::kMaxGridWidths; ++i)
      p.wtab[i] = plan->widths[i];
  const cudaError_t e = spd::launch_msd(*plan, p, max_passes, reinterpret_cast<cudaStream_t>(stream));
  delete mp;
  return check_cuda(e);
}

spd_status spd_plan_set_segment(spd_plan* plan, int32_t segment) {
  if (plan && plan->bd_general) {  // the general BoxDIT kernel: tiles of 2048, 4096 or 8192 starts
    if (segment != 2048 && segment != 4096 && segment != 8192) return SPD_ERR_INVALID_ARG;
    // plans above level kBdgSplit run levels 0.. kBdgSplit - 1 on these tiles
    // (the rest on tiles of their own), the others every level
    const int32_t old_tile = plan->tile;
    plan->tile = segment;
    int32_t len[spd::kMaxLevels], off[spd::kBdgOffsets];
    if (!spd::bdg_two_part(*plan) &&
        sizeof(float) * (size_t)spd::bdg_layout(*plan, segment, true, len, off) > spd::kBdgMaxSmem) {
      plan->tile = old_tile;
      return SPD_ERR_UNSUPPORTED;
    }
    plan->tiles_per_row = (plan->n_starts + plan->tile - 1) / plan->tile;
    return SPD_OK;
  }
  if (!plan || plan->family == kExhaustive || !segment_ok(*plan, segment)) return SPD_ERR_INVALID_ARG;
  plan->tile = segment_tile(plan->desc.nt, segment);
  plan->tiles_per_row = (plan->n_starts + plan->tile - 1) / plan->tile;
  return SPD_OK;
}

spd_status spd_plan_set_starts(spd_plan* plan, int64_t n_starts) {
  if (!plan || n_starts < 1 || n_starts > plan->desc.nt) return SPD_ERR_INVALID_ARG;
  plan->n_starts = n_starts;
  plan->tiles_per_row = (n_starts + plan->tile - 1) / plan->tile;  // CTAs of the search per row
  return SPD_OK;
}

spd_status spd_batch_create(const spd_plan_desc* grid, const int64_t* ndm, const int64_t* nt,
                            const int64_t* ld, int32_t n_ranges, spd_batch** out) {
  if (!out) return SPD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!grid || !ndm || !nt || n_ranges < 1 || n_ranges > spd::kMaxRanges) return SPD_ERR_INVALID_ARG;
  if (grid->algo == SPD_ALGO_EXHAUSTIVE) return SPD_ERR_UNSUPPORTED;
  int64_t ntmax = 0, units = 0;
  for (int r = 0; r < n_ranges; ++r) {
    const int64_t l = ld ? ld[r] : nt[r];
    if (ndm[r] < 1 || nt[r] < 1 || l < nt[r] || ndm[r] > ((int64_t)1 << 24) || nt[r] > ((int64_t)1 << 40))
      return SPD_ERR_INVALID_ARG;
    ntmax = nt[r] > ntmax ? nt[r] : ntmax;
  }
  spd_plan_desc d = *grid;
  d.ndm = 1;
  d.nt = ntmax;
  d.ld = ntmax;
  spd_plan* g = nullptr;
  spd_status st = spd_plan_create(&d, &g);
  if (st != SPD_OK) return st;
  spd_batch* b = new (std::nothrow) spd_batch();
  if (!b) {
    spd_plan_destroy(g);
    return SPD_ERR_HOST_ALLOC;
  }
  b->grid = *g;
  spd_plan_destroy(g);
  b->n = n_ranges;
  b->segment = kDefaultSegment;
  b->wait_ns = 1000000000LL;
  for (int r = 0; r < n_ranges; ++r) {
    b->ndm[r] = ndm[r];
    b->nt[r] = nt[r];
    b->ld[r] = ld ? ld[r] : nt[r];
    units += ndm[r] * ((nt[r] + segment_tile(nt[r], b->segment) - 1) / segment_tile(nt[r], b->segment));
  }
  if (units > ((int64_t)1 << 40)) {
    delete b;
    return SPD_ERR_INVALID_ARG;
  }
  *out = b;
  return SPD_OK;
}

spd_status spd_batch_destroy(spd_batch* batch) {
  delete batch;
  return SPD_OK;
}

spd_status spd_batch_set_segment(spd_batch* batch, int32_t segment) {
  if (!batch || !segment_ok(batch->grid, segment)) return SPD_ERR_INVALID_ARG;
  batch->segment = segment;
  return SPD_OK;
}

spd_status spd_batch_set_wait_ns(spd_batch* batch, int64_t wait_ns) {
  if (!batch || wait_ns < 0 || wait_ns > 60000000000LL) return SPD_ERR_INVALID_ARG;
  batch->wait_ns = wait_ns;
  return SPD_OK;
}

spd_status spd_batch_set_ctas_per_sm(spd_batch* batch, int32_t ctas_per_sm) {
  if (!batch || ctas_per_sm < 0 || ctas_per_sm > 64) return SPD_ERR_INVALID_ARG;
  batch->ctas_per_sm = ctas_per_sm;
  return SPD_OK;
}

spd_status spd_batch_workspace_size(const spd_batch* batch, size_t* bytes) {
  if (!batch || !bytes) return SPD_ERR_INVALID_ARG;
  *bytes = BatchLayout(*batch).total;
  return SPD_OK;
}

spd_status spd_batch_execute(const spd_batch* batch, const spd_range_io* io, void* d_ws, size_t ws_bytes,
                             spd_stream_t stream) {
  if (!batch || !io) return SPD_ERR_INVALID_ARG;
  const BatchLayout bl(*batch);
  if (ws_bytes < bl.total) return SPD_ERR_WORKSPACE_TOO_SMALL;
  if (!d_ws || ((uintptr_t)d_ws % kAlign) != 0) return SPD_ERR_INVALID_ARG;
  const spd_plan& g = batch->grid;
  const int esize = dtype_size(g.desc.dtype);
  for (int r = 0; r < batch->n; ++r) {
    const spd_range_io& a = io[r];
    if (!a.d_x || !a.d_snr || !a.d_width_idx || !a.d_mu || !a.d_sigma) return SPD_ERR_INVALID_ARG;
    if (((uintptr_t)a.d_x % esize) || ((uintptr_t)a.d_snr % 4) || ((uintptr_t)a.d_width_idx % 2) ||
        ((uintptr_t)a.d_mu % 4) || ((uintptr_t)a.d_sigma % 4) || ((uintptr_t)a.d_ready % 4))
      return SPD_ERR_INVALID_ARG;
  }
  spd::SearchParams* sp = new (std::nothrow) spd::SearchParams();
  if (!sp) return SPD_ERR_HOST_ALLOC;
  spd::SearchParams& p = *sp;
  fill_grid(p, g);
  p.table = 0;
  p.n_ranges = batch->n;
  p.wait_ns = batch->wait_ns;
  p.ctas_per_sm = batch->ctas_per_sm;
  char* ws = static_cast<char*>(d_ws);
  p.status = reinterpret_cast<int32_t*>(ws + bl.status);
  int64_t units = 0;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(p.status, 0, sizeof(int32_t), s);
  for (int r = 0; r < batch->n && e == cudaSuccess; ++r) {
    const spd_range_io& a = io[r];
    spd::BatchRange& R = p.ranges[r];
    R.x = a.d_x;
    R.snr = a.d_snr;
    R.widx = a.d_width_idx;
    R.mu = a.d_mu;
    R.sigma = a.d_sigma;
    R.ready = a.d_ready;
    R.ndm = batch->ndm[r];
    R.nt = batch->nt[r];
    R.ld = batch->ld[r];
    R.tile = g.bd_general ? g.tile : segment_tile(R.nt, batch->segment);
    R.tiles_per_row = (int32_t)((R.nt + R.tile - 1) / R.tile);
    R.cand_tiles_per_row = (int32_t)((R.nt + spd::kCandTile - 1) / spd::kCandTile);
    R.tile_max = reinterpret_cast<float*>(ws + bl.tile_max[r]);
    R.vec = ((uintptr_t)a.d_snr % 16 == 0 && (uintptr_t)a.d_width_idx % 8 == 0 && R.ld % 4 == 0) ? 1 : 0;
    R.vec_x = ((uintptr_t)a.d_x % 16 == 0 && (R.ld * esize) % 16 == 0) ? 1 : 0;
    R.unit_first = units;
    units += R.ndm * R.tiles_per_row;
    e = cudaMemsetAsync(R.tile_max, 0x80, sizeof(float) * (size_t)(R.ndm * R.cand_tiles_per_row), s);
  }
  p.n_units = units;
  if (e == cudaSuccess)
    e = g.family == kIgrid ? spd::launch_igrid_batch(g, p, s) : spd::launch_boxdit_batch(g, p, s);
  delete sp;
  return check_cuda(e);
}

spd_status spd_batch_status(const spd_batch* batch, const void* d_ws, spd_stream_t stream) {
  if (!batch || !d_ws) return SPD_ERR_INVALID_ARG;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, static_cast<const char*>(d_ws) + BatchLayout(*batch).status,
                                  sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaPeekAtLastError();
  if (e != cudaSuccess) return SPD_ERR_CUDA;
  return h ? SPD_ERR_TIMEOUT : SPD_OK;
}

spd_status spd_batch_candidates(const spd_batch* batch, int32_t range, const float* d_snr,
                                const uint16_t* d_width_idx, float threshold, int32_t peak_radius,
                                spd_candidate* d_out, int64_t cap, int64_t* d_count, void* d_ws,
                                size_t ws_bytes, int32_t use_tile_max, spd_stream_t stream) {
  if (!batch || range < 0 || range >= batch->n) return SPD_ERR_INVALID_ARG;
  const spd_plan rp = range_plan(*batch, range);
  spd_status st = check_cand_args(&rp, d_snr, d_width_idx, threshold, peak_radius, d_out, cap, d_count);
  if (st != SPD_OK) return st;
  const BatchLayout bl(*batch);
  if (ws_bytes < bl.total) return SPD_ERR_WORKSPACE_TOO_SMALL;
  if (!d_ws || ((uintptr_t)d_ws % kAlign) != 0) return SPD_ERR_INVALID_ARG;
  spd::CandParams* cp = new (std::nothrow) spd::CandParams();
  if (!cp) return SPD_ERR_HOST_ALLOC;
  fill_cand_params(*cp, &rp, d_snr, d_width_idx, threshold, peak_radius, d_out, cap, d_count);
  char* ws = static_cast<char*>(d_ws);
  cp->tile_max = use_tile_max ? reinterpret_cast<const float*>(ws + bl.tile_max[range]) : nullptr;
  cp->counts = reinterpret_cast<int32_t*>(ws + bl.counts);
  cp->gsum = reinterpret_cast<int32_t*>(ws + bl.gsum);
  cp->goff = reinterpret_cast<int64_t*>(ws + bl.goff);
  const cudaError_t e = spd::launch_candidates(rp, *cp, reinterpret_cast<cudaStream_t>(stream));
  delete cp;
  return check_cuda(e);
}

int32_t spd_net_param_count(void) { return spd::net_param_count(); }

spd_status spd_net_decimate(const void* d_x, int32_t dtype, int64_t ndm, int64_t nt, int64_t ld,
                            const float* d_mu, const float* d_sigma, float* d_out, spd_stream_t stream) {
  if (!d_x || !d_mu || !d_sigma || !d_out || dtype < SPD_F32 || dtype > SPD_U8) return SPD_ERR_INVALID_ARG;
  if (ndm < 1 || nt < 16 || ld < nt || ndm > ((int64_t)1 << 24) || nt > ((int64_t)1 << 40)) return SPD_ERR_INVALID_ARG;
  const int esize = dtype_size(dtype);
  if (((uintptr_t)d_x % esize) || ((uintptr_t)d_out % 4) || ((uintptr_t)d_mu % 4) || ((uintptr_t)d_sigma % 4))
    return SPD_ERR_INVALID_ARG;
  const bool vec = (uintptr_t)d_x % 16 == 0 && (ld * esize) % 16 == 0;
  return check_cuda(spd::launch_net_decimate(d_x, dtype, esize, ndm, nt, ld, vec, d_mu, d_sigma, d_out,
                                             reinterpret_cast<cudaStream_t>(stream)));
}

spd_status spd_net_forward(const float* d_params, const float* d_blocks, int64_t n_blocks, float* d_logits,
                           spd_stream_t stream) {
  if (!d_params || !d_blocks || !d_logits || n_blocks < 0 || ((uintptr_t)d_params % 4) ||
      ((uintptr_t)d_blocks % 4) || ((uintptr_t)d_logits % 4))
    return SPD_ERR_INVALID_ARG;
  if (n_blocks == 0) return SPD_OK;
  return check_cuda(spd::launch_net_forward(d_params, d_blocks, n_blocks, d_logits,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

spd_status spd_net_gradient(const float* d_params, const float* d_blocks, const float* d_labels,
                            int64_t n_blocks, float* d_grad_sum, float* d_loss_sum, spd_stream_t stream) {
  if (!d_params || !d_blocks || !d_labels || !d_grad_sum || !d_loss_sum || n_blocks < 1) return SPD_ERR_INVALID_ARG;
  if (((uintptr_t)d_params % 4) || ((uintptr_t)d_blocks % 4) || ((uintptr_t)d_labels % 4) ||
      ((uintptr_t)d_grad_sum % 4) || ((uintptr_t)d_loss_sum % 4))
    return SPD_ERR_INVALID_ARG;
  return check_cuda(spd::launch_net_grad(d_params, d_blocks, d_labels, n_blocks, d_grad_sum, d_loss_sum, nullptr,
                                         reinterpret_cast<cudaStream_t>(stream)));
}

size_t spd_net_gradient_workspace_size(void) { return spd::net_grad_workspace_bytes(); }

spd_status spd_net_gradient_ordered(const float* d_params, const float* d_blocks, const float* d_labels,
                                    int64_t n_blocks, float* d_grad_sum, float* d_loss_sum, void* d_ws,
                                    size_t ws_bytes, spd_stream_t stream) {
  if (!d_params || !d_blocks || !d_labels || !d_grad_sum || !d_loss_sum || !d_ws || n_blocks < 1)
    return SPD_ERR_INVALID_ARG;
  if (((uintptr_t)d_params % 4) || ((uintptr_t)d_blocks % 4) || ((uintptr_t)d_labels % 4) ||
      ((uintptr_t)d_grad_sum % 4) || ((uintptr_t)d_loss_sum % 4) || ((uintptr_t)d_ws % 4))
    return SPD_ERR_INVALID_ARG;
  if (ws_bytes < spd::net_grad_workspace_bytes()) return SPD_ERR_WORKSPACE_TOO_SMALL;
  return check_cuda(spd::launch_net_grad(d_params, d_blocks, d_labels, n_blocks, d_grad_sum, d_loss_sum,
                                         static_cast<float*>(d_ws), reinterpret_cast<cudaStream_t>(stream)));
}

spd_status spd_net_adam(float* d_params, float* d_m, float* d_v, const float* d_grad_sum, int64_t n_blocks,
                        float lr, int32_t step, spd_stream_t stream) {
  if (!d_params || !d_m || !d_v || !d_grad_sum || n_blocks < 1 || step < 1 || !(lr >= 0.f) || std::isinf(lr))
    return SPD_ERR_INVALID_ARG;
  return check_cuda(spd::launch_net_adam(d_params, d_m, d_v, d_grad_sum, n_blocks, lr, step,
                                         reinterpret_cast<cudaStream_t>(stream)));
}

spd_status spd_net_select(const float* d_logits, int64_t n, float threshold, int64_t* d_list, int64_t cap,
                          int64_t* d_count, spd_stream_t stream) {
  if (!d_logits || !d_count || n < 0 || cap < 0 || (cap > 0 && !d_list) || std::isnan(threshold) ||
      ((uintptr_t)d_logits % 4) || ((uintptr_t)d_list % 8) || ((uintptr_t)d_count % 8))
    return SPD_ERR_INVALID_ARG;
  return check_cuda(spd::launch_net_select(d_logits, n, threshold, d_list, cap, d_count,
                                           reinterpret_cast<cudaStream_t>(stream)));
}

spd_status spd_net_gather(const void* d_x, int32_t dtype, int64_t ndm, int64_t nt, int64_t ld,
                          const int64_t* d_list, int64_t n, int32_t block, int32_t left, int32_t width,
                          void* d_out, int64_t ld_out, spd_stream_t stream) {
  if (dtype == SPD_U8) return SPD_ERR_UNSUPPORTED;  // no -inf code
  if (!d_x || !d_out || dtype < SPD_F32 || dtype > SPD_BF16 || n < 0 || (n > 0 && !d_list))
    return SPD_ERR_INVALID_ARG;
  if (ndm < 1 || nt < 1 || ld < nt || block < 1 || left < 0 || width < 1 || ld_out < width ||
      n > (int64_t)INT32_MAX || ld_out > ((int64_t)1 << 25))
    return SPD_ERR_INVALID_ARG;
  const int esize = dtype_size(dtype);
  if (((uintptr_t)d_x % esize) || ((uintptr_t)d_list % 8) || ((uintptr_t)d_out % 16) || ((ld_out * esize) % 16))
    return SPD_ERR_INVALID_ARG;
  const bool vec = (uintptr_t)d_x % 16 == 0 && (ld * esize) % 16 == 0;
  return check_cuda(spd::launch_net_gather(d_x, dtype, esize, ndm, nt, ld, d_list, n, block, left, width, d_out,
                                           ld_out, vec, reinterpret_cast<cudaStream_t>(stream)));
}

spd_status spd_sync_status(const spd_plan* plan, spd_stream_t stream) {
  if (!plan) return SPD_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaPeekAtLastError();
  return check_cuda(e);
}

spd_status spd_candidates_status(const int64_t* d_count, int64_t cap, int64_t* total, spd_stream_t stream) {
  if (!d_count || ((uintptr_t)d_count % 8) || cap < 0) return SPD_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaPeekAtLastError();
  int64_t n = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&n, d_count, sizeof(n), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return SPD_ERR_CUDA;
  if (total) *total = n;
  return n > cap ? SPD_ERR_BUFFER_TOO_SMALL : SPD_OK;
}

spd_status spd_proposal_create(const spd_plan_desc* grid, int32_t peak_radius, int64_t max_blocks,
                               spd_proposal** out) {
  if (!out) return SPD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!grid || peak_radius < 0 || peak_radius > spd::kMaxPeakRadius || max_blocks < 1) return SPD_ERR_INVALID_ARG;
  const spd_plan_desc& g = *grid;
  if (g.ndm < 1 || g.nt < kPropBlock || g.nt % kPropBlock || g.ld < g.nt || g.ndm > ((int64_t)1 << 24) ||
      g.nt > ((int64_t)1 << 40))
    return SPD_ERR_INVALID_ARG;
  if (g.dtype < SPD_F32 || g.dtype > SPD_U8) return SPD_ERR_INVALID_ARG;
  if (g.dtype == SPD_U8) return SPD_ERR_UNSUPPORTED;  // the compact rows need -inf past a row's ends
  const int64_t bpr = g.nt / kPropBlock;
  if (max_blocks > g.ndm * bpr) max_blocks = g.ndm * bpr;
  // geometry of the grid: widest width and largest start separation
  spd_plan_desc d = g;
  d.ndm = 1;
  d.nt = 1 << 16;
  d.ld = d.nt;
  spd_plan* probe = nullptr;
  spd_status st = spd_plan_create(&d, &probe);
  if (st != SPD_OK) return st;
  const int lend = probe->lend;
  int sep = 1;
  for (int32_t v : probe->seps) sep = v > sep ? v : sep;
  spd_plan_destroy(probe);
  if (kPropBlock % sep) return SPD_ERR_UNSUPPORTED;  // every level's starts must fall on block starts
  const int left = ((std::max(peak_radius, 1) + sep - 1) / sep) * sep;
  // after the block: its right-hand peak-test neighbours and their widest boxcars
  const int width = left + kPropBlock + peak_radius + lend;
  const int64_t ld_c = ((int64_t)width + 63) / 64 * 64;  // 16-byte aligned rows of any input type
  d = g;
  d.ndm = max_blocks;
  d.nt = width;
  d.ld = ld_c;
  spd_plan* plan = nullptr;
  st = spd_plan_create(&d, &plan);
  if (st != SPD_OK) return st;
  spd_proposal* q = new (std::nothrow) spd_proposal();
  if (!q) {
    spd_plan_destroy(plan);
    return SPD_ERR_HOST_ALLOC;
  }
  q->plan = *plan;
  spd_plan_destroy(plan);
  // the block's starts and the right-hand neighbours of its peak test; the
  // samples after them only feed boxcars
  const int64_t ns = (int64_t)left + kPropBlock + peak_radius;
  q->plan.n_starts = ns;
  q->plan.tiles_per_row = (ns + q->plan.tile - 1) / q->plan.tile;
  q->src = g;
  q->radius = peak_radius;
  q->left = left;
  q->width = width;
  q->ld_c = ld_c;
  q->max_blocks = max_blocks;
  q->bpr = bpr;
  *out = q;
  return SPD_OK;
}

spd_status spd_proposal_destroy(spd_proposal* prop) {
  delete prop;
  return SPD_OK;
}

spd_status spd_proposal_workspace_size(const spd_proposal* prop, size_t* bytes) {
  if (!prop || !bytes) return SPD_ERR_INVALID_ARG;
  *bytes = PropLayout(*prop).total;
  return SPD_OK;
}

spd_status spd_proposal_widths(const spd_proposal* prop, int32_t* widths, int32_t* seps, int32_t cap, int32_t* n) {
  if (!prop) return SPD_ERR_INVALID_ARG;
  return spd_plan_widths(&prop->plan, widths, seps, cap, n);
}

}  // extern "C"

namespace {
spd_status check_proposal_args(const spd_proposal* prop, const void* d_x, const spd_noise* noise, float threshold,
                               spd_candidate* d_out, int64_t cap, int64_t* d_count, void* d_ws, size_t ws_bytes) {
  if (!prop || !d_x || !noise || !d_count || cap < 0 || (cap > 0 && !d_out) || std::isnan(threshold))
    return SPD_ERR_INVALID_ARG;
  if (noise->mode != 0 && noise->mode != 1) return SPD_ERR_INVALID_ARG;
  if (!noise->mu || !noise->sigma || ((uintptr_t)noise->mu % 4) || ((uintptr_t)noise->sigma % 4) ||
      ((uintptr_t)d_count % 8) || ((uintptr_t)d_out % 8) || ((uintptr_t)d_x % dtype_size(prop->src.dtype)))
    return SPD_ERR_INVALID_ARG;
  if (ws_bytes < PropLayout(*prop).total) return SPD_ERR_WORKSPACE_TOO_SMALL;
  if (!d_ws || ((uintptr_t)d_ws % kAlign) != 0) return SPD_ERR_INVALID_ARG;
  return SPD_OK;
}

// Steps 3 of spd_propose_search (also spd_search_blocks): gather the n blocks
// `ids` (device, increasing) and their rows' statistics, search them and select
// their candidates with the block map.  Arguments already checked; n >= 1.
spd_status search_blocks(const spd_proposal* prop, const void* d_x, const spd_noise* noise, const int64_t* ids,
                         int64_t n, float threshold, spd_candidate* d_out, int64_t cap, int64_t* d_count,
                         void* d_ws, cudaStream_t s) {
  const spd_plan_desc& g = prop->src;
  const PropLayout L(*prop);
  char* ws = static_cast<char*>(d_ws);
  const int esize = dtype_size(g.dtype);
  const bool vec = (uintptr_t)d_x % 16 == 0 && (g.ld * esize) % 16 == 0;
  void* xc = ws + L.xc;
  float* yc = reinterpret_cast<float*>(ws + L.yc);
  uint16_t* wc = reinterpret_cast<uint16_t*>(ws + L.wc);
  float* muc = reinterpret_cast<float*>(ws + L.muc);
  float* sgc = reinterpret_cast<float*>(ws + L.sgc);
  cudaError_t e = spd::launch_net_gather(d_x, g.dtype, esize, g.ndm, g.nt, g.ld, ids, n, kPropBlock, prop->left,
                                         prop->width, xc, prop->ld_c, vec, s);
  const int64_t len = noise->mode == 1 ? (int64_t)prop->plan.widths.size() : 1;
  if (e == cudaSuccess) e = spd::launch_gather_rows(noise->mu, len, ids, n, prop->bpr, g.ndm, 0.0f, muc, s);
  if (e == cudaSuccess) e = spd::launch_gather_rows(noise->sigma, len, ids, n, prop->bpr, g.ndm, 1.0f, sgc, s);
  if (e != cudaSuccess) return SPD_ERR_CUDA;
  spd_plan q = prop->plan;  // the compact rows of this call
  q.desc.ndm = n;
  const spd_noise nc{noise->mode, muc, sgc};
  spd_status st = do_execute(&q, xc, &nc, yc, wc, ws + L.ws, L.ws_bytes, s);
  if (st != SPD_OK) return st;
  const BlockMap map{prop->left, prop->left + kPropBlock, ids, prop->bpr, g.nt, kPropBlock};
  return do_candidates(&q, yc, wc, threshold, prop->radius, d_out, cap, d_count, ws + L.ws, L.ws_bytes, true, s,
                       &map);
}
}  // namespace

extern "C" {

spd_status spd_search_blocks(const spd_proposal* prop, const void* d_x, const spd_noise* noise,
                             const int64_t* d_ids, int64_t n_ids, float threshold, spd_candidate* d_out,
                             int64_t cap, int64_t* d_count, void* d_ws, size_t ws_bytes, spd_stream_t stream) {
  spd_status st = check_proposal_args(prop, d_x, noise, threshold, d_out, cap, d_count, d_ws, ws_bytes);
  if (st != SPD_OK) return st;
  if (n_ids < 0 || (n_ids > 0 && (!d_ids || ((uintptr_t)d_ids % 8)))) return SPD_ERR_INVALID_ARG;
  if (n_ids > prop->max_blocks) return SPD_ERR_BUFFER_TOO_SMALL;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n_ids == 0) return check_cuda(cudaMemsetAsync(d_count, 0, sizeof(int64_t), s));
  return search_blocks(prop, d_x, noise, d_ids, n_ids, threshold, d_out, cap, d_count, d_ws, s);
}

spd_status spd_propose_search(const spd_proposal* prop, const float* d_params, const void* d_x,
                              const spd_noise* noise, float logit_threshold, float threshold,
                              spd_candidate* d_out, int64_t cap, int64_t* d_count, int64_t* n_blocks,
                              void* d_ws, size_t ws_bytes, spd_stream_t stream) {
  if (n_blocks) *n_blocks = 0;
  spd_status st = check_proposal_args(prop, d_x, noise, threshold, d_out, cap, d_count, d_ws, ws_bytes);
  if (st != SPD_OK) return st;
  if (!d_params || ((uintptr_t)d_params % 4) || std::isnan(logit_threshold)) return SPD_ERR_INVALID_ARG;
  const spd_plan_desc& g = prop->src;
  const PropLayout L(*prop);
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_ws);
  const int64_t nw = (int64_t)prop->plan.widths.size();
  const int64_t nblk = g.ndm * prop->bpr;
  const int esize = dtype_size(g.dtype);
  const bool vec = (uintptr_t)d_x % 16 == 0 && (g.ld * esize) % 16 == 0;
  float* dec = reinterpret_cast<float*>(ws + L.dec);
  float* logits = reinterpret_cast<float*>(ws + L.logits);
  int64_t* ids = reinterpret_cast<int64_t*>(ws + L.ids);
  int64_t* cnt = reinterpret_cast<int64_t*>(ws + L.cnt);
  // the network reads each row normalised by its width-1 statistics
  const float* mu0 = noise->mu;
  const float* sg0 = noise->sigma;
  cudaError_t e = cudaSuccess;
  if (noise->mode == 1) {
    mu0 = reinterpret_cast<const float*>(ws + L.mu0);
    sg0 = reinterpret_cast<const float*>(ws + L.sg0);
    e = cudaMemcpy2DAsync(ws + L.mu0, sizeof(float), noise->mu, nw * sizeof(float), sizeof(float), g.ndm,
                          cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(ws + L.sg0, sizeof(float), noise->sigma, nw * sizeof(float), sizeof(float), g.ndm,
                            cudaMemcpyDeviceToDevice, s);
  }
  if (e == cudaSuccess) e = spd::launch_net_decimate(d_x, g.dtype, esize, g.ndm, g.nt, g.ld, vec, mu0, sg0, dec, s);
  if (e == cudaSuccess) e = spd::launch_net_forward(d_params, dec, nblk, logits, s);
  if (e == cudaSuccess) e = spd::launch_net_select(logits, nblk, logit_threshold, ids, nblk, cnt, s);
  // the number of flagged blocks sizes the rest: read it back
  int64_t n = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n, cnt, sizeof(n), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return SPD_ERR_CUDA;
  if (n_blocks) *n_blocks = n;
  if (n > prop->max_blocks) return SPD_ERR_BUFFER_TOO_SMALL;
  if (n == 0) return check_cuda(cudaMemsetAsync(d_count, 0, sizeof(int64_t), s));
  return search_blocks(prop, d_x, noise, ids, n, threshold, d_out, cap, d_count, d_ws, s);
}

}  // extern "C"
