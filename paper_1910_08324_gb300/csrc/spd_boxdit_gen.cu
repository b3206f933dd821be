// spd_boxdit_gen.cu -- BoxDIT with any even L^i_max, per iteration (Sec. 3.1,
// Alg. 1): the general kernel behind plans whose maximum widths are not one
// of 8, 16, 32 for every iteration (spd_boxdit.cu streams those).
//
// Iteration i (level i) has unit 2^i, starts s = n 2^i and the widths
// c_i + m 2^i, m = 1..k_i, with c_i = sum_{j<i} k_j 2^j (= L^{i-1}_MAX).  The
// kernel runs Alg. 1 as the paper states it, on one tile of T starts of one
// row (T = 2048 or 4096, chosen per plan so that two CTAs fit on an SM):
//   * the shifted decimated series x^i of the tile live in shared memory:
//     x^0 over the tile and its level-0 lookahead, x^1 summed in pairs straight
//     from the input (x^1[u] = x^0[2u + k_0] + x^0[2u + k_0 + 1], the
//     decimation of Sec. 3.1 with its shift of L^0_max / D), and each x^{i+1}
//     from x^i in shared memory (x^{i+1}[u] = x^i[2u + k_i] + x^i[2u + k_i + 1]),
//     every series as long as the levels above still need it;
//   * level i evaluates its T / 2^i positions (one per thread at a time,
//     consecutive positions on consecutive lanes): the sum starts from the
//     base X^{i-1} at the position (kept by level i - 1) and adds
//     x^i[n], x^i[n + 1], ... in order, each partial sum times the width's
//     scale being a candidate (strict '>', so the smaller width wins a tie);
//     the full sum of k_i blocks at an even position is the next level's base;
//   * each level merges its maxima into the tile's Y and W in shared memory
//     (levels in increasing width order, strict '>'), one barrier per level;
//     the tile is then stored with vector stores, and its maximum goes to the
//     candidate-tile key.
// The series past the tile (the halo, up to the widest boxcar) are re-read by
// the neighbouring tiles' CTAs; the widest boxcar of a plan is at most 32768
// samples.  Samples past the end of the row are -inf, so a boxcar needing them
// never wins (the s + L <= nt rule); starts at or past the plan's n_starts are
// not stored.
#include "spd_common.cuh"

namespace spd {

// Window lengths and shared-memory offsets (floats) of a general BoxDIT plan
// with tiles of T starts (see the kernel's comment).
int bdg_layout(const spd_plan& plan, int T, bool table, int32_t* len, int32_t* off) {
  int lt = 0;
  while ((2 << lt) <= T) ++lt;  // log2 T
  auto P = [&](int i) { return i <= lt ? T >> i : 1; };
  const int top = plan.top;
  for (int i = 0; i < kMaxLevels; ++i) len[i] = 0;
  len[top] = P(top) + plan.n_top - 1;
  for (int i = top - 1; i >= 0; --i) {
    const int k = plan.lvl_k[i];
    const int a = P(i) + k - 1, b = 2 * len[i + 1] + k;
    len[i] = a > b ? a : b;
  }
  // level 0 keeps only its own window: x^1 is summed straight from the input
  len[0] = T + (top == 0 ? plan.n_top : plan.lvl_k[0]) - 1;
  int ma = 0, mb = 0;
  for (int i = 1; i <= top; ++i) {
    if (i & 1)
      ma = ma > len[i] + 1 ? ma : len[i] + 1;
    else
      mb = mb > len[i] + 1 ? mb : len[i] + 1;
  }
  int o = 0;
  off[kBdgX0] = o;
  o += al4(len[0]);
  off[kBdgXA] = o;
  o += al4(ma);
  off[kBdgXB] = o;
  o += al4(mb);
  off[kBdgBA] = o;
  o += al4(T / 2);
  off[kBdgBB] = o;
  o += al4(T / 4);
  off[kBdgY] = o;
  o += T;
  off[kBdgW] = o;
  o += T / 2;
  off[kBdgAB] = o;
  o += table ? al4(2 * ((int)plan.widths.size() + kAbPad)) : 0;
  return o;
}

namespace {

template <bool TABLE>
__device__ __forceinline__ void bdg_unit(const SearchParams& p, const Unit& U, float* smem) {
  const int t = threadIdx.x;
  const int T = U.T;
  const int64_t t0 = U.t0;
  const int dt = p.dtype;
  float2* AB = reinterpret_cast<float2*>(smem + p.gen_off[kBdgAB]);
  float mu, inv;
  row_noise<TABLE>(p, U.mu, U.sigma, U.row, AB, mu, inv);
  float* X0 = smem + p.gen_off[kBdgX0];
  float* XA = smem + p.gen_off[kBdgXA];
  float* XB = smem + p.gen_off[kBdgXB];
  float* BA = smem + p.gen_off[kBdgBA];
  float* BB = smem + p.gen_off[kBdgBB];
  float* Y = smem + p.gen_off[kBdgY];
  uint16_t* W = reinterpret_cast<uint16_t*>(smem + p.gen_off[kBdgW]);
  int lt = 0;
  while ((2 << lt) <= T) ++lt;
  // levels with positions in this tile: a level of unit 2^i > T has one, at t0,
  // when 2^i divides t0 (and then so does every lower unit)
  int tt = p.top;
  while (tt > lt && (t0 & ((1LL << tt) - 1)) != 0) --tt;

  // ---- x^0 over the tile's level-0 window, x^1 in pairs from the input ----
  {
    const int n0 = p.gen_len[0];
    for (int q = t; 4 * q < n0; q += kThreads)
      *reinterpret_cast<float4*>(X0 + 4 * q) = load_z4d(U.xrow, t0 + 4 * q, U.nt, dt, U.vec_x, mu, inv);
    if (tt >= 1) {
      const int k0 = p.lvl_k[0], n1 = p.gen_len[1];
      const bool v1 = U.vec_x && (k0 & 3) == 0;
      for (int q = t; 2 * q < n1; q += kThreads) {
        const float4 v = load_z4d(U.xrow, t0 + k0 + 4 * q, U.nt, dt, v1, mu, inv);
        *reinterpret_cast<float2*>(XA + 2 * q) = make_float2(v.x + v.y, v.z + v.w);
      }
    }
  }
  __syncthreads();

  // ---- levels 0..tt: evaluate, merge, decimate; one barrier per level ----
  for (int i = 0; i <= tt; ++i) {
    const int P = i <= lt ? T >> i : 1;
    const int k = p.lvl_k[i];
    const int nu = (i == p.top) ? p.n_top : k;  // block counts that are candidates
    const int mend = (i < tt) ? k : nu;         // blocks summed (the next level needs all k)
    const int first = p.lvl_first[i];
    const float* Xi = (i == 0) ? X0 : ((i & 1) ? XA : XB);
    const float* Bi = (i & 1) ? BA : BB;
    float* Bn = (i & 1) ? BB : BA;
    for (int n = t; n < P; n += kThreads) {
      float S = i ? Bi[n] : 0.0f;
      float best = ninf();
      int bq = 0;
      const float* xs = Xi + n;
      int m = 0;
#pragma unroll 4
      for (; m < nu; ++m) {
        S += xs[m];
        float v;
        if constexpr (TABLE) {
          const float2 ab = AB[first + m];
          v = fmaf(S, ab.x, ab.y);
        } else {
          v = S * p.wscale[first + m];
        }
        if (v > best) {
          best = v;
          bq = m;
        }
      }
      for (; m < mend; ++m) S += xs[m];
      if (i < tt && (n & 1) == 0) Bn[n >> 1] = S;
      const int s = n << i;
      if (i == 0 || best > Y[s]) {
        Y[s] = best;
        W[s] = (uint16_t)(first + bq);
      }
    }
    if (i >= 1 && i < tt) {  // x^{i+1} from x^i, shifted by k_i (Sec. 3.1's decimation)
      float* Xn = (i & 1) ? XB : XA;
      const int nn = p.gen_len[i + 1];
      for (int u = t; u < nn; u += kThreads) {
        const float2 v = *reinterpret_cast<const float2*>(Xi + 2 * u + k);  // k even: aligned pair
        Xn[u] = v.x + v.y;
      }
    }
    __syncthreads();
  }

  // ---- store the tile; its maximum goes to the candidate-tile key ----
  const int64_t sleft = U.ns - t0;
  const int srel = (int)(sleft < (int64_t)T ? sleft : (int64_t)T);
  float tmax = ninf();
  for (int q = t; 4 * q < srel; q += kThreads) {
    float y[4];
    int w[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      y[r] = Y[4 * q + r];
      w[r] = W[4 * q + r];
      if (4 * q + r < srel) tmax = fmaxf(tmax, y[r]);
    }
    store4(U.yrow, U.wrow, t0 + 4 * q, U.ns, U.vec, y, w);
  }
  tile_max_atomic(U.tm_row, t0, tmax);
}

template <bool TABLE>
__global__ void __launch_bounds__(kThreads, 2) boxdit_gen_kernel(const SearchParams p) {
  extern __shared__ __align__(16) float smem[];
  bdg_unit<TABLE>(p, plan_unit(p, blockIdx.x), smem);
}

// Batched search: persistent CTAs stride over the units of every range.
__global__ void __launch_bounds__(kThreads, 2) boxdit_gen_batch_kernel(const SearchParams p) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int flag;
  for (int64_t u = blockIdx.x; u < p.n_units; u += gridDim.x) {
    Unit U;
    if (!batch_unit(p, u, U, &flag)) continue;
    bdg_unit<false>(p, U, smem);
    __syncthreads();
  }
}

}  // namespace

size_t boxdit_gen_smem_bytes(const spd_plan& plan, bool table) {
  int32_t len[kMaxLevels], off[kBdgOffsets];
  return sizeof(float) * (size_t)bdg_layout(plan, plan.tile, table, len, off);
}

cudaError_t launch_boxdit_gen(const spd_plan& plan, const SearchParams& p, cudaStream_t s) {
  const bool table = p.table != 0;
  const size_t smem = boxdit_gen_smem_bytes(plan, table);
  const int64_t nblk = plan.desc.ndm * plan.tiles_per_row;
  return table ? launch_one(boxdit_gen_kernel<true>, smem, nblk, p, s)
               : launch_one(boxdit_gen_kernel<false>, smem, nblk, p, s);
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
