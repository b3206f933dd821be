// spd_net.cu -- block proposal network (sm_103a): x16 decimation of the series,
// forward pass with BF16 tensor-core convolutions, gradients and Adam.
//
// The network (definition in the oracle's net module, restated here):
//   a1 = bf16(relu(b1 + W1 * bf16(x))),  a2 = bf16(relu(b2 + W2 * a1)),  h3 = b3 + W3 * a2
//   g[c] = max_p relu(h3[c][p]),    z = b4 + W4 . g
// over one block of 256 decimated samples; "*" is a 1D correlation with kernel
// 9 and zero padding 4 over 16 channels (1 input channel for layer 1).  The
// weights of layers 1..3 enter as bf16 values, every sum accumulates in FP32.
//
// All three layers are implicit GEMMs on the tensor cores: per block, M = 256
// positions, N = 16 output channels and, for layers 2 and 3, K = 9 taps x 16
// input channels as mma.sync m16n8k16 bf16 -> f32 (one K-step per tap, the tap
// a row offset of the activation operand); layer 1 (one input channel) is one
// K-step over an im2col of the block's 9 taps (padded to 16), built in shared
// memory.  Fragments are loaded with ldmatrix.  Activations live in shared memory as [position + 4][channel] rows of
// 16 bf16 and weights as [tap][out][in] rows of 16, each row's 16-byte halves
// swizzled by bit 2 of its index (conflict-free fragment loads without padding).
// The contraction per block is small (N = 16 output channels) and each layer's
// input is the previous layer's output in shared memory, so the warp-level MMA
// keeps a block's three layers inside one CTA without TMEM round trips.
//
// Gradients (straight-through for the bf16 roundings; the max pool passes its
// gradient to one position per channel): the layer-3 terms touch only the 16
// pooled positions and stay FP32 loops; the three dense contractions run on the
// tensor cores as the same bf16 mma.sync implicit GEMMs with FP32 accumulate:
//   dW2[co][ci][k] = sum_p dh2[p][co] a1[p + k - 4][ci]     (M = co, N = ci, K = p per tap)
//   da1[p][ci]     = sum_{k, co} W2[8 - k][co][ci] dh2[p + k - 4][co]   (the forward's
//                    convolution with the taps flipped and the channels swapped)
//   dW1[c][k], db1[c] = sum_p dh1[p][c] (bf16(x[p + k - 4]), 1)   (M = c, N = 9 taps and a ones column)
// The activations and weights are bf16 values already; the upstream gradient dh
// is split into two bf16 terms, hi = bf16(dh) and lo = bf16(dh - hi), each
// multiplied on the tensor cores, so a product keeps ~16 significant bits.
// Each CTA accumulates its blocks' gradients in shared memory (every entry
// written by one thread or one warp, in a fixed order) and adds them to the
// global sum once.
#include <cuda_bf16.h>

#include "spd_common.cuh"

namespace spd {
namespace {

constexpr int NC = 16, NK = 9, NP = 256, PAD = 4, NPP = NP + 2 * PAD;
constexpr int kNetThreads = 128;
constexpr int kNetParams = 4817;
constexpr int kNetMaxGradCtas = 1024;  // CTAs of a gradient launch (rows of the ordered workspace)
constexpr int oW1 = 0, ob1 = 144, oW2 = 160, ob2 = 2464, oW3 = 2480, ob3 = 4784, oW4 = 4800, ob4 = 4816;
// Activation rows [position][16 channels] and weight rows [tap][out][16 in] are 32
// bytes of bf16 with the two 16-byte halves of a row swapped when bit 2 of the row
// index is set: every 8-row ldmatrix phase is then conflict-free at any row offset
// (rows r and r + 4 fall in different banks), without padding.
__device__ __forceinline__ int swz(int row, int col) { return col ^ (((row >> 2) & 1) << 3); }

struct NetSmem {
  float b1[NC], b2[NC], b3[NC], w4[NC], b4;
  alignas(16) __nv_bfloat16 w1b[NC][NC];     // [out][tap, 9..15 zero; swizzled by out]
  alignas(16) __nv_bfloat16 w2[NK][NC][NC];  // [tap][out][in, swizzled by out]
  alignas(16) __nv_bfloat16 w3[NK][NC][NC];
  alignas(16) float x[NPP];
  alignas(16) __nv_bfloat16 a1[NPP][NC];  // [padded position][channel, swizzled by position]
  alignas(16) __nv_bfloat16 a2[NPP][NC];
  float wmax[4][NC];
  int warg[4][NC];
  float g[NC];
  int arg[NC];
  float z;
};

struct GradSmem {  // training only
  float G[kNetParams];
  // upstream gradient of a layer's output as two bf16 terms (hi, lo), rows
  // p + PAD (zero padding rows) like the activations: dh2, then dh1
  alignas(16) __nv_bfloat16 dh[2][NPP][NC];
  alignas(16) __nv_bfloat16 w2t[NK][NC][NC];  // [8 - tap][ci][co, swizzled by ci]: W2 for da1
  float dh3[NC];
  float db2[kNetThreads / 32][NC];  // per-warp partial sums of the layer-2 bias gradient
};

__device__ __forceinline__ float bf(__nv_bfloat16 v) { return __bfloat162float(v); }

// Weights into shared memory (bf16 copies for the tensor-core layers).
__device__ void load_weights(const float* __restrict__ P, NetSmem& s) {
  for (int i = threadIdx.x; i < NC * NC; i += blockDim.x) {  // P: W1[co][k]
    const int co = i / NC, k = i % NC;
    s.w1b[co][swz(co, k)] = __float2bfloat16_rn(k < NK ? P[oW1 + co * NK + k] : 0.f);
  }
  for (int i = threadIdx.x; i < NC; i += blockDim.x) {
    s.b1[i] = P[ob1 + i];
    s.b2[i] = P[ob2 + i];
    s.b3[i] = P[ob3 + i];
    s.w4[i] = P[oW4 + i];
  }
  if (threadIdx.x == 0) s.b4 = P[ob4];
  for (int i = threadIdx.x; i < NC * NC * NK; i += blockDim.x) {  // P: W[co][ci][k]
    const int co = i / (NC * NK), ci = (i / NK) % NC, k = i % NK;
    s.w2[k][co][swz(co, ci)] = __float2bfloat16_rn(P[oW2 + i]);
    s.w3[k][co][swz(co, ci)] = __float2bfloat16_rn(P[oW3 + i]);
  }
  // zero padding rows of the activations and the input
  for (int i = threadIdx.x; i < 2 * PAD * NC; i += blockDim.x) {
    const int r = i / NC, c = i % NC, row = r < PAD ? r : NP + r;
    s.a1[row][c] = __float2bfloat16_rn(0.f);
    s.a2[row][c] = __float2bfloat16_rn(0.f);
  }
  for (int i = threadIdx.x; i < 2 * PAD; i += blockDim.x) s.x[i < PAD ? i : NP + i] = 0.f;
}

// Four 8x8 bf16 matrices from shared memory (lanes 8m .. 8m + 7 give the row
// addresses of matrix m; 16-byte aligned rows): thread (g, q) = (lane / 4,
// lane % 4) receives row g, columns 2q and 2q + 1 of each matrix.
__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], const __nv_bfloat16* p) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// As ldsm4, transposed: thread (g, q) receives rows 2q and 2q + 1 of column g.
__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], const __nv_bfloat16* p) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One tensor-core layer: out[p][co] = sum_{k, ci} w[k][co][ci] in[p + k - 4][ci]
// for the warp's 4 tiles of 16 positions and both tiles of 8 channels.
// ZERO: start from 0 (else add to acc).
template <bool ZERO = true>
__device__ __forceinline__ void conv_mma(const __nv_bfloat16 (*in)[NC], const __nv_bfloat16 (*w)[NC][NC],
                                         float (&acc)[4][2][4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lr = lane & 7, lm = lane >> 3;  // row within, and index of, the 8x8 matrix this lane addresses
  if constexpr (ZERO) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  }
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    // B of both channel tiles: matrices (tile 0, in 0-7), (tile 0, in 8-15), (tile 1, ...), (tile 1, ...)
    uint32_t b[4];
    const int brow = 8 * (lm >> 1) + lr;
    ldsm4(b, &w[k][brow][swz(brow, 8 * (lm & 1))]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // A of positions 64 warp + 16 i .. + 15 (stored row p + k: offset -4 + 4): matrices
      // (rows 0-7, in 0-7), (rows 8-15, in 0-7), (rows 0-7, in 8-15), (rows 8-15, in 8-15)
      uint32_t a[4];
      const int arow = 64 * warp + 16 * i + k + lr + 8 * (lm & 1);
      ldsm4(a, &in[arow][swz(arow, 8 * (lm >> 1))]);
      mma_bf16(acc[i][0], a[0], a[1], a[2], a[3], b[0], b[1]);
      mma_bf16(acc[i][1], a[0], a[1], a[2], a[3], b[2], b[3]);
    }
  }
}

// Epilogue of a tensor-core layer: out[p + PAD][co] = bf16(relu(acc + bias[co]))
// for the warp's four 16-position tiles (fragment layout of mma m16n8k16).
__device__ __forceinline__ void store_act(const float (&acc)[4][2][4], const float* bias,
                                          __nv_bfloat16 (*out)[NC]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gq = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int p = 64 * warp + 16 * i + gq, co = 8 * j + 2 * tq;
      __nv_bfloat162 lo, hi;
      lo.x = __float2bfloat16_rn(fmaxf(acc[i][j][0] + bias[co], 0.f));
      lo.y = __float2bfloat16_rn(fmaxf(acc[i][j][1] + bias[co + 1], 0.f));
      hi.x = __float2bfloat16_rn(fmaxf(acc[i][j][2] + bias[co], 0.f));
      hi.y = __float2bfloat16_rn(fmaxf(acc[i][j][3] + bias[co + 1], 0.f));
      *reinterpret_cast<__nv_bfloat162*>(&out[p + PAD][swz(p + PAD, co)]) = lo;
      *reinterpret_cast<__nv_bfloat162*>(&out[p + 8 + PAD][swz(p + 8 + PAD, co)]) = hi;
    }
}

// Forward pass of the block already in s.x; leaves a1, a2, g, arg and z in s.
__device__ void net_block_forward(NetSmem& s) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, gq = lane >> 2, tq = lane & 3;
  // layer 1: im2col of the bf16 input into the rows of a2 (free until layer 2's
  // epilogue; its zero padding rows are not touched): row p + PAD holds
  // bf16(x[p + tap - 4]), taps 0..8, and zeros for taps 9..15
  for (int r = t; r < NP; r += kNetThreads) {
    uint32_t v[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const float x0 = 2 * h < NK ? s.x[r + 2 * h] : 0.f;
      const float x1 = 2 * h + 1 < NK ? s.x[r + 2 * h + 1] : 0.f;
      const __nv_bfloat162 pr = __floats2bfloat162_rn(x0, x1);
      v[h] = *reinterpret_cast<const uint32_t*>(&pr);
    }
    const int row = r + PAD, sw = (row >> 2) & 1;
    uint4* dst = reinterpret_cast<uint4*>(&s.a2[row][0]);
    dst[sw] = make_uint4(v[0], v[1], v[2], v[3]);      // taps 0..7
    dst[sw ^ 1] = make_uint4(v[4], v[5], v[6], v[7]);  // taps 8..15
  }
  __syncthreads();
  float acc[4][2][4];
  {
    const int lr = lane & 7, lm = lane >> 3;
    uint32_t b[4];
    const int brow = 8 * (lm >> 1) + lr;
    ldsm4(b, &s.w1b[brow][swz(brow, 8 * (lm & 1))]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t a[4];
      const int arow = PAD + 64 * warp + 16 * i + lr + 8 * (lm & 1);
      ldsm4(a, &s.a2[arow][swz(arow, 8 * (lm >> 1))]);
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
      mma_bf16(acc[i][0], a[0], a[1], a[2], a[3], b[0], b[1]);
      mma_bf16(acc[i][1], a[0], a[1], a[2], a[3], b[2], b[3]);
    }
  }
  store_act(acc, s.b1, s.a1);
  __syncthreads();
  conv_mma(s.a1, s.w2, acc);
  store_act(acc, s.b2, s.a2);
  __syncthreads();
  conv_mma(s.a2, s.w3, acc);
  // max pool: the thread's maximum (first position on ties) of its two channels per tile
  float mv[2][2];
  int mp[2][2];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      mv[j][e] = -1.f;
      mp[j][e] = 0;
    }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int co = 8 * j + 2 * tq + e;
        const int p = 64 * warp + 16 * i + gq;
        const float v0 = fmaxf(acc[i][j][e] + s.b3[co], 0.f);      // row p
        const float v1 = fmaxf(acc[i][j][2 + e] + s.b3[co], 0.f);  // row p + 8
        if (v0 > mv[j][e]) mv[j][e] = v0, mp[j][e] = p;
        if (v1 > mv[j][e]) mv[j][e] = v1, mp[j][e] = p + 8;
      }
  // across the 8 row groups of the warp (lanes with the same tq)
#pragma unroll
  for (int o = 4; o < 32; o <<= 1)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float ov = __shfl_xor_sync(kFull, mv[j][e], o);
        const int op = __shfl_xor_sync(kFull, mp[j][e], o);
        if (ov > mv[j][e] || (ov == mv[j][e] && op < mp[j][e])) mv[j][e] = ov, mp[j][e] = op;
      }
  if (gq == 0)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        s.wmax[warp][8 * j + 2 * tq + e] = mv[j][e];
        s.warg[warp][8 * j + 2 * tq + e] = mp[j][e];
      }
  __syncthreads();
  if (t < NC) {  // warps cover increasing positions: the first warp wins ties
    float v = s.wmax[0][t];
    int a = s.warg[0][t];
    for (int w = 1; w < 4; ++w)
      if (s.wmax[w][t] > v) v = s.wmax[w][t], a = s.warg[w][t];
    s.g[t] = v;
    s.arg[t] = a;
  }
  __syncthreads();
  if (t < 32) {
    float zz = t < NC ? s.w4[t] * s.g[t] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zz += __shfl_xor_sync(kFull, zz, o);
    if (t == 0) s.z = s.b4 + zz;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kNetThreads, 7) net_forward_kernel(const float* __restrict__ P,
                                                                   const float* __restrict__ X, int64_t nb,
                                                                   float* __restrict__ logits) {
  extern __shared__ __align__(16) unsigned char raw[];
  NetSmem& s = *reinterpret_cast<NetSmem*>(raw);
  load_weights(P, s);
  static_assert(NP == 2 * kNetThreads, "two input samples per thread");
  const int t = threadIdx.x;
  // the next block's input is loaded into registers while the current one is evaluated
  float x0 = 0.f, x1 = 0.f;
  if (blockIdx.x < nb) {
    x0 = X[(int64_t)blockIdx.x * NP + t];
    x1 = X[(int64_t)blockIdx.x * NP + kNetThreads + t];
  }
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    __syncthreads();
    s.x[PAD + t] = x0;
    s.x[PAD + kNetThreads + t] = x1;
    const int64_t bn = b + gridDim.x;
    if (bn < nb) {
      x0 = X[bn * NP + t];
      x1 = X[bn * NP + kNetThreads + t];
    }
    __syncthreads();
    net_block_forward(s);
    if (t == 0) logits[b] = s.z;
  }
}

// Split v into two bf16 terms: hi = bf16(v), lo = bf16(v - hi).
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// C[m][n] += sum over the 256 positions p of A[p][m] B[p + boff][n] for the
// 16 x 16 block (m, n), where A rows are those of dh (split h: rows p + PAD) and
// B rows those of `bmat` (rows p + boff); both operands are read transposed
// (ldmatrix .trans), so that M and N index channels and K positions.  One warp;
// c[nt][e]: the m16n8 fragment of n-tile nt.
__device__ __forceinline__ void gemm_pos(const __nv_bfloat16 (*dh)[NPP][NC], const __nv_bfloat16 (*bmat)[NC],
                                         int boff, float (&c)[2][4]) {
  const int lane = threadIdx.x & 31, lr = lane & 7, lm = lane >> 3;
#pragma unroll 4
  for (int st = 0; st < NP / 16; ++st) {
    uint32_t bb[4];
    const int brow = 16 * st + boff + 8 * (lm & 1) + lr;  // matrices: (p 0-7, n 0-7), (p 8-15, n 0-7), (p 0-7, n 8-15), ...
    ldsm4t(bb, &bmat[brow][swz(brow, 8 * (lm >> 1))]);
    const int arow = 16 * st + PAD + 8 * (lm >> 1) + lr;  // matrices: (p 0-7, m 0-7), (p 0-7, m 8-15), (p 8-15, m 0-7), ...
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t aa[4];
      ldsm4t(aa, &dh[h][arow][swz(arow, 8 * (lm & 1))]);
      mma_bf16(c[0], aa[0], aa[1], aa[2], aa[3], bb[0], bb[1]);
      mma_bf16(c[1], aa[0], aa[1], aa[2], aa[3], bb[2], bb[3]);
    }
  }
}

// Forward + backward of the CTA's blocks; gradients summed into G (global) and
// the summed loss into *loss (or, ordered, into this CTA's row of partials).
__global__ void __launch_bounds__(kNetThreads, 3) net_grad_kernel(const float* __restrict__ P,
                                                                const float* __restrict__ X,
                                                                const float* __restrict__ Y, int64_t nb,
                                                                float* __restrict__ Gout, float* __restrict__ loss,
                                                                float* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char raw[];
  NetSmem& s = *reinterpret_cast<NetSmem*>(raw);
  GradSmem& q = *reinterpret_cast<GradSmem*>(raw + ((sizeof(NetSmem) + 15) / 16) * 16);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, gq = lane >> 2, tq = lane & 3;
  load_weights(P, s);
  for (int i = t; i < kNetParams; i += kNetThreads) q.G[i] = 0.f;
  for (int i = t; i < NK * NC * NC; i += kNetThreads) {  // w2t[8 - k][ci][co] = W2[co][ci][k]
    const int co = i / (NC * NK), ci = (i / NK) % NC, k = i % NK;
    q.w2t[NK - 1 - k][ci][swz(ci, co)] = __float2bfloat16_rn(P[oW2 + i]);
  }
  for (int i = t; i < 2 * 2 * PAD * NC; i += kNetThreads) {  // zero padding rows of dh
    const int h = i / (2 * PAD * NC), r = (i / NC) % (2 * PAD), c = i % NC;
    q.dh[h][r < PAD ? r : NP + r][c] = __float2bfloat16_rn(0.f);
  }
  float lsum = 0.f;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    __syncthreads();
    for (int i = t; i < NP; i += kNetThreads) s.x[PAD + i] = X[b * NP + i];
    __syncthreads();
    net_block_forward(s);
    const float z = s.z, y = Y[b];
    const float dz = 1.f / (1.f + __expf(-z)) - y;
    if (t == 0) {
      lsum += fmaxf(z, 0.f) + log1pf(__expf(-fabsf(z))) - y * z;
      q.G[ob4] += dz;
    }
    if (t < NC) {
      q.G[oW4 + t] += dz * s.g[t];
      q.dh3[t] = s.g[t] > 0.f ? dz * s.w4[t] : 0.f;
    }
    __syncthreads();
    // layer 3: weights and bias from the pooled positions
    for (int i = t; i < NC * NC * NK; i += kNetThreads) {
      const int c = i / (NC * NK), ci = (i / NK) % NC, k = i % NK;
      q.G[oW3 + i] += q.dh3[c] * bf(s.a2[s.arg[c] + k][swz(s.arg[c] + k, ci)]);
    }
    if (t < NC) q.G[ob3 + t] += q.dh3[t];
    // dh2 = (a2 > 0) (W3^T dh3 at the taps of the pooled positions), split into two
    // bf16 terms; this thread's channel is t % 16 (its bias-gradient partial sum)
    {
      float db = 0.f;
      for (int i = t; i < NP * NC; i += kNetThreads) {
        const int p = i >> 4, ci = i & 15;
        float d = 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int k = p - s.arg[c] + PAD;  // a2[p] feeds h3[c][arg] through tap k
          if (k >= 0 && k < NK) d = fmaf(bf(s.w3[k][c][swz(c, ci)]), q.dh3[c], d);
        }
        d = bf(s.a2[p + PAD][swz(p + PAD, ci)]) > 0.f ? d : 0.f;
        db += d;
        __nv_bfloat16 hi, lo;
        split_bf16(d, hi, lo);
        q.dh[0][p + PAD][swz(p + PAD, ci)] = hi;
        q.dh[1][p + PAD][swz(p + PAD, ci)] = lo;
      }
      db += __shfl_xor_sync(kFull, db, 16);  // the two threads of the warp with this channel
      if (lane < NC) q.db2[warp][lane] = db;
    }
    __syncthreads();
    if (t < NC) q.G[ob2 + t] += (q.db2[0][t] + q.db2[1][t]) + (q.db2[2][t] + q.db2[3][t]);
    // layer 2 on the tensor cores: dW2 (taps warp, warp + 4, warp + 8 of this warp)
    // and da1 (this warp's 64 positions)
    {
#pragma unroll 1
      for (int k = warp; k < NK; k += kNetThreads / 32) {
        float c[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        gemm_pos(q.dh, s.a1, k, c);  // a1[p + k - 4] sits in row p + k
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int co = gq + 8 * (e >> 1), ci = 8 * nt + 2 * tq + (e & 1);
            q.G[oW2 + (co * NC + ci) * NK + k] += c[nt][e];
          }
      }
    }
    float acc[4][2][4];
    conv_mma<true>(q.dh[0], q.w2t, acc);
    conv_mma<false>(q.dh[1], q.w2t, acc);
    // the layer-1 im2col (bf16 input taps 0..8, a ones column 9 for the bias) in the
    // rows of a2, which the backward no longer reads
    for (int r = t; r < NP; r += kNetThreads) {
      uint32_t v[8];
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const float x0 = 2 * h < NK ? s.x[r + 2 * h] : (2 * h == NK ? 1.f : 0.f);
        const float x1 = 2 * h + 1 < NK ? s.x[r + 2 * h + 1] : (2 * h + 1 == NK ? 1.f : 0.f);
        const __nv_bfloat162 pr = __floats2bfloat162_rn(x0, x1);
        v[h] = *reinterpret_cast<const uint32_t*>(&pr);
      }
      const int row = r + PAD, sw = (row >> 2) & 1;
      uint4* dst = reinterpret_cast<uint4*>(&s.a2[row][0]);
      dst[sw] = make_uint4(v[0], v[1], v[2], v[3]);
      dst[sw ^ 1] = make_uint4(v[4], v[5], v[6], v[7]);
    }
    __syncthreads();  // every warp is done with dh2: it becomes dh1
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int p = 64 * warp + 16 * i + gq + 8 * (e >> 1), ci = 8 * j + 2 * tq + (e & 1);
          const float d = bf(s.a1[p + PAD][swz(p + PAD, ci)]) > 0.f ? acc[i][j][e] : 0.f;
          __nv_bfloat16 hi, lo;
          split_bf16(d, hi, lo);
          q.dh[0][p + PAD][swz(p + PAD, ci)] = hi;
          q.dh[1][p + PAD][swz(p + PAD, ci)] = lo;
        }
    __syncthreads();
    // layer 1 on the tensor cores (one warp): dW1 (columns 0..8) and db1 (column 9)
    if (warp == 0) {
      float c[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
      gemm_pos(q.dh, s.a2, PAD, c);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int co = gq + 8 * (e >> 1), n = 8 * nt + 2 * tq + (e & 1);
          if (n < NK)
            q.G[oW1 + co * NK + n] += c[nt][e];
          else if (n == NK)
            q.G[ob1 + co] += c[nt][e];
        }
    }
  }
  __syncthreads();
  if (partials) {  // ordered: this CTA's row of partial sums (gradient, then loss)
    float* row = partials + (int64_t)blockIdx.x * (kNetParams + 1);
    for (int i = t; i < kNetParams; i += kNetThreads) row[i] = q.G[i];
    if (t == 0) row[kNetParams] = lsum;
  } else {
    for (int i = t; i < kNetParams; i += kNetThreads) atomicAdd(Gout + i, q.G[i]);
    if (t == 0) atomicAdd(loss, lsum);
  }
}

// Sum of the CTAs' partial rows in CTA order (deterministic): gradient entries,
// then the loss.
__global__ void net_reduce_kernel(const float* __restrict__ partials, int rows, float* __restrict__ Gout,
                                  float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > kNetParams) return;
  float acc = 0.f;
  for (int r = 0; r < rows; ++r) acc += partials[(int64_t)r * (kNetParams + 1) + i];
  if (i < kNetParams)
    Gout[i] = acc;
  else
    *loss = acc;
}

// Adam on the mean gradient G / nb (bias-corrected, step counts from 1).
__global__ void net_adam_kernel(float* __restrict__ P, float* __restrict__ M, float* __restrict__ V,
                                const float* __restrict__ G, float inv_nb, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNetParams) return;
  const float g = G[i] * inv_nb;
  const float m = 0.9f * M[i] + 0.1f * g;
  const float v = 0.999f * V[i] + 0.001f * g * g;
  M[i] = m;
  V[i] = v;
  P[i] -= lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
}

// x16 decimation: out[r][j] = (sum of samples 16 j .. 16 j + 15 - 16 mu_r) / (4 sigma_r).
__global__ void __launch_bounds__(256) net_decimate_kernel(const void* __restrict__ x, int dtype, int esize,
                                                            int64_t ndm, int64_t nt, int64_t ld, int vec,
                                                            const float* __restrict__ mu,
                                                            const float* __restrict__ sigma,
                                                            float* __restrict__ out) {
  const int64_t nd = nt / 16;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ndm * nd) return;
  const int64_t r = i / nd, j = i % nd;
  const unsigned char* row = static_cast<const unsigned char*>(x) + (r * ld + 16 * j) * esize;
  float4 a, b, c, d;
  cvt8<false>(load_raw8(row, 0, 16, dtype, vec != 0), 0, 16, dtype, 0.f, 1.f, a, b);
  cvt8<false>(load_raw8(row, 8, 16, dtype, vec != 0), 8, 16, dtype, 0.f, 1.f, c, d);
  const float s = ((a.x + a.y) + (a.z + a.w)) + ((b.x + b.y) + (b.z + b.w)) + ((c.x + c.y) + (c.z + c.w)) +
                  ((d.x + d.y) + (d.z + d.w));
  out[i] = (s - 16.f * mu[r]) / (4.f * sigma[r]);
}

// Flagged blocks: the ids i < n with logits[i] > thr, written to list in
// increasing order (at most cap of them); *count receives their full number.
// CTA c takes the ids of tile c (tile ids in a row of kSelThreads-wide rounds):
// it first counts the flagged ids of every earlier tile (the logits stay in L2,
// and n / tile CTAs read n^2 / (2 tile) values in all), then writes its own in
// order with warp ballots and a scan over the warps.  No scratch memory, one
// launch, deterministic output.
constexpr int kSelThreads = 1024;
__global__ void __launch_bounds__(kSelThreads) net_select_kernel(const float* __restrict__ logits, int64_t n,
                                                                  float thr, int64_t tile,
                                                                  int64_t* __restrict__ list, int64_t cap,
                                                                  int64_t* __restrict__ count) {
  __shared__ int wsum[kSelThreads / 32];
  __shared__ long long red[kSelThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t first = (int64_t)blockIdx.x * tile;
  // flagged ids before this tile
  long long c = 0;
  for (int64_t i = t; i < first; i += kSelThreads) c += logits[i] > thr ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
  if (lane == 0) red[warp] = c;
  __syncthreads();
  long long base = 0;
#pragma unroll 1
  for (int w = 0; w < kSelThreads / 32; ++w) base += red[w];
  // this tile, kSelThreads ids per round
  const int64_t last = first + tile < n ? first + tile : n;
  for (int64_t r0 = first; r0 < last; r0 += kSelThreads) {
    const int64_t i = r0 + t;
    const bool f = i < last && logits[i] > thr;
    const unsigned m = __ballot_sync(kFull, f);
    __syncthreads();  // wsum of the previous round has been read
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll 1
    for (int w = 0; w < kSelThreads / 32; ++w) {
      const int v = wsum[w];
      before += w < warp ? v : 0;
      total += v;
    }
    if (f) {
      const long long slot = base + before + __popc(m & ((1u << lane) - 1u));
      if (slot < cap) list[slot] = i;
    }
    base += total;
  }
  if (blockIdx.x == gridDim.x - 1 && t == 0) *count = base;
}

// Gather of flagged blocks: out[k][c] = x[r][b * block - left + c] for c < width,
// with (r, b) = (list[k] / bpr, list[k] % bpr), and -inf where that position lies
// outside [0, nt) or c >= width (the row padding up to ld_out).  One thread
// writes 16 bytes; ids outside [0, ndm * bpr) give rows of -inf.
template <int ES>
__global__ void __launch_bounds__(256) net_gather_kernel(const unsigned char* __restrict__ x, int64_t ndm,
                                                          int64_t nt, int64_t ld, int64_t bpr, int block,
                                                          int left, int width, const int64_t* __restrict__ list,
                                                          unsigned char* __restrict__ out, int64_t ld_out, int vec,
                                                          uint32_t neg_inf) {
  constexpr int kPer = 16 / ES;  // samples per thread
  const int64_t k = blockIdx.x;
  const int64_t c0 = ((int64_t)blockIdx.y * blockDim.x + threadIdx.x) * kPer;
  if (c0 >= ld_out) return;
  const int64_t id = list[k];
  const bool ok_id = id >= 0 && id < ndm * bpr;
  const int64_t r = ok_id ? id / bpr : 0;
  const int64_t p0 = (ok_id ? (id % bpr) * (int64_t)block : 0) - left + c0;  // source position of c0
  unsigned char* dst = out + (k * ld_out + c0) * ES;
  const unsigned char* src = x + (r * ld) * ES;
  if (ok_id && vec && c0 + kPer <= width && p0 >= 0 && p0 + kPer <= nt && ((p0 * ES) & 15) == 0) {
    *reinterpret_cast<uint4*>(dst) = __ldg(reinterpret_cast<const uint4*>(src + p0 * ES));
    return;
  }
  uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int e = 0; e < kPer; ++e) {
    const int64_t q = p0 + e;
    const bool in = ok_id && c0 + e < width && q >= 0 && q < nt;
    uint32_t v;
    if (ES == 4)
      v = in ? __ldg(reinterpret_cast<const uint32_t*>(src) + q) : neg_inf;
    else
      v = in ? (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(src) + q) : neg_inf;
    if (ES == 4)
      w[e] = v;
    else
      w[e >> 1] |= (v & 0xffffu) << (16 * (e & 1));
  }
  *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

size_t net_smem(bool grad) {
  size_t s = ((sizeof(NetSmem) + 15) / 16) * 16;
  return grad ? s + sizeof(GradSmem) : s;
}

template <class KernelT>
cudaError_t net_grid(KernelT kern, size_t smem, int64_t nb, int* grid) {
  int per_sm = 0, sms = 0;
  const cudaError_t e = persistent_config(reinterpret_cast<const void*>(kern), smem, &per_sm, &sms, kNetThreads);
  if (e != cudaSuccess) return e;
  int64_t g = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  *grid = (int)(g < nb ? g : nb);
  return cudaSuccess;
}

}  // namespace

int net_param_count() { return kNetParams; }

cudaError_t launch_net_forward(const float* P, const float* X, int64_t nb, float* logits, cudaStream_t s) {
  int grid = 0;
  const size_t smem = net_smem(false);
  cudaError_t e = net_grid(net_forward_kernel, smem, nb, &grid);
  if (e != cudaSuccess || grid == 0) return e;
  net_forward_kernel<<<grid, kNetThreads, smem, s>>>(P, X, nb, logits);
  return cudaGetLastError();
}

size_t net_grad_workspace_bytes() { return sizeof(float) * (size_t)kNetMaxGradCtas * (kNetParams + 1); }

cudaError_t launch_net_grad(const float* P, const float* X, const float* Y, int64_t nb, float* G, float* loss,
                            float* partials, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (!partials) {
    e = cudaMemsetAsync(G, 0, sizeof(float) * kNetParams, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
  }
  int grid = 0;
  const size_t smem = net_smem(true);
  e = net_grid(net_grad_kernel, smem, nb, &grid);
  if (e != cudaSuccess || grid == 0) return e;
  if (grid > kNetMaxGradCtas) grid = kNetMaxGradCtas;
  net_grad_kernel<<<grid, kNetThreads, smem, s>>>(P, X, Y, nb, G, loss, partials);
  if (partials && (e = cudaGetLastError()) == cudaSuccess)
    net_reduce_kernel<<<(kNetParams + 1 + 255) / 256, 256, 0, s>>>(partials, grid, G, loss);
  return cudaGetLastError();
}

cudaError_t launch_net_adam(float* P, float* M, float* V, const float* G, int64_t nb, float lr, int step,
                            cudaStream_t s) {
  const float c1 = 1.f / (1.f - powf(0.9f, (float)step)), c2 = 1.f / (1.f - powf(0.999f, (float)step));
  net_adam_kernel<<<(kNetParams + 255) / 256, 256, 0, s>>>(P, M, V, G, 1.f / (float)nb, lr, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_net_select(const float* logits, int64_t n, float thr, int64_t* list, int64_t cap,
                              int64_t* count, cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(count, 0, sizeof(int64_t), s);
  // tiles of at least 8 rounds, at most 256 CTAs (the prefix counts read n^2 / (2 tile) logits)
  int64_t tile = 8 * kSelThreads;
  while (n > 256 * tile) tile *= 2;
  net_select_kernel<<<(unsigned)((n + tile - 1) / tile), kSelThreads, 0, s>>>(logits, n, thr, tile, list, cap, count);
  return cudaGetLastError();
}

cudaError_t launch_net_gather(const void* x, int dtype, int esize, int64_t ndm, int64_t nt, int64_t ld,
                              const int64_t* list, int64_t n, int block, int left, int width, void* out,
                              int64_t ld_out, bool vec, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t per_row = ld_out * esize / 16;  // threads per output row
  const dim3 grid((unsigned)n, (unsigned)((per_row + 255) / 256));
  const int64_t bpr = (nt + block - 1) / block;
  const auto* xs = static_cast<const unsigned char*>(x);
  auto* o = static_cast<unsigned char*>(out);
  if (esize == 4) {
    net_gather_kernel<4><<<grid, 256, 0, s>>>(xs, ndm, nt, ld, bpr, block, left, width, list, o, ld_out,
                                              vec ? 1 : 0, 0xff800000u);
  } else {
    const uint32_t ninf = dtype == SPD_BF16 ? 0xff80u : 0xfc00u;  // -inf of bf16 / f16
    net_gather_kernel<2><<<grid, 256, 0, s>>>(xs, ndm, nt, ld, bpr, block, left, width, list, o, ld_out,
                                              vec ? 1 : 0, ninf);
  }
  return cudaGetLastError();
}

namespace {
// dst[k][j] = src[ids[k] / bpr][j], j < len: the noise statistics of each
// flagged block's row (len 1 for white noise, the plan's widths for a table);
// `fill` for an id outside [0, ndm * bpr) (its gathered samples are all -inf)
__global__ void __launch_bounds__(256) gather_rows_kernel(const float* __restrict__ src, int64_t len,
                                                          const int64_t* __restrict__ ids, int64_t n, int64_t bpr,
                                                          int64_t ndm, float fill, float* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * len; i += stride) {
    const int64_t k = i / len, j = i - k * len;
    const int64_t id = ids[k];
    dst[i] = (id >= 0 && id < ndm * bpr) ? src[(id / bpr) * len + j] : fill;
  }
}
}  // namespace

cudaError_t launch_gather_rows(const float* src, int64_t len, const int64_t* ids, int64_t n, int64_t bpr,
                               int64_t ndm, float fill, float* dst, cudaStream_t s) {
  const int64_t total = n * len;
  if (total == 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  gather_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, len, ids, n, bpr, ndm, fill, dst);
  return cudaGetLastError();
}

cudaError_t launch_net_decimate(const void* x, int dtype, int esize, int64_t ndm, int64_t nt, int64_t ld,
                                bool vec, const float* mu, const float* sigma, float* out, cudaStream_t s) {
  const int64_t n = ndm * (nt / 16);
  if (n == 0) return cudaSuccess;
  net_decimate_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, dtype, esize, ndm, nt, ld, vec ? 1 : 0, mu,
                                                                   sigma, out);
  return cudaGetLastError();
}

}  // namespace spd
