// Learned fallback: a small MLP trained online on well-populated cells and
// evaluated for vertices whose cell holds too few samples (Sec. 3.3 motivates
// a fallback for low-density voxels; the network is this library's).
//
// Network: input 80 = per axis sin/cos(pi 2^k p), k = 0..11, of the position
// normalized to a box (72), the normal (3), 5 zeros; three hidden layers of
// 64 with ReLU; linear RGB output.  BF16 weights and activations, FP32
// accumulation, on the tensor cores with mma.sync.m16n8k16 (operands staged in
// shared memory and loaded with ldmatrix).  A warp handles 16 samples: the
// FP32 result fragment of one layer, after bias, ReLU and BF16 packing, is
// directly the A fragment of the next layer, so activations never leave
// registers in inference.  Training: a CTA of 8 warps takes 128 samples;
// forward and delta chains run per warp, the weight gradients X^T dZ are
// CTA-level products over the 128 samples, reduced into an FP32 gradient with
// atomics; Adam updates FP32 master weights and refreshes the BF16 copies.
//
// Parameter vector (FP32, this order): W1 [64][80], b1 [64], W2 [64][64], b2,
// W3 [64][64], b3, W4 [3][64], b4 [3]  (W as [out][in]).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "pps.h"
#include "pps_internal.h"

namespace pps {
namespace mlp {

constexpr int kIn = 80, kHid = 64, kOut = 3;
constexpr int kP = 80 * 64 + 64 + 2 * (64 * 64 + 64) + 3 * 64 + 3;  // 13699
constexpr int oW1 = 0, oB1 = 5120, oW2 = 5184, oB2 = 9280, oW3 = 9344, oB3 = 13440, oW4 = 13504,
              oB4 = 13696;
// BF16 weights in global memory: W1 [64][80], W2 [64][64], W3 [64][64], W4 [16][64]
// (rows 3..15 of W4 zero, so the output layer is one 8-wide and the first
// backward product one 16-deep tile).
constexpr int bW1 = 0, bW2 = 5120, bW3 = 9216, bW4 = 13312, kWb = 14336;
// shared-memory row strides (BF16 elements), padded so ldmatrix rows fall in
// different banks
constexpr int sIn = 88, sHid = 72, sDy = 24;
constexpr int kWarps = 8, kThreads = kWarps * 32, kSamples = kWarps * 16;  // training CTA

struct Dev {
  float* master;  // [kP]
  float* m;       // [kP] Adam first moment
  float* v;       // [kP] Adam second moment
  float* grad;    // [kP] gradient accumulator
  __nv_bfloat16* wb;  // [kWb] BF16 weights
  int32_t* idx;   // [batch] training sample vertex indices
  float lo[3], inv[3];
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x2(uint32_t& r0, uint32_t& r1, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];"
               : "=r"(r0), "=r"(r1)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t& r0, uint32_t& r1, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];"
               : "=r"(r0), "=r"(r1)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + D, FP32 accumulate.
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack2(float x, float y) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);  // x in the low half
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float lo_f(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float hi_f(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// ---------------------------------------------------------------- encoding
// Encoded columns c and c + 1 (c even) of one vertex: a (sin, cos) pair of
// one axis and frequency, two normal components, or padding.
__device__ __forceinline__ float2 enc_pair(int c, const float (&pn)[3], const float (&nr)[3]) {
  if (c < 72) {
    const int a = c / 24, k = (c % 24) / 2;
    float s, co;
    sincospif(pn[a] * static_cast<float>(1 << k), &s, &co);
    return make_float2(s, co);
  }
  if (c == 72) return make_float2(nr[0], nr[1]);
  if (c == 74) return make_float2(nr[2], 0.f);
  return make_float2(0.f, 0.f);
}

struct VertexIn {
  float pn[3], nr[3];
};

__device__ __forceinline__ VertexIn load_vertex(const Dev& d, const VertexPtrs& v, int64_t j) {
  VertexIn o;
  if (j < 0) {
    o = VertexIn{{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    return o;
  }
  const float x[3] = {__ldg(v.px + j), __ldg(v.py + j), __ldg(v.pz + j)};
#pragma unroll
  for (int a = 0; a < 3; ++a)
    o.pn[a] = fminf(fmaxf(__fmul_rn(__fsub_rn(x[a], d.lo[a]), d.inv[a]), 0.f), 1.f);
  o.nr[0] = __ldg(v.nx + j);
  o.nr[1] = __ldg(v.ny + j);
  o.nr[2] = __ldg(v.nz + j);
  return o;
}

// A fragments of the encoded input for this lane's rows g (va) and g + 8 (vb).
__device__ __forceinline__ void encode_frag(uint32_t (&a)[5][4], const VertexIn& va,
                                            const VertexIn& vb, int t) {
#pragma unroll
  for (int kk = 0; kk < 5; ++kk) {
    const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
    const float2 p00 = enc_pair(c0, va.pn, va.nr), p01 = enc_pair(c0, vb.pn, vb.nr);
    const float2 p10 = enc_pair(c1, va.pn, va.nr), p11 = enc_pair(c1, vb.pn, vb.nr);
    a[kk][0] = pack2(p00.x, p00.y);
    a[kk][1] = pack2(p01.x, p01.y);
    a[kk][2] = pack2(p10.x, p10.y);
    a[kk][3] = pack2(p11.x, p11.y);
  }
}

// ---------------------------------------------------------------- layers
// C[nt] (16 x 8 tiles) = A (16 x 16 KT) * W^T + bias, W in shared memory as
// [out][in] rows of `stride` elements (B operand, column-major K x N).
template <int KT, int NT>
__device__ __forceinline__ void layer_fwd(float (&c)[NT][4], const uint32_t (&a)[KT][4],
                                          const __nv_bfloat16* W, int stride, const float* bias,
                                          int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const float b0 = bias ? __ldg(bias + nt * 8 + 2 * t) : 0.f;
    const float b1 = bias ? __ldg(bias + nt * 8 + 2 * t + 1) : 0.f;
    c[nt][0] = b0;
    c[nt][1] = b1;
    c[nt][2] = b0;
    c[nt][3] = b1;
    (void)g;
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      uint32_t w0, w1;
      ldsm_x2(w0, w1, W + (nt * 8 + (lane & 7)) * stride + kt * 16 + ((lane >> 3) & 1) * 8);
      mma(c[nt], a[kt], w0, w1);
    }
  }
}

// ReLU and BF16 packing: the result tiles become the next layer's A fragments.
template <int NT>
__device__ __forceinline__ void relu_pack(uint32_t (&a)[NT / 2][4], const float (&c)[NT][4]) {
#pragma unroll
  for (int k = 0; k < NT / 2; ++k) {
    a[k][0] = pack2(fmaxf(c[2 * k][0], 0.f), fmaxf(c[2 * k][1], 0.f));
    a[k][1] = pack2(fmaxf(c[2 * k][2], 0.f), fmaxf(c[2 * k][3], 0.f));
    a[k][2] = pack2(fmaxf(c[2 * k + 1][0], 0.f), fmaxf(c[2 * k + 1][1], 0.f));
    a[k][3] = pack2(fmaxf(c[2 * k + 1][2], 0.f), fmaxf(c[2 * k + 1][3], 0.f));
  }
}

// Shared-memory copy of the BF16 weights with padded rows.
struct SmemW {
  __nv_bfloat16 w1[64 * sIn];
  __nv_bfloat16 w2[64 * sHid];
  __nv_bfloat16 w3[64 * sHid];
  __nv_bfloat16 w4[16 * sHid];
};

__device__ __forceinline__ void load_weights(SmemW& s, const __nv_bfloat16* wb) {
  for (int i = threadIdx.x; i < 64 * kIn; i += blockDim.x) s.w1[(i / kIn) * sIn + i % kIn] = wb[bW1 + i];
  for (int i = threadIdx.x; i < 64 * kHid; i += blockDim.x) {
    s.w2[(i / kHid) * sHid + i % kHid] = wb[bW2 + i];
    s.w3[(i / kHid) * sHid + i % kHid] = wb[bW3 + i];
  }
  for (int i = threadIdx.x; i < 16 * kHid; i += blockDim.x) s.w4[(i / kHid) * sHid + i % kHid] = wb[bW4 + i];
}

// Forward of 16 vertices held by one warp; returns the output tile (cols 0..7,
// 0..2 meaningful) and optionally keeps the hidden activations as A fragments.
struct Hidden {
  uint32_t h1[4][4], h2[4][4], h3[4][4];
};

__device__ __forceinline__ void forward16(float (&y)[1][4], Hidden& h, const uint32_t (&x0)[5][4],
                                          const SmemW& s, const float* master, int lane) {
  float c[8][4];
  layer_fwd<5, 8>(c, x0, s.w1, sIn, master + oB1, lane);
  relu_pack<8>(h.h1, c);
  layer_fwd<4, 8>(c, h.h1, s.w2, sHid, master + oB2, lane);
  relu_pack<8>(h.h2, c);
  layer_fwd<4, 8>(c, h.h2, s.w3, sHid, master + oB3, lane);
  relu_pack<8>(h.h3, c);
  // output layer: W4 rows 0..7 (3..7 zero); bias only on columns 0..2
  const int t = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i) y[0][i] = 0.f;
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) {
    uint32_t w0, w1;
    ldsm_x2(w0, w1, s.w4 + (lane & 7) * sHid + kt * 16 + ((lane >> 3) & 1) * 8);
    mma(y[0], h.h3[kt], w0, w1);
  }
  const float b0 = 2 * t < kOut ? __ldg(master + oB4 + 2 * t) : 0.f;
  const float b1 = 2 * t + 1 < kOut ? __ldg(master + oB4 + 2 * t + 1) : 0.f;
  y[0][0] += b0;
  y[0][1] += b1;
  y[0][2] += b0;
  y[0][3] += b1;
}

// ---------------------------------------------------------------- inference
// For every vertex whose cell count is below `max_count` (and that did not
// overflow), or every vertex when `all`: evaluate the network and write its RGB
// (and status PPS_STATUS_MLP unless `all`).  Vertices are compacted per warp
// into groups of 16 with ballots.
__global__ void __launch_bounds__(256) k_mlp_infer(Dev d, VertexPtrs v, size_t n, OutPtrs o,
                                                   uint32_t max_count, int all) {
  __shared__ SmemW s;
  __shared__ int32_t queue[8][48];
  load_weights(s, d.wb);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const size_t nwarps = static_cast<size_t>(gridDim.x) * (blockDim.x >> 5);
  const size_t gw = static_cast<size_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
  const size_t per = ((n + nwarps - 1) / nwarps + 31) / 32 * 32;
  const size_t beg = gw * per, end = min(n, beg + per);
  int qn = 0;
  for (size_t base = beg;; base += 32) {
    if (base < end) {
      const size_t j = base + lane;
      bool cand = false;
      if (j < end) {
        if (all) {
          cand = true;
        } else {
          const uint8_t st = o.status[j];
          cand = st != PPS_STATUS_OVERFLOW && o.count[j] < max_count;
        }
      }
      const unsigned mask = __ballot_sync(0xFFFFFFFFu, cand);
      if (cand) queue[warp][qn + __popc(mask & ((1u << lane) - 1u))] = static_cast<int32_t>(j);
      qn += __popc(mask);
      __syncwarp();
    }
    const bool last = base >= end;
    while (qn >= 16 || (last && qn > 0)) {
      const int rows = min(qn, 16);
      const int64_t ja = g < rows ? queue[warp][g] : -1;
      const int64_t jb = g + 8 < rows ? queue[warp][g + 8] : -1;
      uint32_t x0[5][4];
      encode_frag(x0, load_vertex(d, v, ja), load_vertex(d, v, jb), t);
      float y[1][4];
      Hidden h;
      forward16(y, h, x0, s, d.master, lane);
      if (t == 0) {
        if (ja >= 0) {
          o.r[ja] = y[0][0];
          o.g[ja] = y[0][1];
          if (!all) o.status[ja] = PPS_STATUS_MLP;
        }
        if (jb >= 0) {
          o.r[jb] = y[0][2];
          o.g[jb] = y[0][3];
          if (!all) o.status[jb] = PPS_STATUS_MLP;
        }
      } else if (t == 1) {
        if (ja >= 0) o.b[ja] = y[0][0];
        if (jb >= 0) o.b[jb] = y[0][2];
      }
      __syncwarp();
      // drop the 16 evaluated entries from the queue
      const int rest = qn - rows;
      const int32_t moved = lane < rest ? queue[warp][rows + lane] : 0;
      __syncwarp();
      if (lane < rest) queue[warp][lane] = moved;
      __syncwarp();
      qn = rest;
    }
    if (last) break;
  }
}

// ---------------------------------------------------------------- training
// Training samples: for sample i, the first of 16 candidate vertices (Philox,
// key (seed, frame), counter (i, step, try, 0); index = high half of x0 * n)
// whose cell count is >= min_count; -1 if none.
__global__ void k_mlp_select(const uint32_t* count, size_t n, uint32_t seed, uint32_t frame,
                             uint32_t step, uint32_t batch, uint32_t min_count, int32_t* idx) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  int32_t pick = -1;
  for (uint32_t tr = 0; tr < 16 && pick < 0; ++tr) {
    uint32_t x0 = i, x1 = step, x2 = tr, x3 = 0u, k0 = seed, k1 = frame;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      if (r) {
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
      }
      const uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
      const uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
      const uint32_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
      x0 = n0;
      x1 = lo1;
      x2 = n2;
      x3 = lo0;
    }
    const uint32_t cand = static_cast<uint32_t>((static_cast<unsigned long long>(x0) * n) >> 32);
    if (count[cand] >= min_count) pick = static_cast<int32_t>(cand);
  }
  idx[i] = pick;
}

struct SmemTrain {
  SmemW w;
  __nv_bfloat16 x0[kSamples * sIn];
  __nv_bfloat16 h1[kSamples * sHid], h2[kSamples * sHid], h3[kSamples * sHid];
  __nv_bfloat16 z1[kSamples * sHid], z2[kSamples * sHid], z3[kSamples * sHid];
  __nv_bfloat16 dy[kSamples * sDy];
};

__device__ __forceinline__ void put2(__nv_bfloat16* base, int row, int col, int stride, uint32_t w) {
  *reinterpret_cast<uint32_t*>(base + row * stride + col) = w;
}

// Store result-layout tiles (as packed A fragments of 16 x 16 k-tiles) to
// shared memory rows [r0, r0 + 16).
template <int KT>
__device__ __forceinline__ void store_frag(__nv_bfloat16* base, int stride, int r0,
                                           const uint32_t (&a)[KT][4], int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    put2(base, r0 + g, 16 * k + 2 * t, stride, a[k][0]);
    put2(base, r0 + g + 8, 16 * k + 2 * t, stride, a[k][1]);
    put2(base, r0 + g, 16 * k + 8 + 2 * t, stride, a[k][2]);
    put2(base, r0 + g + 8, 16 * k + 8 + 2 * t, stride, a[k][3]);
  }
}

// dH (16 x 64) = dZ (16 x 16 KT) * W, W in shared memory as [out][in] rows
// (B operand K = out, N = in: row-major K x N, loaded transposed).
template <int KT>
__device__ __forceinline__ void layer_bwd(float (&c)[8][4], const uint32_t (&a)[KT][4],
                                          const __nv_bfloat16* W, int stride, int lane) {
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      uint32_t w0, w1;
      ldsm_x2_t(w0, w1, W + (kt * 16 + (lane & 15)) * stride + nt * 8);
      mma(c[nt], a[kt], w0, w1);
    }
  }
}

// Mask a delta tile by (activation > 0), round to BF16 and pack as A fragments.
__device__ __forceinline__ void mask_pack(uint32_t (&dz)[4][4], const float (&c)[8][4],
                                          const uint32_t (&h)[4][4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t* hk = h[k];
    dz[k][0] = pack2(lo_f(hk[0]) > 0.f ? c[2 * k][0] : 0.f, hi_f(hk[0]) > 0.f ? c[2 * k][1] : 0.f);
    dz[k][1] = pack2(lo_f(hk[1]) > 0.f ? c[2 * k][2] : 0.f, hi_f(hk[1]) > 0.f ? c[2 * k][3] : 0.f);
    dz[k][2] = pack2(lo_f(hk[2]) > 0.f ? c[2 * k + 1][0] : 0.f,
                     hi_f(hk[2]) > 0.f ? c[2 * k + 1][1] : 0.f);
    dz[k][3] = pack2(lo_f(hk[3]) > 0.f ? c[2 * k + 1][2] : 0.f,
                     hi_f(hk[3]) > 0.f ? c[2 * k + 1][3] : 0.f);
  }
}

// Weight gradient tile dW[m0..m0+15][n0..n0+7] += dZ^T X over kSamples rows:
// A = dZ^T (m = output, k = sample) and B = X (k = sample, n = input) are both
// read transposed from their row-per-sample shared-memory layout.
__device__ __forceinline__ void dw_tile(float (&acc)[4], const __nv_bfloat16* dz, int sdz,
                                        const __nv_bfloat16* x, int sx, int m0, int n0, int lane) {
  acc[0] = acc[1] = acc[2] = acc[3] = 0.f;
#pragma unroll
  for (int k0 = 0; k0 < kSamples; k0 += 16) {
    uint32_t a[4];
    ldsm_x4_t(a, dz + (k0 + (lane & 7) + ((lane >> 4) << 3)) * sdz + m0 + ((lane >> 3) & 1) * 8);
    uint32_t b0, b1;
    ldsm_x2_t(b0, b1, x + (k0 + (lane & 15)) * sx + n0);
    mma(acc, a, b0, b1);
  }
}

// One batch of samples (kSamples per CTA): forward, backward, and atomic
// accumulation of the gradient of L = 1/(2 batch) sum (y - t)^2.
__global__ void __launch_bounds__(kThreads, 1) k_mlp_grad(Dev d, VertexPtrs v, const float* tr,
                                                          const float* tg, const float* tb,
                                                          const int32_t* idx, uint32_t batch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemTrain& s = *reinterpret_cast<SmemTrain*>(smem_raw);
  load_weights(s.w, d.wb);
  for (int i = threadIdx.x; i < kSamples * sDy / 2; i += blockDim.x)
    reinterpret_cast<uint32_t*>(s.dy)[i] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = warp * 16;
  const uint32_t s0 = blockIdx.x * kSamples + r0;
  const int64_t ja = s0 + g < batch ? idx[s0 + g] : -1;
  const int64_t jb = s0 + g + 8 < batch ? idx[s0 + g + 8] : -1;
  uint32_t x0[5][4];
  encode_frag(x0, load_vertex(d, v, ja), load_vertex(d, v, jb), t);
  store_frag<5>(s.x0, sIn, r0, x0, lane);
  float y[1][4];
  Hidden h;
  forward16(y, h, x0, s.w, d.master, lane);
  store_frag<4>(s.h1, sHid, r0, h.h1, lane);
  store_frag<4>(s.h2, sHid, r0, h.h2, lane);
  store_frag<4>(s.h3, sHid, r0, h.h3, lane);
  // output delta (y - target) / batch for columns 0..2, BF16
  const float invb = 1.0f / static_cast<float>(batch);
  float dy[4] = {0.f, 0.f, 0.f, 0.f};
  if (t < 2) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int64_t j = r ? jb : ja;
      if (j < 0) continue;
      const float t0 = t == 0 ? __ldg(tr + j) : __ldg(tb + j);
      const float t1 = t == 0 ? __ldg(tg + j) : 0.f;
      dy[2 * r] = (y[0][2 * r] - t0) * invb;
      dy[2 * r + 1] = t == 0 ? (y[0][2 * r + 1] - t1) * invb : 0.f;
    }
  }
  uint32_t ady[1][4];
  ady[0][0] = pack2(dy[0], dy[1]);
  ady[0][1] = pack2(dy[2], dy[3]);
  ady[0][2] = 0u;
  ady[0][3] = 0u;
  put2(s.dy, r0 + g, 2 * t, sDy, ady[0][0]);
  put2(s.dy, r0 + g + 8, 2 * t, sDy, ady[0][1]);
  // delta chain: dH3 = dY W4, dZ3 = mask; dH2 = dZ3 W3; ... ; dZ1
  float c[8][4];
  uint32_t dz[4][4];
  layer_bwd<1>(c, ady, s.w.w4, sHid, lane);
  mask_pack(dz, c, h.h3);
  store_frag<4>(s.z3, sHid, r0, dz, lane);
  layer_bwd<4>(c, dz, s.w.w3, sHid, lane);
  mask_pack(dz, c, h.h2);
  store_frag<4>(s.z2, sHid, r0, dz, lane);
  layer_bwd<4>(c, dz, s.w.w2, sHid, lane);
  mask_pack(dz, c, h.h1);
  store_frag<4>(s.z1, sHid, r0, dz, lane);
  __syncthreads();
  // weight gradients over the CTA's samples: 40 + 32 + 32 + 4 tiles of 16 x 8
  for (int tile = warp; tile < 108; tile += kWarps) {
    const __nv_bfloat16 *dzs, *xs;
    int sx, off, in_dim, m0, n0, mmax;
    if (tile < 40) {
      dzs = s.z1; xs = s.x0; sx = sIn; off = oW1; in_dim = kIn; m0 = (tile / 10) * 16; n0 = (tile % 10) * 8; mmax = 64;
    } else if (tile < 72) {
      const int u = tile - 40;
      dzs = s.z2; xs = s.h1; sx = sHid; off = oW2; in_dim = kHid; m0 = (u / 8) * 16; n0 = (u % 8) * 8; mmax = 64;
    } else if (tile < 104) {
      const int u = tile - 72;
      dzs = s.z3; xs = s.h2; sx = sHid; off = oW3; in_dim = kHid; m0 = (u / 8) * 16; n0 = (u % 8) * 8; mmax = 64;
    } else {
      const int u = tile - 104;  // output layer: m = 0..15 (0..2 real), n = 0..63
      dzs = s.dy; xs = s.h3; sx = sHid; off = oW4; in_dim = kHid; m0 = 0; n0 = u * 16; mmax = kOut;
    }
    const int sdz = dzs == s.dy ? sDy : sHid;
    const int reps = tile >= 104 ? 2 : 1;  // output-layer tiles cover 16 inputs
    for (int rep = 0; rep < reps; ++rep) {
      float acc[4];
      dw_tile(acc, dzs, sdz, xs, sx, m0, n0 + rep * 8, lane);
      const int m_a = m0 + g, m_b = m0 + g + 8, n_a = n0 + rep * 8 + 2 * t;
      if (m_a < mmax) {
        atomicAdd(d.grad + off + m_a * in_dim + n_a, acc[0]);
        atomicAdd(d.grad + off + m_a * in_dim + n_a + 1, acc[1]);
      }
      if (m_b < mmax) {
        atomicAdd(d.grad + off + m_b * in_dim + n_a, acc[2]);
        atomicAdd(d.grad + off + m_b * in_dim + n_a + 1, acc[3]);
      }
    }
  }
  // bias gradients: column sums of the deltas
  for (int col = threadIdx.x; col < 3 * kHid + kOut; col += blockDim.x) {
    const __nv_bfloat16* z;
    int stride, cc, off;
    if (col < 64) { z = s.z1; stride = sHid; cc = col; off = oB1; }
    else if (col < 128) { z = s.z2; stride = sHid; cc = col - 64; off = oB2; }
    else if (col < 192) { z = s.z3; stride = sHid; cc = col - 128; off = oB3; }
    else { z = s.dy; stride = sDy; cc = col - 192; off = oB4; }
    float sum = 0.f;
    for (int r = 0; r < kSamples; ++r) sum += __bfloat162float(z[r * stride + cc]);
    atomicAdd(d.grad + off + cc, sum);
  }
}

// Adam on the FP32 master weights; clears the gradient and refreshes the BF16
// copies.  bc1 = 1 - beta1^step, bc2 = 1 - beta2^step.
__global__ void k_mlp_adam(Dev d, float lr, float b1, float b2, float eps, float bc1, float bc2,
                           int apply) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kP) return;
  float w = d.master[i];
  if (apply) {
    const float gr = d.grad[i];
    const float m = b1 * d.m[i] + (1.f - b1) * gr;
    const float vv = b2 * d.v[i] + (1.f - b2) * gr * gr;
    d.m[i] = m;
    d.v[i] = vv;
    w -= lr * (m / bc1) / (sqrtf(vv / bc2) + eps);
    d.master[i] = w;
    d.grad[i] = 0.f;
  }
  // BF16 copy (biases have none)
  int dst = -1;
  if (i < oB1) dst = bW1 + i;
  else if (i >= oW2 && i < oB2) dst = bW2 + (i - oW2);
  else if (i >= oW3 && i < oB3) dst = bW3 + (i - oW3);
  else if (i >= oW4 && i < oB4) dst = bW4 + (i - oW4);
  if (dst >= 0) d.wb[dst] = __float2bfloat16_rn(w);
}

}  // namespace mlp
}  // namespace pps

// ---------------------------------------------------------------- C ABI
struct pps_mlp {
  pps_mlp_params p{};
  int device = 0;
  pps::mlp::Dev dev{};
  size_t idx_cap = 0;
  uint32_t step = 0;  // Adam steps taken
};

namespace {

int mfail(int code, const std::string& msg) { return pps::record_error(code, msg.c_str()); }

#define MLP_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return mfail(PPS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

pps::VertexPtrs vptrs(const pps_vertices* v) {
  pps::VertexPtrs d;
  d.px = v->px;
  d.py = v->py;
  d.pz = v->pz;
  d.nx = v->nx;
  d.ny = v->ny;
  d.nz = v->nz;
  d.r = v->r;
  d.g = v->g;
  d.b = v->b;
  d.id = v->id;
  d.id_base = v->id_base;
  d.stream_id = v->stream_id;
  return d;
}

int check_mlp(pps_mlp* m) {
  if (!m) return mfail(PPS_EINVAL, "mlp is NULL");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != m->device)
    return mfail(PPS_EINVAL, "the network's device is not the current device");
  return PPS_OK;
}

size_t grad_smem() { return sizeof(pps::mlp::SmemTrain); }

int refresh_bf16(pps_mlp* m, cudaStream_t st) {
  pps::mlp::k_mlp_adam<<<(pps::mlp::kP + 255) / 256, 256, 0, st>>>(m->dev, 0.f, 0.f, 0.f, 0.f, 1.f,
                                                                    1.f, 0);
  MLP_CUDA(cudaGetLastError());
  return PPS_OK;
}

}  // namespace

extern "C" {

int pps_mlp_create(pps_mlp** out, const pps_mlp_params* p, const float* init_host) {
  if (!out || !p) return mfail(PPS_EINVAL, "NULL argument");
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (!(p->box_max[a] > p->box_min[a])) return mfail(PPS_EINVAL, "box_max must exceed box_min");
  if (p->batch == 0 || p->batch % pps::mlp::kSamples)
    return mfail(PPS_EINVAL, "batch must be a positive multiple of 128");
  if (!(p->lr > 0.f) || !(p->beta1 >= 0.f && p->beta1 < 1.f) || !(p->beta2 >= 0.f && p->beta2 < 1.f) ||
      !(p->eps > 0.f))
    return mfail(PPS_EINVAL, "bad Adam parameters");
  for (uint32_t r : p->reserved)
    if (r) return mfail(PPS_EINVAL, "reserved fields must be zero");
  pps_mlp* m = new (std::nothrow) pps_mlp();
  if (!m) return mfail(PPS_ENOMEM, "host allocation failed");
  m->p = *p;
  cudaGetDevice(&m->device);
  for (int a = 0; a < 3; ++a) {
    m->dev.lo[a] = p->box_min[a];
    m->dev.inv[a] = 1.0f / (p->box_max[a] - p->box_min[a]);
  }
  const size_t P = pps::mlp::kP;
  cudaError_t e = cudaMalloc(&m->dev.master, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->dev.m, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->dev.v, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->dev.grad, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->dev.wb, pps::mlp::kWb * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->dev.idx, p->batch * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(m->dev.m, 0, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->dev.v, 0, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->dev.grad, 0, P * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->dev.wb, 0, pps::mlp::kWb * sizeof(__nv_bfloat16));
  std::vector<float> w(P, 0.f);
  if (init_host) {
    std::memcpy(w.data(), init_host, P * sizeof(float));
  } else {
    // He initialisation, zero biases
    std::mt19937 rng(p->seed);
    const int fan[4] = {80, 64, 64, 64};
    const int off[4] = {pps::mlp::oW1, pps::mlp::oW2, pps::mlp::oW3, pps::mlp::oW4};
    const int cnt[4] = {64 * 80, 64 * 64, 64 * 64, 3 * 64};
    for (int l = 0; l < 4; ++l) {
      std::normal_distribution<float> nd(0.f, std::sqrt(2.f / fan[l]));
      for (int i = 0; i < cnt[l]; ++i) w[off[l] + i] = nd(rng);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpy(m->dev.master, w.data(), P * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (cudaFuncSetAttribute(pps::mlp::k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(grad_smem())) != cudaSuccess)
      e = cudaGetLastError();
  }
  if (e == cudaSuccess && refresh_bf16(m, nullptr) != PPS_OK) e = cudaErrorUnknown;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(m->dev.master);
    cudaFree(m->dev.m);
    cudaFree(m->dev.v);
    cudaFree(m->dev.grad);
    cudaFree(m->dev.wb);
    cudaFree(m->dev.idx);
    delete m;
    cudaGetLastError();
    return mfail(e == cudaErrorMemoryAllocation ? PPS_ENOMEM : PPS_ECUDA,
                 std::string("pps_mlp_create: ") + cudaGetErrorString(e));
  }
  m->idx_cap = p->batch;
  *out = m;
  return PPS_OK;
}

int pps_mlp_destroy(pps_mlp* m) {
  if (!m) return PPS_OK;
  cudaDeviceSynchronize();
  cudaFree(m->dev.master);
  cudaFree(m->dev.m);
  cudaFree(m->dev.v);
  cudaFree(m->dev.grad);
  cudaFree(m->dev.wb);
  cudaFree(m->dev.idx);
  delete m;
  return PPS_OK;
}

int pps_mlp_set_weights(pps_mlp* m, const float* host, size_t count) {
  if (int rc = check_mlp(m)) return rc;
  if (!host || count != static_cast<size_t>(pps::mlp::kP))
    return mfail(PPS_EINVAL, "weights: need exactly 13699 floats");
  const size_t P = pps::mlp::kP;
  MLP_CUDA(cudaMemcpy(m->dev.master, host, P * sizeof(float), cudaMemcpyHostToDevice));
  MLP_CUDA(cudaMemset(m->dev.m, 0, P * sizeof(float)));
  MLP_CUDA(cudaMemset(m->dev.v, 0, P * sizeof(float)));
  MLP_CUDA(cudaMemset(m->dev.grad, 0, P * sizeof(float)));
  m->step = 0;
  if (int rc = refresh_bf16(m, nullptr)) return rc;
  MLP_CUDA(cudaDeviceSynchronize());
  return PPS_OK;
}

int pps_mlp_get_weights(pps_mlp* m, float* host, size_t count) {
  if (int rc = check_mlp(m)) return rc;
  if (!host || count != static_cast<size_t>(pps::mlp::kP))
    return mfail(PPS_EINVAL, "weights: need exactly 13699 floats");
  MLP_CUDA(cudaDeviceSynchronize());
  MLP_CUDA(cudaMemcpy(host, m->dev.master, count * sizeof(float), cudaMemcpyDeviceToHost));
  return PPS_OK;
}

int pps_mlp_gradient(pps_mlp* m, const pps_vertices* v, const float* tr, const float* tg,
                     const float* tb, const int32_t* idx, uint32_t batch, float* grad_out,
                     void* stream) {
  if (int rc = check_mlp(m)) return rc;
  if (!v || !tr || !tg || !tb || !idx || !grad_out) return mfail(PPS_EINVAL, "NULL argument");
  if (batch == 0 || batch % pps::mlp::kSamples)
    return mfail(PPS_EINVAL, "batch must be a positive multiple of 128");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  MLP_CUDA(cudaMemsetAsync(grad_out, 0, pps::mlp::kP * sizeof(float), st));
  pps::mlp::Dev d = m->dev;
  d.grad = grad_out;
  pps::mlp::k_mlp_grad<<<batch / pps::mlp::kSamples, pps::mlp::kThreads, grad_smem(), st>>>(
      d, vptrs(v), tr, tg, tb, idx, batch);
  MLP_CUDA(cudaGetLastError());
  return PPS_OK;
}

int pps_mlp_train(pps_mlp* m, const pps_vertices* v, size_t n, const pps_output* filtered,
                  uint32_t frame, void* stream) {
  if (int rc = check_mlp(m)) return rc;
  if (!v || !filtered || !filtered->r || !filtered->g || !filtered->b || !filtered->count)
    return mfail(PPS_EINVAL, "vertices and filtered r, g, b, count are required");
  if (n == 0 || m->p.steps == 0) return PPS_OK;
  if (n >= (1ull << 31)) return mfail(PPS_EINVAL, "n too large");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t B = m->p.batch;
  for (uint32_t s = 0; s < m->p.steps; ++s) {
    pps::mlp::k_mlp_select<<<(B + 255) / 256, 256, 0, st>>>(filtered->count, n, m->p.seed, frame, s,
                                                             B, m->p.train_min_count, m->dev.idx);
    MLP_CUDA(cudaGetLastError());
    pps::mlp::k_mlp_grad<<<B / pps::mlp::kSamples, pps::mlp::kThreads, grad_smem(), st>>>(
        m->dev, vptrs(v), filtered->r, filtered->g, filtered->b, m->dev.idx, B);
    MLP_CUDA(cudaGetLastError());
    ++m->step;
    const float bc1 = 1.f - std::pow(m->p.beta1, static_cast<float>(m->step));
    const float bc2 = 1.f - std::pow(m->p.beta2, static_cast<float>(m->step));
    pps::mlp::k_mlp_adam<<<(pps::mlp::kP + 255) / 256, 256, 0, st>>>(
        m->dev, m->p.lr, m->p.beta1, m->p.beta2, m->p.eps, bc1, bc2, 1);
    MLP_CUDA(cudaGetLastError());
  }
  return PPS_OK;
}

static int launch_infer(pps_mlp* m, const pps_vertices* v, size_t n, const pps::OutPtrs& o, int all,
                        cudaStream_t st) {
  if (n == 0) return PPS_OK;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t warps_needed = (n + 511) / 512;
  const int grid = static_cast<int>(std::min<size_t>(static_cast<size_t>(sms) * 4,
                                                     std::max<size_t>(1, (warps_needed + 7) / 8)));
  pps::mlp::k_mlp_infer<<<grid, 256, 0, st>>>(m->dev, vptrs(v), n, o, m->p.infer_max_count, all);
  MLP_CUDA(cudaGetLastError());
  return PPS_OK;
}

int pps_mlp_infer(pps_mlp* m, const pps_vertices* v, size_t n, const pps_output* out, void* stream) {
  if (int rc = check_mlp(m)) return rc;
  if (!v || !out || !out->r || !out->g || !out->b || !out->count || !out->status)
    return mfail(PPS_EINVAL, "vertices and output r, g, b, count, status are required");
  pps::OutPtrs o{out->r, out->g, out->b, out->count, out->status};
  return launch_infer(m, v, n, o, 0, static_cast<cudaStream_t>(stream));
}

int pps_mlp_forward(pps_mlp* m, const pps_vertices* v, size_t n, float* r, float* g, float* b,
                    void* stream) {
  if (int rc = check_mlp(m)) return rc;
  if (!v || !r || !g || !b) return mfail(PPS_EINVAL, "NULL argument");
  pps::OutPtrs o{r, g, b, nullptr, nullptr};
  return launch_infer(m, v, n, o, 1, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
