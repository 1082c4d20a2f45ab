// Learned fallback: a small MLP trained online on well-populated cells and
// evaluated for vertices whose cell holds too few samples (Sec. 3.3 motivates
// a fallback for low-density voxels; the network is this library's).
//
// Network: input 80 = per axis sin/cos(pi 2^k p), k = 0..11, of the position
// normalized to a box (72), the normal (3), 5 zeros; three hidden layers of
// 64 with ReLU; linear RGB output.  BF16 weights and activations, FP32
// accumulation, on the fifth-generation tensor cores: tcgen05.mma from
// shared-memory tiles in the canonical no-swizzle layout into tensor memory,
// tcgen05.ld back to registers for the bias / ReLU / rounding epilogues.
// Inference: a CTA of 128 threads evaluates 128 vertices per tile.
// Training: one cooperative launch per call takes all its Adam steps.  A CTA
// of 384 threads takes 128 samples at a time through the forward pass, the
// delta chain and the weight and bias gradients dZ^T X and dZ^T 1 (products
// over the samples, reading the row-per-sample tiles as MN-major operands):
// eight warps run the products, two of them sharing each 32-lane quarter of
// tensor memory and splitting every epilogue by columns, while four warps
// draw, gather and encode the next samples.  The gradients are added to an
// FP32 accumulator with vector reductions; after a grid barrier every thread
// applies Adam to its share of the FP32 master weights and refreshes their
// BF16 copies, and a second barrier starts the next step.
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
constexpr int kSamples = 128;  // training samples per CTA (the MMA's M)

struct Dev {
  float* master;  // [kP]
  float* m;       // [kP] Adam first moment
  float* v;       // [kP] Adam second moment
  float* grad;    // [kP] gradient accumulator
  __nv_bfloat16* wb;  // [kWb] BF16 weights
  unsigned int* err;  // device error word (a tensor-core wait that gave up)
  float lo[3], inv[3];
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t pack2(float x, float y) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);  // x in the low half
  return *reinterpret_cast<const uint32_t*>(&h);
}
// ReLU and BF16 rounding of two values in one conversion (x in the low half):
// rounding is monotonic and keeps 0, so max(round(v), 0) = round(max(v, 0)).
__device__ __forceinline__ uint32_t pack2_relu(float x, float y) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(y), "f"(x));
  return d;
}
__device__ __forceinline__ float lo_f(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float hi_f(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

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

// ---------------------------------------------------------------- inference
// For every vertex whose cell count is below `max_count` (and that did not
// overflow), or every vertex when `all`, the network's RGB (and status
// PPS_STATUS_MLP unless `all`).  Two kernels: k_mlp_compact lists the
// vertices to evaluate; k_mlp_infer_tc evaluates them 128 at a time on the
// fifth-generation tensor cores.
// One pass: each thread looks at 4 consecutive vertices (one 16-byte load of
// their counts and one 4-byte load of their statuses when `vec`: both arrays
// aligned for it), a CTA-wide scan places its CTA's candidates, and one atomic
// per CTA (1,024 vertices) reserves their places in the list.
constexpr int kCompactPer = 4;
__global__ void __launch_bounds__(256) k_mlp_compact(size_t n, const uint8_t* status,
                                                     const uint32_t* count, uint32_t max_count,
                                                     int all, int vec, int32_t* list,
                                                     uint32_t* counter) {
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t j0 = (static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x) * kCompactPer;
  bool f[kCompactPer];
  uint32_t mine = 0;
  if (vec && j0 + kCompactPer <= n) {
    uint32_t c[4] = {0u, 0u, 0u, 0u}, sw = 0u;
    if (!all) {
      const uint4 c4 = __ldcs(reinterpret_cast<const uint4*>(count + j0));
      sw = __ldcs(reinterpret_cast<const unsigned int*>(status + j0));
      c[0] = c4.x;
      c[1] = c4.y;
      c[2] = c4.z;
      c[3] = c4.w;
    }
#pragma unroll
    for (int q = 0; q < kCompactPer; ++q) {
      const uint32_t stq = (sw >> (8 * q)) & 0xFFu;
      f[q] = all || (stq != PPS_STATUS_OVERFLOW && c[q] < max_count);
      mine += f[q] ? 1u : 0u;
    }
  } else {
#pragma unroll
    for (int q = 0; q < kCompactPer; ++q) {
      const size_t j = j0 + q;
      f[q] = j < n && (all || (status[j] != PPS_STATUS_OVERFLOW && count[j] < max_count));
      mine += f[q] ? 1u : 0u;
    }
  }
  // inclusive scan of `mine` over the warp, then over the warps
  uint32_t incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < 8; ++w) {
      const uint32_t c = s_warp[w];
      s_warp[w] = tot;  // exclusive prefix of the warps
      tot += c;
    }
    s_base = tot ? atomicAdd(counter, tot) : 0u;
  }
  __syncthreads();
  uint32_t pos = s_base + s_warp[warp] + incl - mine;
#pragma unroll
  for (int q = 0; q < kCompactPer; ++q)
    if (f[q]) list[pos++] = static_cast<int32_t>(j0 + q);
}

// One CTA of 128 threads takes tiles of 128 listed vertices (the MMA's M).
// Each thread encodes its vertex into a shared-memory tile in the canonical
// K-major layout without swizzle (core matrices of 8 rows x 16 bytes: byte of
// (r, k) = (r / 8 * K / 8 + k / 8) * 128 + r % 8 * 16 + k % 8 * 2); one thread
// issues tcgen05.mma for each layer (A = activations, B = W as [out][in], both
// K-major, BF16; D = FP32 in tensor memory, 64 columns) and commits it to an
// mbarrier; the four warps read their 32 rows back with tcgen05.ld, add the
// bias, apply ReLU, round to BF16 and store the next layer's A tile.  The
// output layer is N = 16 (rows 3..15 of W4 are zero).
namespace tc {
constexpr int kRows = 128;
constexpr uint32_t kTmemCols = 64;

__device__ __forceinline__ uint32_t cm(int r, int k, int K) {
  return static_cast<uint32_t>(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// The activation tile holds the encoded input (K = 80) and, once layer 1's
// product is complete, each hidden layer's output (K = 64) in turn.
struct Smem {
  alignas(128) unsigned char act[kRows * 80 * 2];
  alignas(128) unsigned char w1[64 * 80 * 2];
  alignas(128) unsigned char w2[64 * 64 * 2];
  alignas(128) unsigned char w3[64 * 64 * 2];
  alignas(128) unsigned char w4[16 * 64 * 2];
  float bias[3 * 64 + 16];
  alignas(8) unsigned long long mbar;
  uint32_t tmem;
};
constexpr size_t kSmemBytes = sizeof(Smem) + 128;  // + alignment of the dynamic base

// Shared-memory matrix descriptor: start address, leading byte offset 128
// (the next core matrix along K), stride byte offset `sbo` (the next 8 rows),
// bits 46..48 = 0b001, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(128u >> 4) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N / 8 in bits 17..22, M / 16 in bits 24..28.
__host__ __device__ constexpr uint32_t idesc(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// shared-memory stores of the threads, made visible to the tensor cores
__device__ __forceinline__ void fence_smem_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Wait for the mbarrier phase `parity`; gives up after `limit_ns` (two
// seconds unless given).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity,
                                          unsigned long long limit_ns = 2000000000ull) {
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tmem_ld_x64(uint32_t taddr, uint32_t (&v)[64]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]), "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]), "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void st16(unsigned char* base, uint32_t off, uint4 v) {
  *reinterpret_cast<uint4*>(base + off) = v;
}

// Encoded row of one vertex, 8 columns (16 bytes) at a time: column block
// kb < 9 holds (sin, cos)(pi 2^k p_a) for axis a = kb / 3 and k = 4 (kb % 3)
// .. + 3 -- one sincospif, then three double-angle steps (error at most 8x
// the FP32 rounding, far below BF16's); block 9 holds n_x, n_y, n_z, 0...
// encode_blocks writes blocks KB0 .. KB1 - 1 and, with NORMAL, block 9.
template <int KB0, int KB1, bool NORMAL>
__device__ __forceinline__ void encode_blocks(unsigned char* x, int r, const VertexIn& vi, bool valid) {
#pragma unroll
  for (int kb = KB0; kb < KB1; ++kb) {
    float sn, cs;
    sincospif(vi.pn[kb / 3] * static_cast<float>(1 << (4 * (kb % 3))), &sn, &cs);
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      w[q] = valid ? pack2(sn, cs) : 0u;
      const float s2 = 2.f * sn * cs;
      cs = (cs - sn) * (cs + sn);
      sn = s2;
    }
    st16(x, cm(r, 8 * kb, 80), make_uint4(w[0], w[1], w[2], w[3]));
  }
  if (NORMAL) {
    const uint4 nv = valid ? make_uint4(pack2(vi.nr[0], vi.nr[1]), pack2(vi.nr[2], 0.f), 0u, 0u)
                           : make_uint4(0u, 0u, 0u, 0u);
    st16(x, cm(r, 72, 80), nv);
  }
}
__device__ __forceinline__ void encode_row(unsigned char* x, int r, const VertexIn& vi, bool valid) {
  encode_blocks<0, 9, true>(x, r, vi, valid);
}

// bias + ReLU + BF16 of 64 accumulator columns of row r, into the A tile h
__device__ __forceinline__ void hidden_row(unsigned char* h, int r, const uint32_t (&acc)[64],
                                           const float* bias) {
#pragma unroll
  for (int kb = 0; kb < 8; ++kb) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 8 * kb + 2 * q;
      w[q] = pack2_relu(__uint_as_float(acc[c]) + bias[c], __uint_as_float(acc[c + 1]) + bias[c + 1]);
    }
    st16(h, cm(r, 8 * kb, 64), make_uint4(w[0], w[1], w[2], w[3]));
  }
}

}  // namespace tc

__global__ void __launch_bounds__(128) k_mlp_infer_tc(Dev d, VertexPtrs v, const int32_t* list,
                                                      const uint32_t* counter, OutPtrs o, int all) {
  extern __shared__ unsigned char smem_raw[];
  tc::Smem& s = *reinterpret_cast<tc::Smem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int tid = threadIdx.x, warp = tid >> 5;
  // weights in the canonical layout, 8 elements (one 16-byte chunk of a core
  // matrix row) per load, biases
  const uint4* wb4 = reinterpret_cast<const uint4*>(d.wb);
#pragma unroll 5
  for (int c = tid; c < 64 * kIn / 8; c += blockDim.x)
    tc::st16(s.w1, tc::cm(c / 10, 8 * (c % 10), kIn), __ldg(wb4 + bW1 / 8 + c));
#pragma unroll 4
  for (int c = tid; c < 64 * kHid / 8; c += blockDim.x) {
    tc::st16(s.w2, tc::cm(c / 8, 8 * (c % 8), kHid), __ldg(wb4 + bW2 / 8 + c));
    tc::st16(s.w3, tc::cm(c / 8, 8 * (c % 8), kHid), __ldg(wb4 + bW3 / 8 + c));
  }
  for (int c = tid; c < 16 * kHid / 8; c += blockDim.x)
    tc::st16(s.w4, tc::cm(c / 8, 8 * (c % 8), kHid), __ldg(wb4 + bW4 / 8 + c));
  for (int i = tid; i < 3 * 64 + 16; i += blockDim.x) {
    float b = 0.f;
    if (i < 64) b = d.master[oB1 + i];
    else if (i < 128) b = d.master[oB2 + i - 64];
    else if (i < 192) b = d.master[oB3 + i - 128];
    else if (i < 192 + kOut) b = d.master[oB4 + i - 192];
    s.bias[i] = b;
  }
  const uint32_t mbar = smem_u32(&s.mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s.tmem)),
                 "r"(tc::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_smem_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s.tmem;
  const uint32_t trow = tmem + (static_cast<uint32_t>(warp * 32) << 16);  // this warp's lanes
  const uint32_t aa = smem_u32(s.act);
  const uint32_t count = *counter;
  const uint32_t ntiles = (count + tc::kRows - 1) / tc::kRows;
  uint32_t parity = 0;
  bool ok = true;
  auto row_of = [&](uint32_t tile) -> int64_t {
    const uint32_t i = tile * tc::kRows + tid;
    return tile < ntiles && i < count ? list[i] : -1;
  };
  int64_t j = row_of(blockIdx.x);
  VertexIn vi = load_vertex(d, v, j);
  int64_t jn = row_of(blockIdx.x + gridDim.x);
  for (uint32_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    tc::encode_row(s.act, tid, vi, j >= 0);
    // while this tile goes through the layers: the next tile's vertex (its list
    // entry was read one tile ago, so the loads do not wait for it) and the
    // list entry of the tile after
    const VertexIn vn = load_vertex(d, v, jn);
    const int64_t jnn = row_of(tile + 2 * gridDim.x);
    tc::fence_smem_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    uint32_t acc[64];
#pragma unroll 1
    for (int layer = 0; layer < 4; ++layer) {
      if (tid == 0) {
        const uint32_t a = aa;
        const uint32_t sboa = layer == 0 ? 1280u : 1024u;
        const uint32_t b = smem_u32(layer == 0 ? s.w1 : layer == 1 ? s.w2 : layer == 2 ? s.w3 : s.w4);
        const int ksteps = layer == 0 ? 5 : 4;
        const uint32_t id = layer == 3 ? tc::idesc(128, 16) : tc::idesc(128, 64);
        for (int k = 0; k < ksteps; ++k)
          tc::mma_bf16(tmem, tc::sdesc(a + 256u * k, sboa), tc::sdesc(b + 256u * k, sboa), id,
                       k > 0 ? 1u : 0u);
        tc::commit(mbar);
      }
      ok = __syncthreads_and(tc::mbar_wait(mbar, parity)) != 0;  // the same outcome in every thread
      parity ^= 1u;
      if (!ok) break;
      tc::fence_after();
      if (layer < 3) {
        tc::tmem_ld_x64(trow, acc);
        tc::tmem_wait_ld();
        tc::hidden_row(s.act, tid, acc, s.bias + 64 * layer);
        tc::fence_smem_async();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
      } else {
        uint32_t y[16];
        tc::tmem_ld_x16(trow, y);
        tc::tmem_wait_ld();
        if (j >= 0) {
          o.r[j] = __uint_as_float(y[0]) + s.bias[192];
          o.g[j] = __uint_as_float(y[1]) + s.bias[193];
          o.b[j] = __uint_as_float(y[2]) + s.bias[194];
          if (!all) o.status[j] = PPS_STATUS_MLP;
        }
        tc::fence_before();
        __syncthreads();  // the next tile's MMA overwrites the accumulator
        tc::fence_after();
      }
    }
    j = jn;
    vi = vn;
    jn = jnn;
  }
  if (!ok && tid == 0) atomicOr(d.err, 1u);
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tc::kTmemCols)
                 : "memory");
}

// ---------------------------------------------------------------- training
// Training samples: for sample i, the first of 16 candidate vertices (Philox,
// key (seed, frame), counter (i, step, try, 0); index = high half of x0 * n)
// whose cell count is >= min_count; -1 if none.  Candidates are drawn four at
// a time, their counts fetched together, and the search stops at the first
// group that holds an eligible one (the same answer as drawing all 16).
struct SampleSel {
  const uint32_t* count;
  size_t n;
  uint32_t seed, frame, step, min_count;
};

__device__ __forceinline__ uint32_t sample_candidate(const SampleSel& q, uint32_t i, uint32_t tr) {
  uint32_t x0 = i, x1 = q.step, x2 = tr, x3 = 0u, k0 = q.seed, k1 = q.frame;
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
  return static_cast<uint32_t>((static_cast<unsigned long long>(x0) * q.n) >> 32);
}

__device__ __forceinline__ int32_t select_sample(const SampleSel& q, uint32_t i) {
#pragma unroll 1
  for (uint32_t t0 = 0; t0 < 16; t0 += 4) {
    uint32_t cand[4], cnt[4];
#pragma unroll
    for (uint32_t e = 0; e < 4; ++e) cand[e] = sample_candidate(q, i, t0 + e);
#pragma unroll
    for (int e = 0; e < 4; ++e) cnt[e] = __ldg(q.count + cand[e]);
    int32_t pick = -1;
#pragma unroll
    for (int e = 3; e >= 0; --e)
      if (cnt[e] >= q.min_count) pick = static_cast<int32_t>(cand[e]);
    if (pick >= 0) return pick;
  }
  return -1;
}

// ---------------------------------------------------------------- training on tcgen05
// One CTA of 128 threads takes 128 samples (the MMA's M).  Every tile is kept
// once, row per sample (or per output for the weights), in the canonical
// no-swizzle layout with the row's elements in 16-byte groups; a product that
// runs over the other dimension reads the same bytes as an MN-major operand
// (instruction-descriptor bits 15 / 16), so nothing is transposed:
//   forward   Z_l = X_l W_l^T     A = X_l  K-major,   B = W_l K-major      (M = samples)
//   backward  dX_l = dZ_l W_l      A = dZ_l K-major,   B = W_l MN-major     (M = samples)
//   gradient  gW_l = dZ_l^T X_l    A = dZ_l MN-major,  B = X_l MN-major     (M = outputs)
//   bias      gb_l = dZ_l^T 1      A = dZ_l MN-major,  B = a tile of ones   (M = outputs)
// (M = 128 for the gradients: rows past the layer's outputs read past the
// delta tile and are ignored; a pad behind the tiles keeps those reads inside
// the CTA's shared memory).  Deltas are rounded to BF16 where the oracle
// rounds them; the products sum over the CTA's samples in FP32, and each
// output's gradient row goes to the global gradient with vector reductions.
namespace tct {
// tensor-memory columns: [0, 64) the layer products; then per layer l its
// weight gradient (in(l) columns) and a 16-column block holding its bias
// gradient in every column
constexpr uint32_t kTmemCols = 512;
__host__ __device__ constexpr uint32_t gcol(int l) { return l == 0 ? 64u : 160u + 96u * (l - 1); }
__host__ __device__ constexpr uint32_t bcol(int l) { return l == 0 ? 144u : gcol(l) + 64u; }
static_assert(bcol(3) + 16 <= kTmemCols, "tensor-memory columns");

// Read-past room behind the tiles: a gradient operand of M = 128 reads up to
// 16 row groups of 8 past its start at either descriptor stride.
constexpr int kPad = 32 * 1024;

struct Smem {
  alignas(128) unsigned char w4[16 * 64 * 2];  // W_l [out][in]
  alignas(128) unsigned char w1[64 * 80 * 2];
  alignas(128) unsigned char w2[64 * 64 * 2];
  alignas(128) unsigned char w3[64 * 64 * 2];
  alignas(128) unsigned char x0[2][128 * 80 * 2];  // X_0 [sample][in] of two work items
  alignas(128) unsigned char h[3][128 * 64 * 2];  // X_1..X_3 (hidden outputs) [sample][feature]
  alignas(128) unsigned char ones[128 * 16 * 2];
  alignas(128) unsigned char dz[128 * 64 * 2];  // dY (16 wide), then dZ_2, dZ_1, dZ_0 [sample][out]
  alignas(128) unsigned char pad[kPad];
  float4 tgt[2][128];  // the two work items' targets (w: the sample is valid)
  float bias[3 * 64 + 16];
  alignas(8) unsigned long long mbar;
  uint32_t tmem;
};
constexpr size_t kSmemBytes = sizeof(Smem) + 128;

// descriptor with explicit leading and stride byte offsets
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// An operand tile of R rows by C columns (C contiguous in 16-byte groups).
// As a K-major operand (K = C): core matrices along K are 128 bytes apart
// (LBO), row groups of 8 are C/8 x 128 bytes apart (SBO); a K step of 16
// advances two core matrices.  As an MN-major operand (MN = C, K = R): groups
// of 8 along MN are 128 bytes apart (SBO), groups of 8 along K are C/8 x 128
// bytes apart (LBO); a K step of 16 advances two such groups.
struct Operand {
  uint32_t addr, lbo, sbo, kstep;
};
__device__ __forceinline__ Operand kmajor(const void* p, uint32_t C) {
  return Operand{smem_u32(p), 128u, C * 16u, 256u};
}
__device__ __forceinline__ Operand mnmajor(const void* p, uint32_t C) {
  return Operand{smem_u32(p), C * 16u, 128u, C * 32u};
}

// Issue `ksteps` MMAs of K = 16 into tensor-memory column `dcol`.
__device__ __forceinline__ void issue(uint32_t tmem, uint32_t dcol, Operand a, Operand b, uint32_t n,
                                      int ksteps, bool a_mn, bool b_mn) {
  const uint32_t id = tc::idesc(128, n) | (a_mn ? 1u << 15 : 0u) | (b_mn ? 1u << 16 : 0u);
  for (int k = 0; k < ksteps; ++k)
    tc::mma_bf16(tmem + dcol, desc(a.addr + a.kstep * k, a.lbo, a.sbo),
                 desc(b.addr + b.kstep * k, b.lbo, b.sbo), id, k > 0 ? 1u : 0u);
}

__device__ __forceinline__ void red_v4(float* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p),
               "f"(__uint_as_float(a)), "f"(__uint_as_float(b)), "f"(__uint_as_float(c)),
               "f"(__uint_as_float(d))
               : "memory");
}

__device__ __forceinline__ void sync_tc() {
  tc::fence_smem_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
}
}  // namespace tct

// ---- the training launch
// One launch takes `steps` Adam steps (or computes one gradient, without
// Adam).  A CTA of 384 threads works through 128-sample tiles (the MMA's M),
// one work item (step, tile) at a time:
//  warps 0..7   the chain of products (forward, output delta, backward with
//               the weight and bias gradients) and their epilogues.  Warps w
//               and w + 4 may read the same 32 tensor-memory lanes (samples,
//               or outputs for the gradients), so they split every 64-column
//               product between them, half the columns each.
//  warps 8..11  draw, gather and encode the NEXT work item's samples (thread
//               t: sample t) into the other of two input buffers, so that the
//               samples' memory latency and the encoding overlap the chain.
// With Adam, the CTAs meet at a grid barrier at the end of each step, every
// thread of the grid updates one parameter (Adam), and a second barrier
// publishes the new weights, which the next step stages.
constexpr int kMaxSteps = 8;        // Adam steps per launch
constexpr int kTrainThreads = 384;  // 8 chain warps + 4 sampling warps

struct AdamStep {
  float lr, b1, b2, eps, bc1, bc2;
};

struct TrainArgs {
  Dev d;
  VertexPtrs v;
  const float* tr;
  const float* tg;
  const float* tb;
  const int32_t* idx;  // the samples when given (then one step, no Adam)
  SampleSel sel;       // sel.step: the index of the launch's first step
  float* grad;         // FP32 gradient accumulator, 16-byte aligned
  Ctrl* ctrl;          // grid barrier of the launch (Adam only)
  unsigned int bar_base;  // arrivals counted in ctrl->bar_count before this launch
  uint32_t batch, steps;
  int adam;
  float lr, beta1, beta2, eps;
  float bc1[kMaxSteps], bc2[kMaxSteps];  // Adam's bias corrections, per step
};

// Index of parameter i's BF16 copy, or -1 (biases have none).
__device__ __forceinline__ int bf16_index(int i) {
  if (i < oB1) return bW1 + i;
  if (i >= oW2 && i < oB2) return bW2 + (i - oW2);
  if (i >= oW3 && i < oB3) return bW3 + (i - oW3);
  if (i >= oW4 && i < oB4) return bW4 + (i - oW4);
  return -1;
}

// One Adam update of parameter i from the accumulated gradient, which it
// then clears; refreshes the BF16 copy.  Reads go through L2: the gradient
// was accumulated by other multiprocessors' reductions.
__device__ __forceinline__ void adam_apply(const Dev& d, float* grad, int i, const AdamStep& s) {
  const float gr = __ldcg(grad + i);
  float w = __ldcg(d.master + i);
  const float m = s.b1 * __ldcg(d.m + i) + (1.f - s.b1) * gr;
  const float vv = s.b2 * __ldcg(d.v + i) + (1.f - s.b2) * gr * gr;
  d.m[i] = m;
  d.v[i] = vv;
  w -= s.lr * (m / s.bc1) / (sqrtf(vv / s.bc2) + s.eps);
  d.master[i] = w;
  grad[i] = 0.f;
  const int dst = bf16_index(i);
  if (dst >= 0) d.wb[dst] = __float2bfloat16_rn(w);
}

namespace tct {
__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
               : "r"(taddr));
}

// bias + ReLU + BF16 of 32 accumulator columns (c0 .. c0 + 31) of row r, into
// the A tile h; `bias` points at column c0's bias
__device__ __forceinline__ void hidden_half(unsigned char* h, int r, int c0, const uint32_t (&acc)[32],
                                            const float* bias) {
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 8 * kb + 2 * q;
      w[q] = pack2_relu(__uint_as_float(acc[c]) + bias[c], __uint_as_float(acc[c + 1]) + bias[c + 1]);
    }
    tc::st16(h, tc::cm(r, c0 + 8 * kb, 64), make_uint4(w[0], w[1], w[2], w[3]));
  }
}

// The step's weights in shared memory: BF16 copies in the canonical layout
// and the biases (FP32 masters).  Read through L2: the previous step's Adam
// wrote them during this launch.  The BF16 copies are one contiguous run of
// 16-byte chunks (W1, W2, W3, W4); a thread loads all of its chunks before it
// stores any, so their latencies overlap.
constexpr int kWbChunks = kWb / 8;  // 1792
__device__ __forceinline__ void stage_chunk(Smem& s, int c, uint4 v) {
  if (c < bW2 / 8) tc::st16(s.w1, tc::cm(c / 10, 8 * (c % 10), kIn), v);
  else if (c < bW3 / 8) tc::st16(s.w2, tc::cm((c - bW2 / 8) / 8, 8 * (c % 8), kHid), v);
  else if (c < bW4 / 8) tc::st16(s.w3, tc::cm((c - bW3 / 8) / 8, 8 * (c % 8), kHid), v);
  else tc::st16(s.w4, tc::cm((c - bW4 / 8) / 8, 8 * (c % 8), kHid), v);
}
template <int NT>
__device__ __forceinline__ void stage_weights(Smem& s, const Dev& d, int tid) {
  constexpr int kPer = (kWbChunks + NT - 1) / NT;
  const uint4* wb4 = reinterpret_cast<const uint4*>(d.wb);
  uint4 v[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int c = tid + q * NT;
    v[q] = c < kWbChunks ? __ldcg(wb4 + c) : make_uint4(0u, 0u, 0u, 0u);
  }
  float b = 0.f;
  const int i = tid;
  if (i < 64) b = __ldcg(d.master + oB1 + i);
  else if (i < 128) b = __ldcg(d.master + oB2 + i - 64);
  else if (i < 192) b = __ldcg(d.master + oB3 + i - 128);
  else if (i < 192 + kOut) b = __ldcg(d.master + oB4 + i - 192);
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int c = tid + q * NT;
    if (c < kWbChunks) stage_chunk(s, c, v[q]);
  }
  if (i < 3 * 64 + 16) s.bias[i] = b;
}
}  // namespace tct

// Named barrier 1 over the 256 threads of the product chain (warps 0..7); the
// sampling warps are not held by it.
__device__ __forceinline__ void chain_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ bool chain_bar_and(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
      " bar.red.and.pred q, 1, 256, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(pred ? 1u : 0u)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void chain_sync_tc() {
  tc::fence_smem_async();
  tc::fence_before();
  chain_bar();
  tc::fence_after();
}

// Grid barrier of the training launch on a counter that only grows: each CTA
// adds one arrival and waits until `target` arrivals (this barrier's place in
// the sequence since the counter was last cleared) have been counted, so
// nobody resets anything on the way out.  Bounded like the filter's grid
// barrier (about two seconds, then kErrBarrierTimeout); false when it gave up.
__device__ __forceinline__ bool grid_sync(Ctrl* c, unsigned int target) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(&c->bar_count, 1u);
    const unsigned long long t0 = globaltimer_ns();
    while (static_cast<int>(ld_acquire_u32(&c->bar_count) - target) < 0) {
      if ((ld_acquire_u32(&c->error) & kErrBarrierTimeout) || globaltimer_ns() - t0 > 2000000000ull) {
        atomicOr(&c->error, kErrBarrierTimeout);
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(kTrainThreads, 1) k_mlp_train_tc(TrainArgs a) {
  extern __shared__ unsigned char smem_raw[];
  tct::Smem& s = *reinterpret_cast<tct::Smem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const Dev& d = a.d;
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool chain = warp < 8;               // warps 0..7: products and epilogues
  const bool lower = tid < 128;              // chain warps 0..3
  const int row = tid & 127;                 // sample (or output) row: lane (warp & 3) * 32 + lane
  const uint32_t hc = 32u * ((warp >> 2) & 1);  // a chain warp's 32 columns of a 64-wide product
  const uint32_t ntile = a.batch / kSamples;
  // tiles of this CTA per step, and the work items (step, tile) in order
  const uint32_t mine = blockIdx.x < ntile ? (ntile - 1u - blockIdx.x) / gridDim.x + 1u : 0u;
  const uint32_t items = mine * a.steps;
  for (int c = tid; c < 128 * 16 / 8; c += blockDim.x)  // BF16 1.0 pairs
    tc::st16(s.ones, 16u * c, make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u));
  const uint32_t mbar = smem_u32(&s.mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s.tmem)),
                 "r"(tct::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // sampling warps: draw, gather and encode work item `it` into buffer it & 1
  // (encoded inputs X_0, targets and validity)
  auto prepare = [&](uint32_t it) {
    const uint32_t st = it / mine, tile = blockIdx.x + (it % mine) * gridDim.x;
    SampleSel q = a.sel;
    q.step = a.sel.step + st;
    const uint32_t si = tile * static_cast<uint32_t>(kSamples) + row;
    const int64_t j = si >= a.batch ? -1 : a.idx ? a.idx[si] : select_sample(q, si);
    const VertexIn vi = load_vertex(d, a.v, j);
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j >= 0) t = make_float4(__ldg(a.tr + j), __ldg(a.tg + j), __ldg(a.tb + j), 1.f);
    tc::encode_row(s.x0[it & 1u], row, vi, j >= 0);
    s.tgt[it & 1u][row] = t;
  };
  if (!chain && items > 0) prepare(0);
  tct::sync_tc();
  const uint32_t tmem = s.tmem;
  const uint32_t tq = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);  // this warp's lanes
  uint32_t parity = 0;
  bool ok = true;
  auto wait = [&]() {
    ok = ok && chain_bar_and(tc::mbar_wait(mbar, parity));
    parity ^= 1u;
    tc::fence_after();
  };
  const float invb = 1.0f / static_cast<float>(a.batch);

  for (uint32_t it = 0; it < items && ok; ++it) {
    const uint32_t st = it / mine;
    const bool step_end = it % mine == mine - 1u;
    if (chain) {
      if (it % mine == 0) {  // the step's weights, written by the previous step's Adam
        tct::stage_weights<256>(s, d, tid);
        chain_sync_tc();
      }
      const unsigned char* x0 = s.x0[it & 1u];
      // layer l's input X_l and weight W_l
      auto X = [&](int l) -> const unsigned char* { return l == 0 ? x0 : s.h[l - 1]; };
      auto W = [&](int l) -> const unsigned char* {
        return l == 0 ? s.w1 : l == 1 ? s.w2 : l == 2 ? s.w3 : s.w4;
      };
      // gradient of layer l: gW_l = dZ_l^T X_l and gb_l = dZ_l^T 1 from the delta in s.dz
      auto grad_issue = [&](int l) {
        const uint32_t co = l == 3 ? 16u : 64u, ci = l == 0 ? kIn : kHid;
        tct::issue(tmem, tct::gcol(l), tct::mnmajor(s.dz, co), tct::mnmajor(X(l), ci), ci, 8, true, true);
        tct::issue(tmem, tct::bcol(l), tct::mnmajor(s.dz, co), tct::mnmajor(s.ones, 16), 16, 8, true, true);
      };
      // this warp's half of row `row` of gW_l, and (lower) gb_l[row] or (upper,
      // layer 0) the row's inputs 64..79, into the global gradient
      auto grad_out = [&](int l) {
        const int out_dim = l == 3 ? kOut : kHid, in_dim = l == 0 ? kIn : kHid;
        if ((warp & 3) * 32 >= out_dim) return;  // warp-uniform: rows past the outputs are not read
        const int off = l == 0 ? oW1 : l == 1 ? oW2 : l == 2 ? oW3 : oW4;
        const int boff = l == 0 ? oB1 : l == 1 ? oB2 : l == 2 ? oB3 : oB4;
        uint32_t g[32], e[16];
        tct::tmem_ld_x32(tq + tct::gcol(l) + hc, g);
        if (lower) tc::tmem_ld_x16(tq + tct::bcol(l), e);
        else if (l == 0) tc::tmem_ld_x16(tq + tct::gcol(0) + 64, e);
        tc::tmem_wait_ld();
        if (row < out_dim) {
          float* rp = a.grad + off + row * in_dim;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            tct::red_v4(rp + hc + 4 * q, g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
          if (lower) {
            atomicAdd(a.grad + boff + row, __uint_as_float(e[0]));
          } else if (l == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              tct::red_v4(rp + 64 + 4 * q, e[4 * q], e[4 * q + 1], e[4 * q + 2], e[4 * q + 3]);
          }
        }
      };
      uint32_t acc[32];
      // ---- forward: X_{l+1} = ReLU(X_l W_l^T + b_l), l = 0..2
      for (int l = 0; l < 3 && ok; ++l) {
        const uint32_t C = l == 0 ? kIn : kHid;
        if (tid == 0) {
          tct::issue(tmem, 0, tct::kmajor(X(l), C), tct::kmajor(W(l), C), 64, C / 16, false, false);
          tc::commit(mbar);
        }
        wait();
        if (!ok) break;
        tct::tmem_ld_x32(tq + hc, acc);
        tc::tmem_wait_ld();
        tct::hidden_half(s.h[l], row, static_cast<int>(hc), acc, s.bias + 64 * l + hc);
        chain_sync_tc();
      }
      if (ok) {
        if (tid == 0) {
          tct::issue(tmem, 0, tct::kmajor(s.h[2], kHid), tct::kmajor(s.w4, kHid), 16, 4, false, false);
          tc::commit(mbar);
        }
        wait();
      }
      if (ok) {
        if (lower) {
          uint32_t y[16];
          tc::tmem_ld_x16(tq, y);
          tc::tmem_wait_ld();
          // output delta (y - target) / batch, rounded to BF16, as a 16-wide tile
          const float4 t = s.tgt[it & 1u][row];
          float dy[3] = {0.f, 0.f, 0.f};
          if (t.w != 0.f) {
            const float t3[3] = {t.x, t.y, t.z};
#pragma unroll
            for (int o = 0; o < 3; ++o)
              dy[o] = __bfloat162float(__float2bfloat16_rn(
                  (__uint_as_float(y[o]) + s.bias[192 + o] - t3[o]) * invb));
          }
          tc::st16(s.dz, tc::cm(row, 0, 16), make_uint4(pack2(dy[0], dy[1]), pack2(dy[2], 0.f), 0u, 0u));
        } else {
          tc::st16(s.dz, tc::cm(row, 8, 16), make_uint4(0u, 0u, 0u, 0u));
        }
        chain_sync_tc();
      }
      // ---- backward: for l = 3, 2, 1 the delta dZ_l in s.dz gives dX_l = dZ_l W_l
      // and the gradients of layer l in one commit; then dZ_{l-1} = dX_l masked
      // by X_l > 0 and rounded replaces it
      for (int l = 3; l >= 1 && ok; --l) {
        if (tid == 0) {
          const uint32_t co = l == 3 ? 16u : 64u;
          tct::issue(tmem, 0, tct::kmajor(s.dz, co), tct::mnmajor(W(l), kHid), 64, co / 16, false, true);
          grad_issue(l);
          tc::commit(mbar);
        }
        wait();
        if (!ok) break;
        tct::tmem_ld_x32(tq + hc, acc);
        const unsigned char* xl = X(l);
        uint4 hq[4];
#pragma unroll
        for (int kb = 0; kb < 4; ++kb)
          hq[kb] = *reinterpret_cast<const uint4*>(xl + tc::cm(row, static_cast<int>(hc) + 8 * kb, 64));
        tc::tmem_wait_ld();
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
          const uint32_t hw[4] = {hq[kb].x, hq[kb].y, hq[kb].z, hq[kb].w};
          uint32_t zw[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = 8 * kb + 2 * q;
            zw[q] = pack2(lo_f(hw[q]) > 0.f ? __uint_as_float(acc[c]) : 0.f,
                          hi_f(hw[q]) > 0.f ? __uint_as_float(acc[c + 1]) : 0.f);
          }
          tc::st16(s.dz, tc::cm(row, static_cast<int>(hc) + 8 * kb, 64), make_uint4(zw[0], zw[1], zw[2], zw[3]));
        }
        grad_out(l);
        chain_sync_tc();
      }
      if (ok) {
        if (tid == 0) {
          grad_issue(0);
          tc::commit(mbar);
        }
        wait();
        if (ok) grad_out(0);
      }
    } else if (it + 1 < items) {
      prepare(it + 1);  // the next work item, while the chain runs this one
    }
    // the chain is done with X_0 of this item and the sampling warps with the
    // next item's buffers (made visible to the tensor cores); the chain's
    // outcome reaches every thread
    tc::fence_smem_async();
    tc::fence_before();
    ok = __syncthreads_and(ok) != 0;
    tc::fence_after();
    if (!ok) break;
    if (a.adam && step_end) {
      // every gradient reduction in; Adam, one parameter per thread of the
      // grid; the new weights visible before the next step stages them
      const unsigned int base = a.bar_base + 2u * st * gridDim.x;
      if (!grid_sync(a.ctrl, base + gridDim.x)) {
        ok = false;
        break;
      }
      const AdamStep as{a.lr, a.beta1, a.beta2, a.eps, a.bc1[st], a.bc2[st]};
      for (int i = blockIdx.x * blockDim.x + tid; i < kP; i += gridDim.x * blockDim.x)
        adam_apply(d, a.grad, i, as);
      if (!grid_sync(a.ctrl, base + 2u * gridDim.x)) {
        ok = false;
        break;
      }
    }
  }
  if (!ok && tid == 0) {
    atomicOr(d.err, 1u);
    if (a.ctrl) atomicOr(&a.ctrl->error, kErrBarrierTimeout);  // the other CTAs stop waiting
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tct::kTmemCols)
                 : "memory");
}

// BF16 copies of the master weights (after they were set from the host).
__global__ void k_mlp_refresh_bf16(Dev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kP) return;
  const int dst = bf16_index(i);
  if (dst >= 0) d.wb[dst] = __float2bfloat16_rn(d.master[i]);
}

// Self-test of the bounded wait: an mbarrier that nothing completes; the wait
// gives up after `limit_ns` and the kernel reports it in *err (bit 0).
__global__ void k_selftest_mbar(unsigned long long limit_ns, unsigned int* err) {
  __shared__ alignas(8) unsigned long long mbar;
  const uint32_t a = smem_u32(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(a, 0u, limit_ns)) atomicOr(err, 1u);
}

}  // namespace mlp

cudaError_t launch_selftest_mbar(unsigned long long limit_ns, unsigned int* err, cudaStream_t st) {
  mlp::k_selftest_mbar<<<1, 32, 0, st>>>(limit_ns, err);
  return cudaGetLastError();
}
}  // namespace pps

// ---------------------------------------------------------------- C ABI
struct pps_mlp {
  pps_mlp_params p{};
  int device = 0;
  pps::mlp::Dev dev{};
  uint32_t step = 0;  // Adam steps taken
  int sms = 0;                  // multiprocessors of the device
  pps::Ctrl* ctrl = nullptr;    // training: grid barriers around Adam
  uint32_t bar_arrivals = 0;    // training: arrivals counted in ctrl->bar_count so far
  int32_t* list = nullptr;      // inference: indices of the vertices to evaluate
  uint32_t* counter = nullptr;  // inference: their number
  size_t list_cap = 0;
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
  d.dist = v->dist;
  d.extra = v->extra;
  return d;
}

int check_mlp(pps_mlp* m) {
  if (!m) return mfail(PPS_EINVAL, "mlp is NULL");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != m->device)
    return mfail(PPS_EINVAL, "the network's device is not the current device");
  return PPS_OK;
}


int refresh_bf16(pps_mlp* m, cudaStream_t st) {
  pps::mlp::k_mlp_refresh_bf16<<<(pps::mlp::kP + 255) / 256, 256, 0, st>>>(m->dev);
  MLP_CUDA(cudaGetLastError());
  return PPS_OK;
}

// One training launch: `steps` (at most kMaxSteps) Adam steps on samples drawn
// with `sel` (cooperative: the steps are separated by grid barriers), or, with
// adam false, the gradient of one step over the given samples `idx`.
int launch_train(pps_mlp* m, const pps_vertices* v, const float* tr, const float* tg,
                 const float* tb, const int32_t* idx, const pps::mlp::SampleSel& sel,
                 uint32_t batch, uint32_t steps, bool adam, float* grad, cudaStream_t st) {
  pps::mlp::TrainArgs a{};
  a.d = m->dev;
  a.v = vptrs(v);
  a.tr = tr;
  a.tg = tg;
  a.tb = tb;
  a.idx = idx;
  a.sel = sel;
  a.grad = grad;
  a.ctrl = adam ? m->ctrl : nullptr;
  a.bar_base = m->bar_arrivals;
  a.batch = batch;
  a.steps = steps;
  a.adam = adam ? 1 : 0;
  a.lr = m->p.lr;
  a.beta1 = m->p.beta1;
  a.beta2 = m->p.beta2;
  a.eps = m->p.eps;
  for (uint32_t k = 0; adam && k < steps; ++k) {
    ++m->step;
    a.bc1[k] = 1.f - std::pow(m->p.beta1, static_cast<float>(m->step));
    a.bc2[k] = 1.f - std::pow(m->p.beta2, static_cast<float>(m->step));
  }
  const int grid = static_cast<int>(std::min<uint32_t>(batch / pps::mlp::kSamples,
                                                       static_cast<uint32_t>(m->sms)));
  if (adam) {
    void* args[] = {&a};
    MLP_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(pps::mlp::k_mlp_train_tc),
                                         dim3(grid), dim3(pps::mlp::kTrainThreads), args,
                                         pps::mlp::tct::kSmemBytes, st));
    // counted only for a launch that was made: two barriers per step, one
    // arrival per CTA each
    m->bar_arrivals += 2u * steps * static_cast<uint32_t>(grid);
  } else {
    pps::mlp::k_mlp_train_tc<<<grid, pps::mlp::kTrainThreads, pps::mlp::tct::kSmemBytes, st>>>(a);
    MLP_CUDA(cudaGetLastError());
  }
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
  cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, m->device);
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
  if (e == cudaSuccess) e = cudaMalloc(&m->dev.err, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&m->counter, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->ctrl, sizeof(pps::Ctrl));
  if (e == cudaSuccess) e = cudaMemset(m->ctrl, 0, sizeof(pps::Ctrl));
  if (e == cudaSuccess) e = cudaMemset(m->dev.err, 0, sizeof(unsigned int));
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
    if (cudaFuncSetAttribute(pps::mlp::k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(pps::mlp::tc::kSmemBytes)) != cudaSuccess ||
        cudaFuncSetAttribute(pps::mlp::k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(pps::mlp::tct::kSmemBytes)) != cudaSuccess)
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
    cudaFree(m->dev.err);
    cudaFree(m->counter);
    cudaFree(m->ctrl);
    delete m;
    cudaGetLastError();
    return mfail(e == cudaErrorMemoryAllocation ? PPS_ENOMEM : PPS_ECUDA,
                 std::string("pps_mlp_create: ") + cudaGetErrorString(e));
  }
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
  cudaFree(m->dev.err);
  cudaFree(m->counter);
  cudaFree(m->ctrl);
  cudaFree(m->list);
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
  unsigned int err = 0;
  MLP_CUDA(cudaMemcpy(&err, m->dev.err, sizeof(err), cudaMemcpyDeviceToHost));
  if (err) {
    // reported once: the error word and the grid barrier start afresh
    MLP_CUDA(cudaMemset(m->dev.err, 0, sizeof(unsigned int)));
    MLP_CUDA(cudaMemset(m->ctrl, 0, sizeof(pps::Ctrl)));
    m->bar_arrivals = 0;
    return mfail(PPS_EDEVICE, "a training or inference launch gave up waiting (tensor cores or grid barrier)");
  }
  return PPS_OK;
}

int pps_mlp_gradient(pps_mlp* m, const pps_vertices* v, const float* tr, const float* tg,
                     const float* tb, const int32_t* idx, uint32_t batch, float* grad_out,
                     void* stream) {
  if (int rc = check_mlp(m)) return rc;
  if (!v || !tr || !tg || !tb || !idx || !grad_out) return mfail(PPS_EINVAL, "NULL argument");
  if (reinterpret_cast<uintptr_t>(grad_out) % 16) return mfail(PPS_EINVAL, "grad_out must be 16-byte aligned");
  if (batch == 0 || batch % pps::mlp::kSamples)
    return mfail(PPS_EINVAL, "batch must be a positive multiple of 128");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  MLP_CUDA(cudaMemsetAsync(grad_out, 0, pps::mlp::kP * sizeof(float), st));
  return launch_train(m, v, tr, tg, tb, idx, pps::mlp::SampleSel{}, batch, 1, false, grad_out, st);
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
  for (uint32_t s0 = 0; s0 < m->p.steps; s0 += pps::mlp::kMaxSteps) {
    const uint32_t cnt = std::min<uint32_t>(m->p.steps - s0, pps::mlp::kMaxSteps);
    const pps::mlp::SampleSel sel{filtered->count, n, m->p.seed, frame, s0, m->p.train_min_count};
    if (int rc = launch_train(m, v, filtered->r, filtered->g, filtered->b, nullptr, sel, B, cnt, true,
                              m->dev.grad, st))
      return rc;
  }
  return PPS_OK;
}

static int launch_infer(pps_mlp* m, const pps_vertices* v, size_t n, const pps::OutPtrs& o, int all,
                        cudaStream_t st) {
  if (n == 0) return PPS_OK;
  if (n >= (1ull << 31)) return mfail(PPS_EINVAL, "n too large");
  if (m->list_cap < n) {
    // grown to the next power of two, so that frames whose vertex counts vary
    // a little do not reallocate (cudaFree waits for the device)
    size_t cap = 1;
    while (cap < n) cap *= 2;
    cudaFree(m->list);
    m->list = nullptr;
    m->list_cap = 0;
    if (cudaMalloc(&m->list, cap * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      return mfail(PPS_ENOMEM, "inference list allocation failed");
    }
    m->list_cap = cap;
  }
  const int sms = m->sms;
  MLP_CUDA(cudaMemsetAsync(m->counter, 0, sizeof(uint32_t), st));
  const int cgrid = static_cast<int>((n + 256 * pps::mlp::kCompactPer - 1) / (256 * pps::mlp::kCompactPer));
  const int vec = reinterpret_cast<uintptr_t>(o.count) % 16 == 0 &&
                  reinterpret_cast<uintptr_t>(o.status) % 4 == 0;
  pps::mlp::k_mlp_compact<<<cgrid, 256, 0, st>>>(n, o.status, o.count, m->p.infer_max_count, all,
                                                 vec, m->list, m->counter);
  MLP_CUDA(cudaGetLastError());
  const int grid = static_cast<int>(std::min<size_t>(static_cast<size_t>(sms) * 4, (n + 127) / 128));
  pps::mlp::k_mlp_infer_tc<<<grid, 128, pps::mlp::tc::kSmemBytes, st>>>(m->dev, vptrs(v), m->list,
                                                                        m->counter, o, all);
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
