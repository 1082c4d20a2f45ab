// Learned fallback: a small MLP trained online on well-populated cells and
// evaluated for vertices whose cell holds too few samples (Sec. 3.3 motivates
// a fallback for low-density voxels; the network is this library's).
//
// Network: input 80 = per axis sin/cos(pi 2^k p), k = 0..11, of the position
// normalized to a box (72), the normal (3), 5 zeros; three hidden layers of
// 64 with ReLU; linear RGB output.  BF16 weights and activations, FP32
// accumulation, on the fifth-generation tensor cores: tcgen05.mma from
// shared-memory tiles in the canonical K-major layout into tensor memory,
// tcgen05.ld back to registers for the bias / ReLU / rounding epilogues.
// Inference: a CTA of 128 threads evaluates 128 vertices per tile.
// Training: a CTA of 128 threads takes 128 samples through the forward pass,
// the delta chain and the weight gradients X^T dZ (products over the samples,
// from transposed tiles the epilogues write), reduced into an FP32 gradient
// with atomics; Adam updates FP32 master weights and refreshes the BF16
// copies.
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
  int32_t* idx;   // [batch] training sample vertex indices
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
// One pass: each thread looks at 4 consecutive vertices, a CTA-wide scan
// places its CTA's candidates, and one atomic per CTA (1,024 vertices)
// reserves their places in the list.
constexpr int kCompactPer = 4;
__global__ void __launch_bounds__(256) k_mlp_compact(size_t n, const uint8_t* status,
                                                     const uint32_t* count, uint32_t max_count,
                                                     int all, int32_t* list, uint32_t* counter) {
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t j0 = (static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x) * kCompactPer;
  bool f[kCompactPer];
  uint32_t mine = 0;
#pragma unroll
  for (int q = 0; q < kCompactPer; ++q) {
    const size_t j = j0 + q;
    f[q] = j < n && (all || (status[j] != PPS_STATUS_OVERFLOW && count[j] < max_count));
    mine += f[q] ? 1u : 0u;
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

// Wait for the mbarrier phase `parity`; gives up after about two seconds.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
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
    if (globaltimer_ns() - t0 > 2000000000ull) return false;
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
__device__ __forceinline__ void encode_row(unsigned char* x, int r, const VertexIn& vi, bool valid) {
#pragma unroll
  for (int kb = 0; kb < 9; ++kb) {
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
  const uint4 nv = valid ? make_uint4(pack2(vi.nr[0], vi.nr[1]), pack2(vi.nr[2], 0.f), 0u, 0u)
                         : make_uint4(0u, 0u, 0u, 0u);
  st16(x, cm(r, 72, 80), nv);
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
      w[q] = pack2(fmaxf(__uint_as_float(acc[c]) + bias[c], 0.f),
                   fmaxf(__uint_as_float(acc[c + 1]) + bias[c + 1], 0.f));
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
  for (uint32_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    tc::encode_row(s.act, tid, vi, j >= 0);
    // the next tile's vertex, loaded while this tile goes through the layers
    const int64_t jn = row_of(tile + gridDim.x);
    const VertexIn vn = load_vertex(d, v, jn);
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

// ---------------------------------------------------------------- training on tcgen05
// One CTA of 128 threads takes 128 samples (the MMA's M).  Every operand is a
// K-major BF16 tile in the canonical no-swizzle layout, so the products that
// run over the samples read transposed copies that the epilogues write beside
// the row-per-sample tiles:
//   forward   Z_l = X_l W_l^T        A = X_l   [sample][in],  B = W_l   [out][in]
//   backward  dH_l = dZ_{l+1} W_{l+1} A = dZ    [sample][out], B = W^T   [in][out]
//   gradient  gW_l^T = X_l^T dZ_l    A = X_l^T [in][sample],  B = dZ^T  [out][sample]
// (M = 128 rows for the gradients: rows past the layer's inputs read the next
// tile and are ignored).  Deltas are rounded to BF16 where the oracle rounds
// them; weight and bias gradients are summed over the CTA's samples in FP32
// and added to the gradient with atomics.
namespace tct {
constexpr uint32_t kTmemCols = 512;  // [0, 64): layer products, then the four gradients

struct Smem {
  alignas(128) unsigned char act[128 * 80 * 2];  // X0, then H1..H3 [sample][feature]
  alignas(128) unsigned char xt0[80 * 128 * 2];  // X0^T [feature][sample]
  alignas(128) unsigned char ht[3][64 * 128 * 2];  // H1^T..H3^T
  alignas(128) unsigned char dz[128 * 64 * 2];   // dY (K = 16), then dZ3, dZ2 [sample][out]
  alignas(128) unsigned char dzt[3][64 * 128 * 2];  // dZ1^T..dZ3^T [out][sample]
  alignas(128) unsigned char dyt[16 * 128 * 2];  // dY^T [out][sample]
  alignas(128) unsigned char w1[64 * 80 * 2];    // W_l [out][in]
  alignas(128) unsigned char w2[64 * 64 * 2];
  alignas(128) unsigned char w3[64 * 64 * 2];
  alignas(128) unsigned char w4[16 * 64 * 2];
  alignas(128) unsigned char wt2[64 * 64 * 2];   // W_l^T [in][out]
  alignas(128) unsigned char wt3[64 * 64 * 2];
  alignas(128) unsigned char wt4[64 * 16 * 2];
  float bias[3 * 64 + 16];
  alignas(8) unsigned long long mbar;
  uint32_t tmem;
};
constexpr size_t kSmemBytes = sizeof(Smem) + 128;

__device__ __forceinline__ void st_b16(unsigned char* base, uint32_t off, float x) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(x);
}
__device__ __forceinline__ float ld_b16(const unsigned char* base, uint32_t off) {
  return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(base + off));
}

// Issue `ksteps` MMAs of K = 16 (A and B advance two core matrices, 256 bytes,
// per step) into tensor-memory column `dcol`; product() also commits them to
// the mbarrier.
__device__ __forceinline__ void issue(uint32_t tmem, uint32_t dcol, uint32_t a, uint32_t sboa,
                                      uint32_t b, uint32_t sbob, uint32_t n, int ksteps) {
  const uint32_t id = tc::idesc(128, n);
  for (int k = 0; k < ksteps; ++k)
    tc::mma_bf16(tmem + dcol, tc::sdesc(a + 256u * k, sboa), tc::sdesc(b + 256u * k, sbob), id,
                 k > 0 ? 1u : 0u);
}

__device__ __forceinline__ void product(uint32_t tmem, uint32_t dcol, uint32_t a, uint32_t sboa,
                                        uint32_t b, uint32_t sbob, uint32_t n, int ksteps,
                                        uint32_t mbar) {
  issue(tmem, dcol, a, sboa, b, sbob, n, ksteps);
  tc::commit(mbar);
}

// Tensor-memory columns of the weight gradient gW_l^T (layer products use
// columns [0, 64)).
__device__ __forceinline__ uint32_t gcol(int l) { return l == 3 ? 64u : 128u + 64u * l; }

__device__ __forceinline__ void sync_tc() {
  tc::fence_smem_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
}
}  // namespace tct

__global__ void __launch_bounds__(128, 1) k_mlp_grad_tc(Dev d, VertexPtrs v, const float* tr,
                                                        const float* tg, const float* tb,
                                                        const int32_t* idx, uint32_t batch) {
  extern __shared__ unsigned char smem_raw[];
  tct::Smem& s = *reinterpret_cast<tct::Smem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int tid = threadIdx.x, warp = tid >> 5;
  // weights: W_l as in inference, and W_l^T for the backward products
  const uint4* wb4 = reinterpret_cast<const uint4*>(d.wb);
  for (int c = tid; c < 64 * kIn / 8; c += blockDim.x)
    tc::st16(s.w1, tc::cm(c / 10, 8 * (c % 10), kIn), __ldg(wb4 + bW1 / 8 + c));
  for (int c = tid; c < 64 * kHid / 8; c += blockDim.x) {
    tc::st16(s.w2, tc::cm(c / 8, 8 * (c % 8), kHid), __ldg(wb4 + bW2 / 8 + c));
    tc::st16(s.w3, tc::cm(c / 8, 8 * (c % 8), kHid), __ldg(wb4 + bW3 / 8 + c));
  }
  for (int c = tid; c < 16 * kHid / 8; c += blockDim.x)
    tc::st16(s.w4, tc::cm(c / 8, 8 * (c % 8), kHid), __ldg(wb4 + bW4 / 8 + c));
  // W[o][in] -> W^T[in][o]: 8 inputs of one output per 16-byte load
  auto scatter_t = [&](unsigned char* dst, int K, int o, int in0, uint4 w) {
    const uint32_t q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      *reinterpret_cast<uint16_t*>(dst + tc::cm(in0 + 2 * e, o, K)) = static_cast<uint16_t>(q[e]);
      *reinterpret_cast<uint16_t*>(dst + tc::cm(in0 + 2 * e + 1, o, K)) = static_cast<uint16_t>(q[e] >> 16);
    }
  };
#pragma unroll 4
  for (int c = tid; c < 64 * 64 / 8; c += blockDim.x) {
    scatter_t(s.wt2, 64, c / 8, 8 * (c % 8), __ldg(wb4 + bW2 / 8 + c));
    scatter_t(s.wt3, 64, c / 8, 8 * (c % 8), __ldg(wb4 + bW3 / 8 + c));
  }
  for (int c = tid; c < 16 * 64 / 8; c += blockDim.x)
    scatter_t(s.wt4, 16, c / 8, 8 * (c % 8), __ldg(wb4 + bW4 / 8 + c));
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
                 "r"(tct::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // this thread's sample: encoded row and its transpose
  const uint32_t si = blockIdx.x * 128u + tid;
  const int64_t j = si < batch ? idx[si] : -1;
  const VertexIn vi = load_vertex(d, v, j);
  tc::encode_row(s.act, tid, vi, j >= 0);
  __syncwarp();
  for (int f = 0; f < kIn; ++f)
    *reinterpret_cast<__nv_bfloat16*>(s.xt0 + tc::cm(f, tid, 128)) =
        *reinterpret_cast<const __nv_bfloat16*>(s.act + tc::cm(tid, f, kIn));
  tct::sync_tc();
  const uint32_t tmem = s.tmem;
  const uint32_t trow = tmem + (static_cast<uint32_t>(warp * 32) << 16);
  uint32_t parity = 0;
  bool ok = true;
  auto wait = [&]() {
    ok = ok && __syncthreads_and(tc::mbar_wait(mbar, parity)) != 0;
    parity ^= 1u;
    tc::fence_after();
  };
  uint32_t acc[64];
  // ---- forward
  for (int layer = 0; layer < 3 && ok; ++layer) {
    if (tid == 0)
      tct::product(tmem, 0, smem_u32(s.act), layer == 0 ? 1280u : 1024u,
                   smem_u32(layer == 0 ? s.w1 : layer == 1 ? s.w2 : s.w3),
                   layer == 0 ? 1280u : 1024u, 64, layer == 0 ? 5 : 4, mbar);
    wait();
    if (!ok) break;
    tc::tmem_ld_x64(trow, acc);
    tc::tmem_wait_ld();
    tc::hidden_row(s.act, tid, acc, s.bias + 64 * layer);
    __syncwarp();
    for (int f = 0; f < 64; ++f)
      *reinterpret_cast<__nv_bfloat16*>(s.ht[layer] + tc::cm(f, tid, 128)) =
          *reinterpret_cast<const __nv_bfloat16*>(s.act + tc::cm(tid, f, 64));
    tct::sync_tc();
  }
  float dy[3] = {0.f, 0.f, 0.f};
  if (ok) {
    if (tid == 0)
      tct::product(tmem, 0, smem_u32(s.act), 1024u, smem_u32(s.w4), 1024u, 16, 4, mbar);
    wait();
  }
  if (ok) {
    uint32_t y[16];
    tc::tmem_ld_x16(trow, y);
    tc::tmem_wait_ld();
    // output delta (y - target) / batch, rounded to BF16; K = 16 tile and its transpose
    const float invb = 1.0f / static_cast<float>(batch);
    if (j >= 0) {
      const float t3[3] = {__ldg(tr + j), __ldg(tg + j), __ldg(tb + j)};
#pragma unroll
      for (int o = 0; o < 3; ++o)
        dy[o] = __bfloat162float(__float2bfloat16_rn(
            (__uint_as_float(y[o]) + s.bias[192 + o] - t3[o]) * invb));
    }
    tc::st16(s.dz, tc::cm(tid, 0, 16), make_uint4(pack2(dy[0], dy[1]), pack2(dy[2], 0.f), 0u, 0u));
    tc::st16(s.dz, tc::cm(tid, 8, 16), make_uint4(0u, 0u, 0u, 0u));
#pragma unroll
    for (int o = 0; o < 16; ++o) tct::st_b16(s.dyt, tc::cm(o, tid, 128), o < 3 ? dy[o] : 0.f);
    tct::sync_tc();
  }
  // ---- backward: dH_l = dZ_{l+1} W_{l+1}, masked by H_l > 0 and rounded; each
  // step also computes the weight gradient of the layer whose delta it reads,
  // gW_{l+1}^T = X_{l+1}^T dZ_{l+1} (K = 128 samples), into its own columns
  auto grad_out = [&](int l) {  // atomics of gW_l^T from tensor-memory columns gcol(l)
    const int in_dim = l == 0 ? kIn : kHid;
    const int off = l == 0 ? oW1 : l == 1 ? oW2 : l == 2 ? oW3 : oW4;
    const uint32_t col = tct::gcol(l);
    if (l < 3) {
      tc::tmem_ld_x64(trow + col, acc);
      tc::tmem_wait_ld();
      if (tid < in_dim)
        for (int o = 0; o < 64; ++o) atomicAdd(d.grad + off + o * in_dim + tid, __uint_as_float(acc[o]));
    } else {
      uint32_t g4[16];
      tc::tmem_ld_x16(trow + col, g4);
      tc::tmem_wait_ld();
      if (tid < in_dim)
        for (int o = 0; o < kOut; ++o) atomicAdd(d.grad + off + o * in_dim + tid, __uint_as_float(g4[o]));
    }
  };
  auto grad_issue = [&](int l) {  // gW_l^T = X_l^T dZ_l (l = 3: dY)
    const unsigned char* ga = l == 0 ? s.xt0 : s.ht[l - 1];
    const unsigned char* gb = l < 3 ? s.dzt[l] : s.dyt;
    tct::issue(tmem, tct::gcol(l), smem_u32(ga), 2048u, smem_u32(gb), 2048u, l < 3 ? 64u : 16u, 8);
  };
  for (int l = 2; l >= 0 && ok; --l) {  // produces dZ3 (l = 2), dZ2, dZ1
    if (tid == 0) {
      if (l == 2)
        tct::issue(tmem, 0, smem_u32(s.dz), 256u, smem_u32(s.wt4), 256u, 64, 1);
      else
        tct::issue(tmem, 0, smem_u32(s.dz), 1024u, smem_u32(l == 1 ? s.wt3 : s.wt2), 1024u, 64, 4);
      grad_issue(l + 1);
      tc::commit(mbar);
    }
    wait();
    if (!ok) break;
    tc::tmem_ld_x64(trow, acc);
    tc::tmem_wait_ld();
    float z[64];
#pragma unroll
    for (int f = 0; f < 64; ++f) {
      const float h = tct::ld_b16(s.ht[l], tc::cm(f, tid, 128));
      z[f] = __bfloat162float(__float2bfloat16_rn(h > 0.f ? __uint_as_float(acc[f]) : 0.f));
    }
    // the products above have completed: dz may be overwritten
    if (l > 0) {
#pragma unroll
      for (int kb = 0; kb < 8; ++kb)
        tc::st16(s.dz, tc::cm(tid, 8 * kb, 64),
                 make_uint4(pack2(z[8 * kb], z[8 * kb + 1]), pack2(z[8 * kb + 2], z[8 * kb + 3]),
                            pack2(z[8 * kb + 4], z[8 * kb + 5]), pack2(z[8 * kb + 6], z[8 * kb + 7])));
    }
#pragma unroll
    for (int f = 0; f < 64; ++f) tct::st_b16(s.dzt[l], tc::cm(f, tid, 128), z[f]);
    grad_out(l + 1);
    tct::sync_tc();
  }
  if (ok) {
    if (tid == 0) {
      grad_issue(0);
      tc::commit(mbar);
    }
    wait();
    if (ok) grad_out(0);
  }
  // ---- bias gradients: sums of the rounded deltas over the samples
  if (ok) {
    for (int c = tid; c < 3 * kHid + kOut; c += blockDim.x) {
      const unsigned char* row = c < 192 ? s.dzt[c / 64] : s.dyt;
      const int o = c < 192 ? c % 64 : c - 192;
      const int ob = c < 64 ? oB1 : c < 128 ? oB2 : c < 192 ? oB3 : oB4;
      float sum = 0.f;
      for (int kb = 0; kb < 16; ++kb) {  // 8 samples per 16-byte chunk
        const uint4 q = *reinterpret_cast<const uint4*>(row + tc::cm(o, 8 * kb, 128));
        sum += (lo_f(q.x) + hi_f(q.x)) + (lo_f(q.y) + hi_f(q.y)) + (lo_f(q.z) + hi_f(q.z)) +
               (lo_f(q.w) + hi_f(q.w));
      }
      atomicAdd(d.grad + ob + o, sum);
    }
  }
  if (!ok && tid == 0) atomicOr(d.err, 1u);
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tct::kTmemCols)
                 : "memory");
}

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
  int sms = 0;                  // multiprocessors of the device
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
  if (e == cudaSuccess) e = cudaMalloc(&m->dev.idx, p->batch * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->dev.err, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&m->counter, sizeof(uint32_t));
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
        cudaFuncSetAttribute(pps::mlp::k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
    cudaFree(m->dev.idx);
    cudaFree(m->dev.err);
    cudaFree(m->counter);
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
  cudaFree(m->dev.err);
  cudaFree(m->counter);
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
  if (err) return mfail(PPS_EDEVICE, "an inference launch gave up waiting for the tensor cores");
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
  pps::mlp::k_mlp_grad_tc<<<batch / 128, 128, pps::mlp::tct::kSmemBytes, st>>>(d, vptrs(v), tr, tg,
                                                                              tb, idx, batch);
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
    pps::mlp::k_mlp_grad_tc<<<B / 128, 128, pps::mlp::tct::kSmemBytes, st>>>(
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
  if (n >= (1ull << 31)) return mfail(PPS_EINVAL, "n too large");
  if (m->list_cap < n) {
    cudaFree(m->list);
    m->list = nullptr;
    m->list_cap = 0;
    if (cudaMalloc(&m->list, n * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      return mfail(PPS_ENOMEM, "inference list allocation failed");
    }
    m->list_cap = n;
  }
  const int sms = m->sms;
  MLP_CUDA(cudaMemsetAsync(m->counter, 0, sizeof(uint32_t), st));
  const int cgrid = static_cast<int>((n + 256 * pps::mlp::kCompactPer - 1) / (256 * pps::mlp::kCompactPer));
  pps::mlp::k_mlp_compact<<<cgrid, 256, 0, st>>>(n, o.status, o.count, m->p.infer_max_count, all,
                                                 m->list, m->counter);
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
