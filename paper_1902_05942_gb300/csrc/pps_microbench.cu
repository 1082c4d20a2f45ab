// Memory-operation rate microbenchmark (measurement only; not part of the
// filter).  Measures how many random 32-bit compare-and-swaps, 16-byte vector
// float reductions, scalar float reductions and 16-byte gathers the GPU
// completes per second over a region of a given size, so that the filter's
// L2 atomic traffic can be stated as a fraction of what the chip sustains.
//
// Addresses are a counter-based scramble of (thread, iteration), aligned to
// the operation's width and spread uniformly over the region; nothing is read
// to form them.  A region well below the L2 size measures L2-resident rates; a
// region well above it measures rates that include DRAM fills.
#include <cstdint>
#include <cuda_runtime.h>

#include "pps_bench.h"

namespace {

__device__ __forceinline__ uint32_t scramble(uint32_t x) {
  // integer finaliser of MurmurHash3 (Appleby): a bijection on 32 bits
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

__global__ void k_rate(unsigned char* base, uint64_t units, uint32_t unit_bytes, int kind,
                       int iters, float* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.f;
  for (int i = 0; i < iters; ++i) {
    const uint64_t h = (static_cast<uint64_t>(scramble(tid * 0x9E3779B9u + i)) << 32) |
                       scramble(tid ^ (0x7F4A7C15u * (i + 1)));
    unsigned char* p = base + (h % units) * unit_bytes;
    switch (kind) {
      case PPS_RATE_RED_V4_F32:
        asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p),
                     "f"(1.f), "f"(2.f), "f"(3.f), "f"(1.f)
                     : "memory");
        break;
      case PPS_RATE_CAS_B32:
        acc += static_cast<float>(atomicCAS(reinterpret_cast<uint32_t*>(p), 0u, tid | 1u) & 1u);
        break;
      case PPS_RATE_RED_F32:
        atomicAdd(reinterpret_cast<float*>(p), 1.f);
        break;
      default: {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
        acc += v.x + v.w;
        break;
      }
    }
  }
  if (acc == 12345.f) sink[0] = acc;  // keeps the gathers and CAS results alive
}

}  // namespace

extern "C" int pps_bench_rate(int kind, size_t region_bytes, size_t ops, void* scratch,
                              void* stream, double* ops_per_second) {
  if (!scratch || !ops_per_second || region_bytes < 4096 || ops == 0 || kind < 0 ||
      kind > PPS_RATE_GATHER_V4)
    return 1;
  const uint32_t unit = 32u;  // one operation per 32-byte sector, like one table cell
  const uint64_t units = region_bytes / unit;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int block = 256;
  const int grid = sms * 8;
  const size_t threads = static_cast<size_t>(grid) * block;
  const int iters = static_cast<int>((ops + threads - 1) / threads);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* sink = reinterpret_cast<float*>(scratch);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 3;
  k_rate<<<grid, block, 0, st>>>(static_cast<unsigned char*>(scratch), units, unit, kind, 1, sink);
  cudaEventRecord(e0, st);
  k_rate<<<grid, block, 0, st>>>(static_cast<unsigned char*>(scratch), units, unit, kind, iters,
                                 sink);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return 3;
  *ops_per_second = static_cast<double>(threads) * iters / (ms * 1e-3);
  return 0;
}
