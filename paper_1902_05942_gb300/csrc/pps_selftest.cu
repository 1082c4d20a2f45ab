// Self-tests of the bounded device waits: each waits on a condition that
// never comes true, gives up after a short limit and reports it through the
// device error word, the same way a stuck frame would.
#include <cuda_runtime.h>

#include <string>

#include "pps.h"
#include "pps_device.cuh"
#include "pps_internal.h"

namespace pps {
namespace {

// Every CTA waits at the grid barrier for one CTA more than the launch has.
__global__ void k_selftest_barrier(Ctrl* c, unsigned long long limit_ns) {
  grid_barrier(c, gridDim.x + 1u, limit_ns);
}

}  // namespace
}  // namespace pps

extern "C" int pps_selftest_wait(int kind, uint32_t limit_us, uint32_t* error_word) {
  if (!error_word) return pps::record_error(PPS_EINVAL, "error_word is NULL");
  if (kind != 0 && kind != 1) return pps::record_error(PPS_EINVAL, "kind must be 0 or 1");
  if (limit_us < 1 || limit_us > 2000000u)
    return pps::record_error(PPS_EINVAL, "limit_us must be in [1, 2000000]");
  *error_word = 0;
  const unsigned long long limit_ns = 1000ull * limit_us;
  void* mem = nullptr;
  const size_t bytes = kind == 0 ? sizeof(pps::Ctrl) : sizeof(unsigned int);
  cudaError_t e = cudaMalloc(&mem, bytes);
  if (e == cudaSuccess) e = cudaMemset(mem, 0, bytes);
  if (e == cudaSuccess) {
    if (kind == 0) {
      pps::k_selftest_barrier<<<4, 32>>>(static_cast<pps::Ctrl*>(mem), limit_ns);
      e = cudaGetLastError();
    } else {
      e = pps::launch_selftest_mbar(limit_ns, static_cast<unsigned int*>(mem), nullptr);
    }
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  unsigned int word = 0;
  if (e == cudaSuccess) {
    const void* src = kind == 0 ? static_cast<const void*>(&static_cast<pps::Ctrl*>(mem)->error) : mem;
    e = cudaMemcpy(&word, src, sizeof(word), cudaMemcpyDeviceToHost);
  }
  cudaFree(mem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    const std::string msg = std::string("pps_selftest_wait: ") + cudaGetErrorString(e);
    return pps::record_error(PPS_ECUDA, msg.c_str());
  }
  *error_word = word;
  return PPS_OK;
}
