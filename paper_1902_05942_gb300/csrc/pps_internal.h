// Host-side declarations shared by the C ABI and the kernel launchers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "pps_device.cuh"

namespace pps {

// Launch geometry of the persistent filter kernel for one call.
struct FusedPlan {
  int grid = 0;          // CTAs (a multiple of the SM count: SMs x CTAs per SM)
  int block = 0;         // threads per CTA
  size_t chunk = 0;      // vertices per CTA (multiple of 4)
  size_t smem = 0;       // dynamic shared memory per CTA (stash of chunk words)
  bool global_stash = false;
};

cudaError_t launch_insert(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                          uint32_t* slot_out, cudaStream_t st);
cudaError_t launch_query(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                         const uint32_t* slot_in, const OutPtrs& o, bool blended,
                         cudaStream_t st);
cudaError_t launch_keys(const KeyConst& kc, const VertexPtrs& v, size_t n, uint32_t* h_out,
                        uint32_t* f_out, cudaStream_t st);
cudaError_t launch_blend(const TableDev& t, float alpha, cudaStream_t st);
cudaError_t launch_clear_dirty(const TableDev& t, cudaStream_t st);
cudaError_t launch_count_occupied(const unsigned char* cells, uint32_t stride, uint32_t fp_off,
                                  uint32_t T, unsigned long long* out, cudaStream_t st);
cudaError_t plan_fused(size_t n, bool temporal, FusedPlan* plan);
cudaError_t launch_fused(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                         const OutPtrs& o, bool temporal, bool blend, float alpha,
                         const FusedPlan& plan, uint32_t* gstash, cudaStream_t st);

bool aligned16(const void* p);

}  // namespace pps
