// Host-side declarations shared by the C ABI and the kernel launchers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "pps_device.cuh"

namespace pps {

// Launch geometry of the persistent filter kernel for one call.
struct FusedPlan {
  int grid = 0;            // CTAs (a multiple of the SM count: SMs x CTAs per SM)
  int block = 0;           // threads per CTA
  int batch = 4;           // vertices per thread per insert step (2 or 4)
  uint32_t cap_tiles = 0;  // tiles one CTA may take (stash capacity)
  size_t smem = 0;         // dynamic shared memory per CTA (stash of cap_tiles tiles)
  bool global_stash = false;
};

cudaError_t launch_insert(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                          uint32_t* id_out, uint32_t tile_base, int batch, cudaStream_t st);
cudaError_t launch_query(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                         const uint32_t* id_in, const OutPtrs& o, bool blended, uint32_t id_limit,
                         cudaStream_t st);
cudaError_t launch_keys(const KeyConst& kc, const VertexPtrs& v, size_t n, uint32_t* h_out,
                        uint32_t* f_out, cudaStream_t st);
cudaError_t launch_blend(const TableDev& t, uint32_t ntiles, float alpha, cudaStream_t st);
cudaError_t launch_clear(const TableDev& t, uint32_t ntiles, cudaStream_t st);
cudaError_t launch_count_nonzero(const void* base, uint32_t stride, uint32_t off, uint32_t width,
                                 uint64_t n, unsigned long long* out, cudaStream_t st);
cudaError_t plan_fused(size_t n, bool temporal, int batch, FusedPlan* plan);
cudaError_t launch_fused(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                         const OutPtrs& o, bool temporal, bool blend, float alpha,
                         const FusedPlan& plan, uint32_t* gstash, cudaStream_t st);

int tile_size();        // vertices (and cell ids) per tile of the split path
int fused_tile_size();  // vertices (and cell ids) per tile of the persistent kernel
bool aligned16(const void* p);

int record_error(int code, const char* msg);  // message for pps_last_error()

}  // namespace pps
