// Host-side declarations shared by the C ABI and the kernel launchers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "pps_device.cuh"

struct pps_params;

namespace pps {

// Launch geometry of the persistent filter kernel for one call.
struct FusedPlan {
  int grid = 0;            // CTAs (a multiple of the SM count: SMs x CTAs per SM)
  int block = 0;           // threads per CTA
  int batch = 4;           // vertices per thread per insert step (2 or 4)
  uint32_t cap_tiles = 0;  // tiles one CTA may take (stash capacity)
  size_t smem = 0;         // dynamic shared memory per CTA (stash of cap_tiles tiles)
  bool global_stash = false;
  bool evict = false;      // the kernel variant for an evicting history
  bool neigh = false;      // the kernel variant with the neighborhood search
  int key_warps = 0;       // > 0: the pipelined insert (k_fused_ws) with this many key warps
  int merge = 2;           // pipelined insert: warp aggregation of equal keys (pps_tuning.merge)
};

// How a table's persistent launch inserts (pps_tuning.insert / key_warps).
struct InsertShape {
  int pipelined = 1;  // 1: key warps and probe warps on alternate chunks; 0: per thread
  int key_warps = 8;  // of the 16 warps of a CTA (4, 8 or 12)
  int merge = 2;      // 1 none, 2 where neighbouring lanes repeat a key, 3 always
};

// One view of a batched launch: its table, key constants, vertices and
// outputs, and its place in the batch's tile space.
struct ViewDesc {
  KeyConst kc;
  TableDev t;
  VertexPtrs v;
  OutPtrs o;
  unsigned long long n;
  uint32_t tile_base;  // first tile of this view in the batch
  uint32_t ntiles;
  int vec, ovec;
  int blended;  // blend this view's cells (temporal table and blending requested)
  int sweep;    // zero this view's slot table by a sweep at the end
};

struct MultiPlan {
  int grid = 0, block = 0, batch = 2;
  uint32_t cap_tiles = 0;
  size_t smem = 0;
  bool global_stash = false;
};

// Plan / launch the batched persistent kernel over `total_tiles` tiles of the
// views in device memory (`views`, nviews entries); `ctrl` carries the grid
// barrier and the tile counter; `gstash` (total_tiles tiles) is used when the
// stash does not fit on chip.
cudaError_t plan_multi(size_t total_tiles, bool temporal, int batch, int block, MultiPlan* plan);
cudaError_t launch_multi(const ViewDesc* views, uint32_t nviews, uint32_t total_tiles, Ctrl* ctrl,
                         bool temporal, float alpha, const MultiPlan& plan, uint32_t* gstash,
                         cudaStream_t st);
bool vec_inputs_host(const VertexPtrs& v);
bool vec_outputs_host(const OutPtrs& o);
bool sweep_pays_host(const TableDev& t, size_t vertices);

cudaError_t launch_insert(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                          uint32_t* id_out, uint32_t tile_base, int batch, cudaStream_t st);
cudaError_t launch_query(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                         const uint32_t* id_in, const OutPtrs& o, bool blended, uint32_t id_limit,
                         cudaStream_t st);
cudaError_t launch_keys(const KeyConst& kc, const VertexPtrs& v, size_t n, uint32_t* h_out,
                        uint32_t* f_out, cudaStream_t st);
cudaError_t launch_blend(const KeyConst& kc, const TableDev& t, uint32_t ntiles, float alpha,
                         cudaStream_t st);
cudaError_t launch_clear(const TableDev& t, uint32_t ntiles, cudaStream_t st);
// Evicting history: lower every entry's priority by `by` (epoch rebase).
cudaError_t launch_hist_age(const TableDev& t, uint32_t by, cudaStream_t st);
// Multi-level accumulation: vertices with fine status LOWCOUNT take the
// coarse resolution's value, count and status COARSE (unless the coarse
// insert overflowed).  `fine_status` may alias o.status.
cudaError_t launch_combine_coarse(size_t n, const uint8_t* fine_status, const OutPtrs& coarse,
                                  const OutPtrs& o, cudaStream_t st);
cudaError_t launch_count_nonzero(const void* base, uint32_t stride, uint32_t off, uint32_t width,
                                 uint64_t n, unsigned long long* out, cudaStream_t st);
cudaError_t plan_fused(size_t n, bool temporal, int batch, FusedPlan* plan, bool evict = false,
                       bool neigh = false, InsertShape shape = InsertShape{}, bool fixed = false);
cudaError_t launch_fused(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                         const OutPtrs& o, bool temporal, bool blend, float alpha,
                         const FusedPlan& plan, uint32_t* gstash, uint32_t* nq, cudaStream_t st);

int tile_size();        // vertices (and cell ids) per tile of the split path
int fused_tile_size();  // vertices (and cell ids) per tile of the persistent kernel
bool aligned16(const void* p);

int record_error(int code, const char* msg);  // message for pps_last_error()
const char* last_error_text();                // the message pps_last_error() returns
std::string device_error_text(unsigned int word);  // the bits of a device error word
// Checks of table parameters shared by pps_create and pps_filter_noalloc
// (PPS_OK, or PPS_EINVAL with the reason recorded for pps_last_error()).
int check_params(const pps_params* p);

// Self-test of the tensor-core kernels' bounded mbarrier wait (pps_mlp.cu).
cudaError_t launch_selftest_mbar(unsigned long long limit_ns, unsigned int* err, cudaStream_t st);

}  // namespace pps

struct pps_table;

namespace pps {
int table_for_batch(pps_table* t, size_t n, ViewDesc* vd, int* batch, int* block, bool* temporal,
                    cudaStream_t st);

}  // namespace pps
