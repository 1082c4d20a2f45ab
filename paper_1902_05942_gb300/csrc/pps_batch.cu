// Batched filtering of several views in one persistent launch replayed from a
// CUDA graph (see pps_batch_create in include/pps.h).
//
// Per frame only the views' cameras and the frame number change.  They live in
// a descriptor array in device memory, uploaded by a copy node at the start
// of the graph from a pinned host buffer; two buffers (and two instantiated
// graphs) alternate so that filling the next frame's descriptors never races
// with the copy of the previous one.
#include <cstring>
#include <string>
#include <vector>

#include "pps.h"
#include "pps_internal.h"

struct pps_batch {
  int device = 0;
  std::vector<pps_table*> tables;
  std::vector<pps::ViewDesc> base;  // descriptors without camera and frame
  uint32_t total_tiles = 0;
  bool temporal = false;
  float alpha = 0.f;
  pps::MultiPlan plan;
  pps::ViewDesc* dviews[2] = {nullptr, nullptr};
  pps::ViewDesc* hviews[2] = {nullptr, nullptr};
  pps::Ctrl* ctrl = nullptr;
  uint32_t* gstash = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  unsigned long long runs = 0;
};

namespace {

int bfail(int code, const std::string& msg) { return pps::record_error(code, msg.c_str()); }

void release(pps_batch* b) {
  for (int k = 0; k < 2; ++k) {
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
    if (b->done[k]) cudaEventDestroy(b->done[k]);
    cudaFree(b->dviews[k]);
    cudaFreeHost(b->hviews[k]);
  }
  cudaFree(b->ctrl);
  cudaFree(b->gstash);
}

}  // namespace

extern "C" {

int pps_batch_create(pps_batch** out, const pps_view* views, uint32_t nviews, int blend,
                     float alpha) {
  if (!out || !views || nviews == 0 || nviews > 4096) return bfail(PPS_EINVAL, "bad views");
  *out = nullptr;
  pps_batch* b = new (std::nothrow) pps_batch();
  if (!b) return bfail(PPS_ENOMEM, "host allocation failed");
  cudaGetDevice(&b->device);
  b->alpha = alpha;
  int batch = 2, block = 512;
  const size_t ftile = static_cast<size_t>(pps::fused_tile_size());
  for (uint32_t i = 0; i < nviews; ++i) {
    const pps_view& v = views[i];
    if (!v.table || !v.out.r || !v.out.g || !v.out.b || (v.n && (!v.v.px || !v.v.py || !v.v.pz ||
        !v.v.nx || !v.v.ny || !v.v.nz || !v.v.r || !v.v.g || !v.v.b))) {
      delete b;
      return bfail(PPS_EINVAL, "view " + std::to_string(i) + ": table, vertices and r, g, b required");
    }
    if (v.v.dist || v.v.extra) {
      delete b;
      return bfail(PPS_EINVAL, "view " + std::to_string(i) + ": batched views take no dist or extra arrays");
    }
    pps::ViewDesc vd{};
    bool tmp = false;
    int bw = 2, blk = 512;
    if (int rc = pps::table_for_batch(v.table, v.n, &vd, &bw, &blk, &tmp, nullptr)) {
      delete b;
      return rc;
    }
    if (i == 0) {
      batch = bw;
      block = blk;
    }
    vd.v = pps::VertexPtrs{v.v.px, v.v.py, v.v.pz, v.v.nx, v.v.ny, v.v.nz, v.v.r, v.v.g, v.v.b,
                           v.v.id, v.v.id_base, v.v.stream_id, v.v.dist, v.v.extra};
    vd.o = pps::OutPtrs{v.out.r, v.out.g, v.out.b, v.out.count, v.out.status};
    vd.n = v.n;
    vd.tile_base = b->total_tiles;
    vd.ntiles = static_cast<uint32_t>((v.n + ftile - 1) / ftile);
    vd.vec = pps::vec_inputs_host(vd.v) ? 1 : 0;
    vd.ovec = pps::vec_outputs_host(vd.o) ? 1 : 0;
    vd.blended = blend && tmp ? 1 : 0;
    vd.sweep = pps::sweep_pays_host(vd.t, v.n) ? 1 : 0;
    b->temporal = b->temporal || tmp;
    b->total_tiles += vd.ntiles;
    b->base.push_back(vd);
    b->tables.push_back(v.table);
  }
  if (blend && (!(alpha <= 1.0f) || alpha != alpha)) {
    delete b;
    return bfail(PPS_EINVAL, "alpha must be finite and <= 1");
  }
  cudaError_t e = pps::plan_multi(b->total_tiles, b->temporal, batch, block, &b->plan);
  const size_t bytes = nviews * sizeof(pps::ViewDesc);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaMalloc(&b->dviews[k], bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&b->hviews[k], bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming);
    if (e == cudaSuccess) std::memcpy(b->hviews[k], b->base.data(), bytes);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->ctrl, sizeof(pps::Ctrl));
  if (e == cudaSuccess) e = cudaMemset(b->ctrl, 0, sizeof(pps::Ctrl));
  if (e == cudaSuccess && b->plan.global_stash)
    e = cudaMalloc(&b->gstash, static_cast<size_t>(b->total_tiles) * ftile * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  // capture: descriptor upload, counter resets, the persistent kernel
  cudaStream_t cs = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->dviews[k], b->hviews[k], bytes, cudaMemcpyHostToDevice, cs);
    for (size_t i = 0; i < b->base.size() && e == cudaSuccess; ++i)
      e = cudaMemsetAsync(b->base[i].t.ctrl, 0, pps::kCtrlFrameBytes, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ctrl, 0, pps::kCtrlFrameBytes, cs);
    if (e == cudaSuccess)
      e = pps::launch_multi(b->dviews[k], nviews, b->total_tiles, b->ctrl, b->temporal, alpha,
                            b->plan, b->gstash, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[k], g, 0);
    if (g) cudaGraphDestroy(g);
  }
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    release(b);
    delete b;
    cudaGetLastError();
    return bfail(e == cudaErrorMemoryAllocation ? PPS_ENOMEM : PPS_ECUDA,
                 std::string("pps_batch_create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return PPS_OK;
}

int pps_batch_run(pps_batch* b, const pps_camera* cams, uint32_t frame, void* stream) {
  if (!b || !cams) return bfail(PPS_EINVAL, "NULL argument");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
    return bfail(PPS_EINVAL, "the batch's device is not the current device");
  const int k = static_cast<int>(b->runs & 1);
  // the buffer's previous upload must have completed before it is refilled
  if (b->runs >= 2) {
    const cudaError_t e = cudaEventSynchronize(b->done[k]);
    if (e != cudaSuccess) return bfail(PPS_ECUDA, std::string("pps_batch_run: ") + cudaGetErrorString(e));
  }
  for (size_t i = 0; i < b->base.size(); ++i) {
    pps::ViewDesc vd = b->base[i];
    vd.kc.cam[0] = cams[i].pos[0];
    vd.kc.cam[1] = cams[i].pos[1];
    vd.kc.cam[2] = cams[i].pos[2];
    vd.kc.frame = frame;
    pps::set_round_keys(vd.kc);
    b->hviews[k][i] = vd;
  }
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGraphLaunch(b->exec[k], st);
  if (e == cudaSuccess) e = cudaEventRecord(b->done[k], st);
  if (e != cudaSuccess) return bfail(PPS_ECUDA, std::string("pps_batch_run: ") + cudaGetErrorString(e));
  ++b->runs;
  return PPS_OK;
}

int pps_batch_destroy(pps_batch* b) {
  if (!b) return PPS_OK;
  cudaDeviceSynchronize();
  release(b);
  delete b;
  return PPS_OK;
}

}  // extern "C"
