// pps_filter_noalloc: one frame of the plain filter without any device
// allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// filter: a plug-in living inside a host application that owns the GPU memory
// budget and forbids its modules to call cudaMalloc, or a real-time render
// thread that must not call cudaMalloc / cudaFree because those calls can
// block or synchronize the whole device.  For them this entry point keeps all
// of its working memory (the hashed slot index, the per-cell accumulators and
// cell records, the off-chip vertex stash and the control block) in one
// statically sized device array defined in this file.  The caller still passes
// its own inputs and outputs.
//
// The array is part of the library image: every GPU that loads the library
// holds it (kScratchBytes) until the process exits.  All calls share it and
// it keeps the last call's contents, so every call first clears the parts it
// uses; calls that overlap on the GPU (different streams, no ordering between
// them) race on it and give wrong results.
//
// Host code cannot use the array's name as a device address: there it is a
// host-side stand-in.  The first call in a CUDA context (a device's primary
// context, with that device current) therefore looks the device address up
// with cudaGetSymbolAddress and remembers it for that context; that first call
// should come before any stream capture.  A new context on the same device
// (after cudaDeviceReset, say) loads the library's kernels anew, so the
// address is looked up again there.
//
// pps_noalloc_stats reads the counters and the device error word that the
// last call left in the array (they live there too), so that a call that went
// wrong on the GPU is reported rather than overwritten by the next call.
#include <cuda.h>

#include <cstddef>
#include <cstring>
#include <mutex>
#include <string>

#include "pps.h"
#include "pps_internal.h"

namespace {

constexpr uint32_t kNoAllocMaxLog2Slots = 20;                // up to 2^20 slots (8 MB)
constexpr size_t kNoAllocMaxVertices = size_t{1} << 19;      // up to 524,288 vertices

constexpr size_t kSlotBytes = (size_t{1} << kNoAllocMaxLog2Slots) * sizeof(unsigned long long);
constexpr size_t kAccBytes = kNoAllocMaxVertices * sizeof(float4);
constexpr size_t kInfoBytes = kNoAllocMaxVertices * sizeof(uint4);
constexpr size_t kStashBytes = kNoAllocMaxVertices * sizeof(uint32_t);
constexpr size_t kCtrlBytes = 256;
constexpr size_t kOffAcc = kSlotBytes;
constexpr size_t kOffInfo = kOffAcc + kAccBytes;
constexpr size_t kOffStash = kOffInfo + kInfoBytes;
constexpr size_t kOffCtrl = kOffStash + kStashBytes;
constexpr size_t kScratchBytes = kOffCtrl + kCtrlBytes;  // 26 MB + 256 B

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The message is kept where pps_last_error() reads it.
int noalloc_fail(int code, const std::string& msg) { return pps::record_error(code, msg.c_str()); }

// The unique id of the calling thread's current CUDA context, through the
// driver's entry points (fetched once; the library does not link the driver
// library itself).  0 when there is no current context.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

int current_context_id(const char* who, unsigned long long* id) {
  static std::once_flag once;
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  if (!get_current || !get_id)
    return noalloc_fail(PPS_ECUDA, std::string(who) + ": driver context queries unavailable");
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) {
    *id = 0;
    return PPS_OK;
  }
  if (get_id(ctx, id) != CUDA_SUCCESS)
    return noalloc_fail(PPS_ECUDA, std::string(who) + ": cuCtxGetId failed");
  return PPS_OK;
}

// Device address of the scratch array in the current context: looked up once
// per context (keyed by the context's unique id, so that a context created
// after a reset of the device never gets the old context's address).
int scratch_address(const char* who, unsigned char** out) {
  static std::mutex mu;
  struct Entry {
    unsigned long long ctx;
    unsigned char* addr;
  };
  static Entry cache[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64)
    return noalloc_fail(PPS_ECUDA, std::string(who) + ": no usable current device");
  unsigned long long ctx = 0;
  if (int rc = current_context_id(who, &ctx)) return rc;
  if (ctx == 0) {
    // no context current on this thread yet: bind (and if need be create)
    // the device's primary context, which the runtime calls below use
    e = cudaSetDevice(dev);
    if (e != cudaSuccess)
      return noalloc_fail(PPS_ECUDA, std::string(who) + ": " + cudaGetErrorString(e));
    if (int rc = current_context_id(who, &ctx)) return rc;
    if (ctx == 0) return noalloc_fail(PPS_ECUDA, std::string(who) + ": no current CUDA context");
  }
  std::lock_guard<std::mutex> lock(mu);
  if (cache[dev].ctx != ctx || !cache[dev].addr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(PPS_ECUDA, std::string(who) + ": cudaGetSymbolAddress: " +
                                         cudaGetErrorString(e));
    cache[dev].ctx = ctx;
    cache[dev].addr = static_cast<unsigned char*>(p);
  }
  *out = cache[dev].addr;
  return PPS_OK;
}

}  // namespace

extern "C" int pps_filter_noalloc(const pps_params* p, const pps_camera* cam, uint32_t frame,
                                  const pps_vertices* v, size_t n, const pps_output* out,
                                  void* stream) {
  if (!p || !cam || !v || !out)
    return noalloc_fail(PPS_EINVAL, "pps_filter_noalloc: params, camera, vertices and output "
                                    "must not be NULL");
  if (pps::check_params(p) != PPS_OK)
    return noalloc_fail(PPS_EINVAL, std::string("pps_filter_noalloc: ") + pps::last_error_text());
  if (p->log2_slots < 4 || p->log2_slots > kNoAllocMaxLog2Slots)
    return noalloc_fail(PPS_EINVAL, "pps_filter_noalloc: log2_slots must be in [4, 20]");
  if (n > kNoAllocMaxVertices)
    return noalloc_fail(PPS_EINVAL, "pps_filter_noalloc: at most 524288 vertices per call");
  if (p->accum_mode != PPS_ACCUM_FP32 || p->hist_mode != PPS_HIST_NONE ||
      p->fallback != PPS_FALLBACK_NONE || p->hist_evict != 0 || p->hist_migrate != 0 ||
      p->normal_search != 0)
    return noalloc_fail(PPS_EINVAL, "pps_filter_noalloc: FP32 accumulation without history, "
                                    "fallback or normal search only");
  if (v->dist || v->extra)
    return noalloc_fail(PPS_EINVAL, "pps_filter_noalloc: no dist or extra arrays");
  if (n && (!v->px || !v->py || !v->pz || !v->nx || !v->ny || !v->nz || !v->r || !v->g ||
            !v->b || !out->r || !out->g || !out->b))
    return noalloc_fail(PPS_EINVAL, "pps_filter_noalloc: vertex and output arrays are required");
  unsigned char* base = nullptr;
  if (int rc = scratch_address("pps_filter_noalloc", &base)) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t T = 1u << p->log2_slots;
  const size_t tile = static_cast<size_t>(pps::fused_tile_size());
  const size_t ids = (n + tile - 1) / tile * tile;

  pps::TableDev t{};
  t.slots = reinterpret_cast<unsigned long long*>(base);
  t.acc = reinterpret_cast<float4*>(base + kOffAcc);
  t.info = reinterpret_cast<uint4*>(base + kOffInfo);
  t.ctrl = reinterpret_cast<pps::Ctrl*>(base + kOffCtrl);
  t.mask = T - 1;
  t.hmask = 0;
  t.max_probes = p->max_probes;
  t.lowcount = p->lowcount_threshold;
  t.fixed = 0;
  t.hist_mode = 0;

  pps::KeyConst kc{};
  kc.cam[0] = cam->pos[0];
  kc.cam[1] = cam->pos[1];
  kc.cam[2] = cam->pos[2];
  kc.k = p->voxel_scale * p->pixel_angle;
  kc.seed = p->seed;
  kc.frame = frame;
  pps::set_round_keys(kc);
  kc.hseed_home = p->hash_seed_home;
  kc.hseed_fp = p->hash_seed_fp;
  kc.mask = T - 1;
  kc.max_probes = p->max_probes;
  kc.lod_min = p->lod_min;
  kc.lod_max = p->lod_max;
  kc.jitter = p->jitter;
  kc.nih = p->normal_in_home_hash;

  // The array keeps whatever the last call left: clear what must start empty.
  cudaError_t e = cudaMemsetAsync(t.slots, 0, static_cast<size_t>(T) * sizeof(unsigned long long), st);
  if (e == cudaSuccess && ids) e = cudaMemsetAsync(t.acc, 0, ids * sizeof(float4), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(t.ctrl, 0, kCtrlBytes, st);
  if (e != cudaSuccess)
    return noalloc_fail(PPS_ECUDA, std::string("pps_filter_noalloc: ") + cudaGetErrorString(e));
  if (n == 0) return PPS_OK;

  pps::VertexPtrs dv;
  dv.px = v->px;
  dv.py = v->py;
  dv.pz = v->pz;
  dv.nx = v->nx;
  dv.ny = v->ny;
  dv.nz = v->nz;
  dv.r = v->r;
  dv.g = v->g;
  dv.b = v->b;
  dv.id = v->id;
  dv.id_base = v->id_base;
  dv.stream_id = v->stream_id;
  dv.dist = v->dist;
  dv.extra = v->extra;
  pps::OutPtrs dout;
  dout.r = out->r;
  dout.g = out->g;
  dout.b = out->b;
  dout.count = out->count;
  dout.status = out->status;

  pps::FusedPlan plan;
  e = pps::plan_fused(n, false, 2, &plan);
  if (e == cudaSuccess)
    e = pps::launch_fused(kc, t, dv, n, dout, false, false, 0.0f, plan,
                          reinterpret_cast<uint32_t*>(base + kOffStash), nullptr, st);
  if (e != cudaSuccess)
    return noalloc_fail(PPS_ECUDA, std::string("pps_filter_noalloc: ") + cudaGetErrorString(e));
  return PPS_OK;
}

extern "C" int pps_noalloc_stats(pps_stats_t* out, void* stream) {
  if (!out) return noalloc_fail(PPS_EINVAL, "pps_noalloc_stats: out must not be NULL");
  unsigned char* base = nullptr;
  if (int rc = scratch_address("pps_noalloc_stats", &base)) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  pps::Ctrl c;
  cudaError_t e = cudaMemcpyAsync(&c, base + kOffCtrl, sizeof(c), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return noalloc_fail(PPS_ECUDA, std::string("pps_noalloc_stats: ") + cudaGetErrorString(e));
  std::memset(out, 0, sizeof(*out));
  out->frame_cells = c.frame_cells;
  out->overflow_vertices = c.overflow_vertices;
  out->vertices = c.vertices;
  out->device_error = c.error;
  if (c.error) {
    // clear the error word and the grid-barrier state for the next call
    e = cudaMemsetAsync(base + kOffCtrl + offsetof(pps::Ctrl, error), 0, 3 * sizeof(unsigned int),
                        st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
      return noalloc_fail(PPS_ECUDA, std::string("pps_noalloc_stats: ") + cudaGetErrorString(e));
    return noalloc_fail(PPS_EDEVICE, "pps_noalloc_stats: " + pps::device_error_text(c.error));
  }
  return PPS_OK;
}
