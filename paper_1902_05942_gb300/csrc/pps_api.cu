// C ABI of the hashed path space filter (see include/pps.h for the contract).
//
// Host-side responsibilities only: argument checks, the per-table frame state
// machine (clean -> open -> blended -> clean), device allocations owned by the
// table, and kernel launches.  Every step of the filter itself runs in the
// kernels of pps_kernels.cu.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <string>

#include "pps.h"
#include "pps_internal.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(const char* what, cudaError_t e) {
  return fail(PPS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define PPS_CUDA(call)                                \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(#call, e_); \
  } while (0)

enum FrameState { kClean = 0, kOpen = 1, kBlended = 2 };

}  // namespace

namespace pps {
// Record an error for pps_last_error() from another translation unit.
int record_error(int code, const char* msg) { return fail(code, msg); }

const char* last_error_text() { return g_err.c_str(); }

// What the bits of a device error word mean, for pps_last_error().
std::string device_error_text(unsigned int word) {
  char buf[64];
  std::snprintf(buf, sizeof(buf), "device error word 0x%x:", word);
  std::string s = buf;
  if (word & kErrBarrierTimeout) s += " a grid-barrier wait timed out;";
  if (word & kErrBadSlot) s += " a lookup got a cell id not of this frame;";
  if (word & kErrCountSaturated)
    s += " a cell reached 2^24 members, past which FP32 counts are not exact"
         " (use fixed-point accumulation);";
  return s;
}
}  // namespace pps

struct pps_table {
  pps_params p{};
  int device = 0;
  uint32_t T = 0;
  uint32_t Th = 0;
  pps::TableDev dev{};
  pps::KeyConst kc{};
  int state = kClean;
  uint32_t frame_tiles = 0;  // split path: tiles (cell-id blocks) used this frame
  pps_tuning tune{};         // launch shape (batch width 0 = library default)
  size_t D = 0;              // capacity of the dense cell arrays
  uint32_t* gstash = nullptr;
  size_t gstash_cap = 0;
  uint32_t* split_ids = nullptr;  // pps_filter on the split kernels: each vertex's cell id
  size_t split_ids_cap = 0;
  uint32_t* neigh_q = nullptr;  // neighborhood search: queue of low-count vertices
  size_t neigh_q_cap = 0;
  void* stage = nullptr;  // pps_filter_host device staging
  size_t stage_cap = 0;
  unsigned long long* scratch_u64 = nullptr;  // 1 word for occupancy counting
  // pps_filter_host_async: two staging slots; the uploads may spread over
  // kUpStreams streams (three measured no faster than one), one download stream
  static constexpr int kUpStreams = 1;
  struct HostSlot {
    void* dev = nullptr;
    size_t cap = 0;
    cudaEvent_t in_ready[kUpStreams] = {}, computed = nullptr, done = nullptr;
    bool used = false;
  };
  HostSlot hslot[2];
  cudaStream_t up[kUpStreams] = {}, down = nullptr;
  uint64_t host_calls = 0;
  uint32_t epoch = 0;           // evicting history: blends so far (priority of this frame)
  pps_table* coarse = nullptr;  // multi-level accumulation: the next coarser resolution
  void* fb = nullptr;           // multi-level scratch: coarse results and fine status
  size_t fb_cap = 0;            // vertices the scratch holds
};

namespace pps {

int check_params(const pps_params* p) {
  if (!p) return fail(PPS_EINVAL, "params is NULL");
  if (p->log2_slots < 4 || p->log2_slots > 30) return fail(PPS_EINVAL, "log2_slots must be in [4, 30]");
  const uint64_t T = 1ull << p->log2_slots;
  if (p->max_probes < 1 || p->max_probes > T || p->max_probes > 4096)
    return fail(PPS_EINVAL, "max_probes must be in [1, min(T, 4096)]");
  if (!(p->voxel_scale > 0.0f) || !std::isfinite(p->voxel_scale))
    return fail(PPS_EINVAL, "voxel_scale must be finite and > 0");
  if (!(p->pixel_angle > 0.0f) || !std::isfinite(p->pixel_angle))
    return fail(PPS_EINVAL, "pixel_angle must be finite and > 0");
  if (p->lod_min <= -126 || p->lod_max >= 127 || p->lod_min > p->lod_max)
    return fail(PPS_EINVAL, "need -126 < lod_min <= lod_max < 127");
  if (p->accum_mode > PPS_ACCUM_FIXED) return fail(PPS_EINVAL, "bad accum_mode");
  if (p->hist_mode > PPS_HIST_FP16) return fail(PPS_EINVAL, "bad hist_mode");
  if (p->jitter > 1 || p->normal_in_home_hash > 1) return fail(PPS_EINVAL, "flags must be 0 or 1");
  if (p->log2_hist_slots != 0 && (p->log2_hist_slots < 4 || p->log2_hist_slots > 30))
    return fail(PPS_EINVAL, "log2_hist_slots must be 0 or in [4, 30]");
  if (p->log2_hist_slots != 0 && p->max_probes > (1ull << p->log2_hist_slots))
    return fail(PPS_EINVAL, "max_probes exceeds the history table size");
  if (p->fallback > PPS_FALLBACK_NEIGHBORS) return fail(PPS_EINVAL, "bad fallback");
  if (p->hist_evict > 1) return fail(PPS_EINVAL, "hist_evict must be 0 or 1");
  if (p->hist_evict && p->hist_mode == PPS_HIST_NONE)
    return fail(PPS_EINVAL, "hist_evict needs a history (hist_mode != NONE)");
  if (p->hist_migrate > 1) return fail(PPS_EINVAL, "hist_migrate must be 0 or 1");
  if (p->hist_migrate && (p->hist_mode == PPS_HIST_NONE || p->hist_evict))
    return fail(PPS_EINVAL, "hist_migrate needs a history without eviction");
  if (p->fallback == PPS_FALLBACK_COARSE && !std::isfinite(2.0f * p->voxel_scale))
    return fail(PPS_EINVAL, "voxel_scale too large for a coarser level");
  if (p->normal_search > 256) return fail(PPS_EINVAL, "normal_search must be 0 .. 256");
  if (p->normal_search && (p->normal_in_home_hash || p->fallback != PPS_FALLBACK_NONE))
    return fail(PPS_EINVAL,
                "normal_search needs normal_in_home_hash = 0 and no low-count fallback");
  return PPS_OK;
}

}  // namespace pps

namespace {

using pps::check_params;

int check_table(pps_table* t) {
  if (!t) return fail(PPS_EINVAL, "table is NULL");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != t->device)
    return fail(PPS_EINVAL, "the table's device is not the current device");
  return PPS_OK;
}

int check_vertices(const pps_vertices* v, size_t n) {
  if (!v) return fail(PPS_EINVAL, "vertices is NULL");
  if (n == 0) return PPS_OK;
  if (!v->px || !v->py || !v->pz || !v->nx || !v->ny || !v->nz || !v->r || !v->g || !v->b)
    return fail(PPS_EINVAL, "all nine vertex arrays are required");
  if (n > (1ull << 40)) return fail(PPS_EINVAL, "n too large");
  return PPS_OK;
}

int check_output(const pps_output* o, size_t n) {
  if (!o) return fail(PPS_EINVAL, "output is NULL");
  if (n && (!o->r || !o->g || !o->b)) return fail(PPS_EINVAL, "output r, g, b are required");
  return PPS_OK;
}

pps::VertexPtrs to_dev(const pps_vertices* v) {
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

pps::OutPtrs to_dev(const pps_output* o) {
  pps::OutPtrs d;
  d.r = o->r;
  d.g = o->g;
  d.b = o->b;
  d.count = o->count;
  d.status = o->status;
  return d;
}

bool temporal(const pps_table* t) { return t->p.hist_mode != PPS_HIST_NONE; }

int batch_of(const pps_table* t) { return t->tune.batch == 4 ? 4 : 2; }

// The library default: the pipelined insert while the slot index fits in L2
// with the accumulators (T <= 2^23 slots, 64 MB); beyond that the table's
// operations go to DRAM and the per-thread insert, whose every thread probes,
// was measured faster (stress workload, T = 2^26: 9.6 vs 10.5 ms per frame).
pps::InsertShape insert_shape(const pps_table* t) {
  pps::InsertShape s;
  const bool big = t->T > (1u << 23);
  s.pipelined = t->tune.insert == 2 || (t->tune.insert == 0 && !big) ? 1 : 0;
  s.key_warps = t->tune.key_warps ? static_cast<int>(t->tune.key_warps) : 8;
  s.merge = t->tune.merge ? static_cast<int>(t->tune.merge) : 2;
  return s;
}

// Empty the cells of the split path's frame (the fused path leaves none behind)
// and reset the frame counters.
int reset_frame(pps_table* t, cudaStream_t st) {
  if (t->state != kClean) {
    PPS_CUDA(pps::launch_clear(t->dev, t->frame_tiles, st));
    t->frame_tiles = 0;
    t->state = kClean;
  }
  PPS_CUDA(cudaMemsetAsync(t->dev.ctrl, 0, pps::kCtrlFrameBytes, st));
  return PPS_OK;
}

// Make the dense cell arrays hold at least `need` cells, keeping the first
// `keep` cells (accumulators, cell info, tile counts and quantized keys).  New accumulators
// start at zero.
int ensure_dense(pps_table* t, size_t need, size_t keep, cudaStream_t st) {
  if (need <= t->D) return PPS_OK;
  if (need > 0xFFFFFFF0ull) return fail(PPS_EINVAL, "more than 2^32 - 16 cells in one frame");
  size_t cap = t->D ? t->D : 1;
  while (cap < need) cap *= 2;
  if (cap > 0xFFFFFFF0ull) cap = 0xFFFFFFF0ull;
  const size_t acc_b = t->dev.fixed ? 32 : 16;
  const size_t nb = cap / 4 + 16;  // tile counts: one per block of >= 4 cells
  void *acc = nullptr, *info = nullptr, *bc = nullptr, *kw = nullptr, *hold = nullptr;
  cudaError_t e = cudaMalloc(&acc, cap * acc_b);
  if (e == cudaSuccess) e = cudaMalloc(&info, cap * sizeof(uint4));
  if (e == cudaSuccess) e = cudaMalloc(&bc, nb * sizeof(uint32_t));
  if (e == cudaSuccess && (t->dev.hist_migrate || t->dev.normal_search))
    e = cudaMalloc(&kw, cap * sizeof(uint4));
  if (e == cudaSuccess && t->dev.hist_migrate) e = cudaMalloc(&hold, cap * sizeof(float4));
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, cap * acc_b, st);
  void* old_acc = t->dev.fixed ? static_cast<void*>(t->dev.acc64) : static_cast<void*>(t->dev.acc);
  if (e == cudaSuccess && keep) {
    e = cudaMemcpyAsync(acc, old_acc, keep * acc_b, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(info, t->dev.info, keep * sizeof(uint4), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bc, t->dev.bcount, (t->D / 4 + 16) * sizeof(uint32_t),
                          cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && kw)
      e = cudaMemcpyAsync(kw, t->dev.kw, keep * sizeof(uint4), cudaMemcpyDeviceToDevice, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(acc);
    cudaFree(info);
    cudaFree(bc);
    cudaFree(kw);
    cudaFree(hold);
    cudaGetLastError();
    return fail(PPS_ENOMEM, std::string("dense cell arrays: ") + cudaGetErrorString(e));
  }
  cudaFree(old_acc);
  cudaFree(t->dev.info);
  cudaFree(t->dev.bcount);
  cudaFree(t->dev.kw);
  cudaFree(t->dev.hold);
  t->dev.kw = static_cast<uint4*>(kw);
  t->dev.hold = static_cast<float4*>(hold);
  if (t->dev.fixed)
    t->dev.acc64 = static_cast<unsigned long long*>(acc);
  else
    t->dev.acc = static_cast<float4*>(acc);
  t->dev.info = static_cast<uint4*>(info);
  t->dev.bcount = static_cast<uint32_t*>(bc);
  t->D = cap;
  return PPS_OK;
}

void set_camera(pps_table* t, const pps_camera* cam, uint32_t frame) {
  t->kc.cam[0] = cam->pos[0];
  t->kc.cam[1] = cam->pos[1];
  t->kc.cam[2] = cam->pos[2];
  t->kc.frame = frame;
  pps::set_round_keys(t->kc);
}

void free_all(pps_table* t) {
  cudaFree(t->dev.slots);
  cudaFree(t->dev.acc);
  cudaFree(t->dev.acc64);
  cudaFree(t->dev.info);
  cudaFree(t->dev.bcount);
  cudaFree(t->dev.kw);
  cudaFree(t->dev.hold);
  cudaFree(t->dev.hcells);
  cudaFree(t->dev.ctrl);
  cudaFree(t->gstash);
  cudaFree(t->split_ids);
  cudaFree(t->neigh_q);
  cudaFree(t->stage);
  cudaFree(t->scratch_u64);
  cudaFree(t->fb);
  for (auto& h : t->hslot) {
    cudaFree(h.dev);
    for (cudaEvent_t e : h.in_ready)
      if (e) cudaEventDestroy(e);
    if (h.computed) cudaEventDestroy(h.computed);
    if (h.done) cudaEventDestroy(h.done);
  }
  for (cudaStream_t s : t->up)
    if (s) cudaStreamDestroy(s);
  if (t->down) cudaStreamDestroy(t->down);
}

// Evicting history: the priority of the coming blend.  Priorities are 8-bit
// epochs 1..255; when they run out, every entry drops by 128 (the order of
// the last 127 epochs survives) and counting resumes at 128.
int next_epoch(pps_table* t, cudaStream_t st) {
  if (!t->dev.hist_evict) return PPS_OK;
  if (t->epoch >= 255) {
    PPS_CUDA(pps::launch_hist_age(t->dev, 128u, st));
    t->epoch -= 128;
  }
  t->dev.hist_rank = ++t->epoch;
  return PPS_OK;
}

// Multi-level scratch for n vertices: the coarse pass's r, g, b, count and
// status, and a fine status array for callers that pass none.
int fallback_scratch(pps_table* t, size_t n, pps::OutPtrs* coarse, uint8_t** fine_status) {
  const size_t nn = (n + 15) & ~static_cast<size_t>(15);
  if (t->fb_cap < nn) {
    cudaFree(t->fb);
    t->fb = nullptr;
    t->fb_cap = 0;
    cudaError_t e = cudaMalloc(&t->fb, nn * (4 * sizeof(float) + 2));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PPS_ENOMEM, "fallback scratch allocation failed");
    }
    t->fb_cap = nn;
  }
  float* base = static_cast<float*>(t->fb);
  coarse->r = base;
  coarse->g = base + t->fb_cap;
  coarse->b = base + 2 * t->fb_cap;
  coarse->count = reinterpret_cast<uint32_t*>(base + 3 * t->fb_cap);
  coarse->status = reinterpret_cast<uint8_t*>(base + 4 * t->fb_cap);
  *fine_status = coarse->status + t->fb_cap;
  return PPS_OK;
}

}  // namespace

extern "C" {

const char* pps_version(void) { return "pps-gb300 0.1 (sm_103a)"; }

int pps_last_error(char* buf, size_t len) {
  if (buf && len) {
    std::strncpy(buf, g_err.c_str(), len - 1);
    buf[len - 1] = '\0';
  }
  return PPS_OK;
}

int pps_create(pps_table** out, const pps_params* p) {
  if (!out) return fail(PPS_EINVAL, "out is NULL");
  *out = nullptr;
  if (int rc = check_params(p)) return rc;
  pps_table* t = new (std::nothrow) pps_table();
  if (!t) return fail(PPS_ENOMEM, "host allocation failed");
  t->p = *p;
  t->T = 1u << p->log2_slots;
  t->Th = 1u << (p->log2_hist_slots ? p->log2_hist_slots : p->log2_slots);
  cudaGetDevice(&t->device);
  const size_t T = t->T;
  const size_t Th = t->Th;
  auto alloc = [&](void** ptr, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) e = cudaMemset(*ptr, 0, bytes);
    return e;
  };
  const bool fixed = p->accum_mode == PPS_ACCUM_FIXED;
  t->dev.fixed = fixed;
  t->dev.hist_migrate = p->hist_migrate ? 1 : 0;  // before the dense arrays are made
  t->dev.normal_search = p->normal_search;
  t->dev.hstride = p->hist_mode == PPS_HIST_FP16 ? 16u : 32u;
  t->dev.hfp_off = p->hist_mode == PPS_HIST_FP16 ? 8u : 16u;
  cudaError_t e = alloc(reinterpret_cast<void**>(&t->dev.slots), T * sizeof(unsigned long long));
  if (e == cudaSuccess && p->hist_mode != PPS_HIST_NONE)
    e = alloc(reinterpret_cast<void**>(&t->dev.hcells), Th * t->dev.hstride);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void**>(&t->dev.ctrl), sizeof(pps::Ctrl));
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void**>(&t->scratch_u64), 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess && ensure_dense(t, std::min<size_t>(T, 1u << 22), 0, nullptr) != PPS_OK)
    e = cudaErrorMemoryAllocation;
  if (e != cudaSuccess) {
    free_all(t);
    delete t;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? PPS_ENOMEM : PPS_ECUDA,
                std::string("pps_create: ") + cudaGetErrorString(e));
  }
  t->dev.mask = t->T - 1;
  t->dev.hmask = t->Th - 1;
  t->dev.max_probes = p->max_probes;
  t->dev.lowcount = p->lowcount_threshold;
  t->dev.hist_mode = static_cast<int>(p->hist_mode);
  t->kc.k = p->voxel_scale * p->pixel_angle;  // fl32(s * theta_px)
  t->kc.seed = p->seed;
  pps::set_round_keys(t->kc);
  t->kc.hseed_home = p->hash_seed_home;
  t->kc.hseed_fp = p->hash_seed_fp;
  t->kc.mask = t->T - 1;
  t->kc.max_probes = p->max_probes;
  t->kc.lod_min = p->lod_min;
  t->kc.lod_max = p->lod_max;
  t->kc.jitter = p->jitter;
  t->kc.nih = p->normal_in_home_hash;
  t->dev.neighbors = p->fallback == PPS_FALLBACK_NEIGHBORS ? 1 : 0;
  t->dev.hist_evict = p->hist_evict ? 1 : 0;
  if (p->fallback == PPS_FALLBACK_COARSE) {
    // the next coarser resolution: s doubled, so every level grows by one
    pps_params pc = *p;
    pc.voxel_scale = 2.0f * p->voxel_scale;
    pc.fallback = PPS_FALLBACK_NONE;
    if (int rc = pps_create(&t->coarse, &pc)) {
      free_all(t);
      delete t;
      return rc;
    }
  }
  *out = t;
  return PPS_OK;
}

int pps_destroy(pps_table* t) {
  if (!t) return PPS_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(t->device);
  cudaDeviceSynchronize();
  pps_destroy(t->coarse);
  free_all(t);
  delete t;
  if (prev >= 0) cudaSetDevice(prev);
  return PPS_OK;
}

int pps_build(pps_table* t, const pps_camera* cam, uint32_t frame, void* stream) {
  if (int rc = check_table(t)) return rc;
  if (!cam) return fail(PPS_EINVAL, "camera is NULL");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (int rc = reset_frame(t, st)) return rc;
  set_camera(t, cam, frame);
  t->state = kOpen;
  if (t->coarse) return pps_build(t->coarse, cam, frame, stream);
  return PPS_OK;
}

int pps_insert(pps_table* t, const pps_vertices* v, size_t n, uint32_t* slot_out, void* stream) {
  if (int rc = check_table(t)) return rc;
  if (int rc = check_vertices(v, n)) return rc;
  if (t->state != kOpen) return fail(PPS_ESTATE, "pps_insert needs pps_build first (and no pps_blend since)");
  if ((t->dev.hist_migrate || t->dev.normal_search) && v->extra)
    return fail(PPS_EINVAL, "a table with hist_migrate or normal_search takes no extra key word");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t tile = static_cast<size_t>(pps::tile_size());
  const size_t tiles = (n + tile - 1) / tile;
  if (int rc = ensure_dense(t, (t->frame_tiles + tiles) * tile, t->frame_tiles * tile, st)) return rc;
  PPS_CUDA(pps::launch_insert(t->kc, t->dev, to_dev(v), n, slot_out, t->frame_tiles,
                              batch_of(t), st));
  t->frame_tiles += static_cast<uint32_t>(tiles);
  if (t->coarse) return pps_insert(t->coarse, v, n, nullptr, stream);
  return PPS_OK;
}

int pps_blend(pps_table* t, float alpha, void* stream) {
  if (int rc = check_table(t)) return rc;
  if (!temporal(t)) return fail(PPS_EINVAL, "pps_blend needs a table with hist_mode != NONE");
  if (!std::isfinite(alpha) || alpha > 1.0f) return fail(PPS_EINVAL, "alpha must be finite and <= 1");
  if (t->state != kOpen) return fail(PPS_ESTATE, "pps_blend needs an open frame (pps_build, pps_insert)");
  if (int rc = next_epoch(t, static_cast<cudaStream_t>(stream))) return rc;
  PPS_CUDA(pps::launch_blend(t->kc, t->dev, t->frame_tiles, alpha,
                             static_cast<cudaStream_t>(stream)));
  t->state = kBlended;
  if (t->coarse) return pps_blend(t->coarse, alpha, stream);
  return PPS_OK;
}

int pps_query(pps_table* t, const pps_vertices* v, size_t n, const uint32_t* slot_in,
              const pps_output* out, void* stream) {
  if (int rc = check_table(t)) return rc;
  if (int rc = check_vertices(v, n)) return rc;
  if (int rc = check_output(out, n)) return rc;
  if (t->state == kClean) return fail(PPS_ESTATE, "pps_query needs an open frame");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t id_limit = t->frame_tiles * static_cast<uint32_t>(pps::tile_size());
  if (!t->coarse) {
    PPS_CUDA(pps::launch_query(t->kc, t->dev, to_dev(v), n, slot_in, to_dev(out),
                               t->state == kBlended, id_limit, st));
    return PPS_OK;
  }
  // multi-level: the fine lookup, the coarse lookup (re-probed), the choice
  pps::OutPtrs c{}, o = to_dev(out);
  uint8_t* fstat = nullptr;
  if (int rc = fallback_scratch(t, n, &c, &fstat)) return rc;
  pps::OutPtrs f = o;
  if (!f.status) f.status = fstat;
  PPS_CUDA(pps::launch_query(t->kc, t->dev, to_dev(v), n, slot_in, f, t->state == kBlended,
                             id_limit, st));
  const pps_table* k = t->coarse;
  PPS_CUDA(pps::launch_query(k->kc, k->dev, to_dev(v), n, nullptr, c, k->state == kBlended,
                             k->frame_tiles * static_cast<uint32_t>(pps::tile_size()), st));
  PPS_CUDA(pps::launch_combine_coarse(n, f.status, c, o, st));
  return PPS_OK;
}

}  // extern "C"

namespace {

// One resolution of pps_filter: the persistent launch over all n vertices.
int filter_one(pps_table* t, const pps_camera* cam, uint32_t frame, const pps_vertices* v,
               size_t n, int blend, float alpha, const pps::OutPtrs& out, cudaStream_t st) {
  if (int rc = reset_frame(t, st)) return rc;
  set_camera(t, cam, frame);
  if (n == 0) return PPS_OK;
  pps::FusedPlan plan;
  PPS_CUDA(pps::plan_fused(n, temporal(t), batch_of(t), &plan, t->dev.hist_evict != 0,
                           t->dev.neighbors != 0, insert_shape(t), t->dev.fixed != 0));
  // cell ids and (off-chip) stash words cover whole tiles: [0, ntiles * tile)
  const size_t ftile = static_cast<size_t>(pps::fused_tile_size());
  const size_t stash_need = (n + ftile - 1) / ftile * ftile;
  if (int rc = ensure_dense(t, stash_need, 0, st)) return rc;
  if (plan.global_stash && t->gstash_cap < stash_need) {
    cudaFree(t->gstash);
    t->gstash = nullptr;
    t->gstash_cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&t->gstash), stash_need * sizeof(uint32_t));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PPS_ENOMEM, "pps_filter: scratch stash allocation failed");
    }
    t->gstash_cap = stash_need;
  }
  if (t->dev.neighbors && t->neigh_q_cap < n) {
    cudaFree(t->neigh_q);
    t->neigh_q = nullptr;
    t->neigh_q_cap = 0;
    if (cudaMalloc(reinterpret_cast<void**>(&t->neigh_q), n * sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      return fail(PPS_ENOMEM, "pps_filter: neighborhood queue allocation failed");
    }
    t->neigh_q_cap = n;
  }
  if (blend)
    if (int rc = next_epoch(t, st)) return rc;
  PPS_CUDA(pps::launch_fused(t->kc, t->dev, to_dev(v), n, out, temporal(t), blend != 0, alpha,
                             plan, t->gstash, t->neigh_q, st));
  t->state = kClean;
  return PPS_OK;
}

}  // namespace

extern "C" {

int pps_filter(pps_table* t, const pps_camera* cam, uint32_t frame, const pps_vertices* v,
               size_t n, int blend, float alpha, const pps_output* out, void* stream) {
  if (int rc = check_table(t)) return rc;
  if (!cam) return fail(PPS_EINVAL, "camera is NULL");
  if (int rc = check_vertices(v, n)) return rc;
  if (int rc = check_output(out, n)) return rc;
  if (blend && !temporal(t)) return fail(PPS_EINVAL, "blend needs a table with hist_mode != NONE");
  if (blend && (!std::isfinite(alpha) || alpha > 1.0f))
    return fail(PPS_EINVAL, "alpha must be finite and <= 1");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (v->dist || v->extra || t->dev.hist_migrate || t->dev.normal_search) {
    // key variants and history migration: the split kernels (the persistent
    // ones are built without them); the insert's cell ids spare the lookup
    // its keys and probes
    if (t->split_ids_cap < n) {
      cudaFree(t->split_ids);
      t->split_ids = nullptr;
      t->split_ids_cap = 0;
      if (cudaMalloc(reinterpret_cast<void**>(&t->split_ids), n * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return fail(PPS_ENOMEM, "pps_filter: cell-id scratch allocation failed");
      }
      t->split_ids_cap = n;
    }
    if (int rc = pps_build(t, cam, frame, stream)) return rc;
    if (int rc = pps_insert(t, v, n, t->split_ids, stream)) return rc;
    if (blend)
      if (int rc = pps_blend(t, alpha, stream)) return rc;
    return pps_query(t, v, n, t->split_ids, out, stream);
  }
  if (!t->coarse) return filter_one(t, cam, frame, v, n, blend, alpha, to_dev(out), st);
  // multi-level: both resolutions, then the choice per vertex
  pps::OutPtrs c{}, o = to_dev(out);
  uint8_t* fstat = nullptr;
  if (n && fallback_scratch(t, n, &c, &fstat)) return PPS_ENOMEM;
  pps::OutPtrs f = o;
  if (!f.status) f.status = fstat;
  if (int rc = filter_one(t, cam, frame, v, n, blend, alpha, f, st)) return rc;
  if (int rc = filter_one(t->coarse, cam, frame, v, n, blend, alpha, c, st)) return rc;
  if (n) PPS_CUDA(pps::launch_combine_coarse(n, f.status, c, o, st));
  return PPS_OK;
}



}  // extern "C"

namespace {

// Device staging of one host call: the nine inputs, r, g, b, count, status.
size_t host_stage_bytes(size_t n) {
  const size_t nn = (n + 3) & ~static_cast<size_t>(3);
  return nn * (9 + 3 + 1) * sizeof(float) + nn;
}

// Upload the host inputs to `stage`, array i on stream st[i % nst]; fill the
// device views.
int host_upload(const pps_vertices* vh, size_t n, const pps_output* oh, void* stage,
                const cudaStream_t* st, int nst, pps_vertices* vd, pps_output* od) {
  const size_t nn = (n + 3) & ~static_cast<size_t>(3);
  float* base = static_cast<float*>(stage);
  const float* src[9] = {vh->px, vh->py, vh->pz, vh->nx, vh->ny, vh->nz, vh->r, vh->g, vh->b};
  float* dst[9];
  for (int i = 0; i < 9; ++i) {
    dst[i] = base + static_cast<size_t>(i) * nn;
    PPS_CUDA(cudaMemcpyAsync(dst[i], src[i], n * sizeof(float), cudaMemcpyHostToDevice,
                             st[i % nst]));
  }
  *vd = pps_vertices{};
  vd->px = dst[0];
  vd->py = dst[1];
  vd->pz = dst[2];
  vd->nx = dst[3];
  vd->ny = dst[4];
  vd->nz = dst[5];
  vd->r = dst[6];
  vd->g = dst[7];
  vd->b = dst[8];
  vd->id_base = vh->id_base;
  vd->stream_id = vh->stream_id;
  *od = pps_output{};
  od->r = base + 9 * nn;
  od->g = base + 10 * nn;
  od->b = base + 11 * nn;
  od->count = oh->count ? reinterpret_cast<uint32_t*>(base + 12 * nn) : nullptr;
  od->status = oh->status ? reinterpret_cast<uint8_t*>(base + 13 * nn) : nullptr;
  return PPS_OK;
}

int host_download(const pps_output* od, size_t n, const pps_output* oh, cudaStream_t st) {
  PPS_CUDA(cudaMemcpyAsync(oh->r, od->r, n * sizeof(float), cudaMemcpyDeviceToHost, st));
  PPS_CUDA(cudaMemcpyAsync(oh->g, od->g, n * sizeof(float), cudaMemcpyDeviceToHost, st));
  PPS_CUDA(cudaMemcpyAsync(oh->b, od->b, n * sizeof(float), cudaMemcpyDeviceToHost, st));
  if (oh->count)
    PPS_CUDA(cudaMemcpyAsync(oh->count, od->count, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  if (oh->status) PPS_CUDA(cudaMemcpyAsync(oh->status, od->status, n, cudaMemcpyDeviceToHost, st));
  return PPS_OK;
}

int check_host_call(pps_table* t, const pps_vertices* vh, size_t n, const pps_output* oh) {
  if (int rc = check_table(t)) return rc;
  if (int rc = check_vertices(vh, n)) return rc;
  if (int rc = check_output(oh, n)) return rc;
  if (vh->id || vh->dist || vh->extra)
    return fail(PPS_EINVAL, "host-buffer filtering takes no id, dist or extra array");
  return PPS_OK;
}

}  // namespace

extern "C" {

int pps_filter_host(pps_table* t, const pps_camera* cam, uint32_t frame, const pps_vertices* vh,
                    size_t n, int blend, float alpha, const pps_output* oh, void* stream) {
  if (int rc = check_host_call(t, vh, n, oh)) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t need = host_stage_bytes(n);
  if (t->stage_cap < need) {
    cudaFree(t->stage);
    t->stage = nullptr;
    t->stage_cap = 0;
    cudaError_t e = cudaMalloc(&t->stage, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PPS_ENOMEM, "pps_filter_host: staging allocation failed");
    }
    t->stage_cap = need;
  }
  pps_vertices vd;
  pps_output od;
  if (int rc = host_upload(vh, n, oh, t->stage, &st, 1, &vd, &od)) return rc;
  if (int rc = pps_filter(t, cam, frame, &vd, n, blend, alpha, &od, stream)) return rc;
  if (int rc = host_download(&od, n, oh, st)) return rc;
  PPS_CUDA(cudaStreamSynchronize(st));
  return PPS_OK;
}

int pps_filter_host_async(pps_table* t, const pps_camera* cam, uint32_t frame,
                          const pps_vertices* vh, size_t n, int blend, float alpha,
                          const pps_output* oh, void* stream) {
  if (int rc = check_host_call(t, vh, n, oh)) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  constexpr int K = pps_table::kUpStreams;
  if (!t->down) {
    for (cudaStream_t& s : t->up) PPS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    PPS_CUDA(cudaStreamCreateWithFlags(&t->down, cudaStreamNonBlocking));
    for (auto& h : t->hslot) {
      for (cudaEvent_t& e : h.in_ready)
        PPS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      PPS_CUDA(cudaEventCreateWithFlags(&h.computed, cudaEventDisableTiming));
      PPS_CUDA(cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming));
    }
  }
  pps_table::HostSlot& h = t->hslot[t->host_calls & 1];
  const size_t need = host_stage_bytes(n);
  if (h.cap < need) {
    if (h.used) PPS_CUDA(cudaEventSynchronize(h.done));
    cudaFree(h.dev);
    h.dev = nullptr;
    h.cap = 0;
    cudaError_t e = cudaMalloc(&h.dev, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PPS_ENOMEM, "pps_filter_host_async: staging allocation failed");
    }
    h.cap = need;
  }
  // uploads once this slot's previous results are home
  if (h.used)
    for (cudaStream_t s : t->up) PPS_CUDA(cudaStreamWaitEvent(s, h.done, 0));
  pps_vertices vd;
  pps_output od;
  if (int rc = host_upload(vh, n, oh, h.dev, t->up, K, &vd, &od)) return rc;
  // the filter on the caller's stream once the inputs are there
  for (int k = 0; k < K; ++k) {
    PPS_CUDA(cudaEventRecord(h.in_ready[k], t->up[k]));
    PPS_CUDA(cudaStreamWaitEvent(st, h.in_ready[k], 0));
  }
  if (int rc = pps_filter(t, cam, frame, &vd, n, blend, alpha, &od, stream)) return rc;
  PPS_CUDA(cudaEventRecord(h.computed, st));
  // downloads once the filter is done
  PPS_CUDA(cudaStreamWaitEvent(t->down, h.computed, 0));
  if (int rc = host_download(&od, n, oh, t->down)) return rc;
  PPS_CUDA(cudaEventRecord(h.done, t->down));
  h.used = true;
  ++t->host_calls;
  return PPS_OK;
}

int pps_host_wait(pps_table* t) {
  if (int rc = check_table(t)) return rc;
  for (auto& h : t->hslot)
    if (h.used) PPS_CUDA(cudaEventSynchronize(h.done));
  return PPS_OK;
}

}  // extern "C"

namespace pps {
// For batched launches: the device description of a table about to filter n
// vertices in one persistent launch (cell-id capacity ensured), its batch
// width, and whether it keeps a history.  The table must be between frames.
int table_for_batch(pps_table* t, size_t n, ViewDesc* vd, int* batch, int* block,
                    bool* temporal_out, cudaStream_t st) {
  if (int rc = check_table(t)) return rc;
  if (t->state != kClean) return fail(PPS_ESTATE, "a table of a batch is in the middle of a frame");
  if (t->p.fallback != PPS_FALLBACK_NONE || t->p.hist_evict || t->p.hist_migrate ||
      t->p.normal_search)
    return fail(PPS_EINVAL, "batched views take tables without a low-count fallback, eviction, "
                            "migration or normal search");
  const size_t ftile = static_cast<size_t>(fused_tile_size());
  if (int rc = ensure_dense(t, (n + ftile - 1) / ftile * ftile, 0, st)) return rc;
  vd->kc = t->kc;
  vd->t = t->dev;
  *batch = batch_of(t);
  *block = t->tune.block == 256 ? 256 : 512;
  *temporal_out = temporal(t);
  return PPS_OK;
}
}  // namespace pps

extern "C" {

int pps_set_tuning(pps_table* t, const pps_tuning* tune) {
  if (int rc = check_table(t)) return rc;
  if (!tune) return fail(PPS_EINVAL, "tuning is NULL");
  if (tune->batch != 0 && tune->batch != 2 && tune->batch != 4)
    return fail(PPS_EINVAL, "batch must be 0, 2 or 4");
  if (tune->insert > 2) return fail(PPS_EINVAL, "insert must be 0, 1 or 2");
  if (tune->block != 0 && tune->block != 256 && tune->block != 512)
    return fail(PPS_EINVAL, "block must be 0, 256 or 512");
  if (tune->key_warps != 0 && tune->key_warps != 4 && tune->key_warps != 8 && tune->key_warps != 12)
    return fail(PPS_EINVAL, "key_warps must be 0, 4, 8 or 12");
  if (tune->merge > 3) return fail(PPS_EINVAL, "merge must be 0, 1, 2 or 3");
  for (uint32_t r : tune->reserved)
    if (r) return fail(PPS_EINVAL, "reserved fields must be zero");
  t->tune = *tune;
  if (t->coarse) t->coarse->tune = *tune;
  return PPS_OK;
}

int pps_get_tuning(pps_table* t, pps_tuning* tune) {
  if (int rc = check_table(t)) return rc;
  if (!tune) return fail(PPS_EINVAL, "tuning is NULL");
  *tune = t->tune;
  tune->batch = static_cast<uint32_t>(batch_of(t));
  tune->insert = insert_shape(t).pipelined ? 2u : 1u;
  tune->key_warps = t->tune.key_warps ? t->tune.key_warps : 8u;
  tune->block = t->tune.block ? t->tune.block : 512u;
  tune->merge = static_cast<uint32_t>(insert_shape(t).merge);
  return PPS_OK;
}

int pps_keys(pps_table* t, const pps_vertices* v, size_t n, uint32_t* h_out, uint32_t* f_out,
             void* stream) {
  if (int rc = check_table(t)) return rc;
  if (int rc = check_vertices(v, n)) return rc;
  if (n && (!h_out || !f_out)) return fail(PPS_EINVAL, "h_out and f_out are required");
  PPS_CUDA(pps::launch_keys(t->kc, to_dev(v), n, h_out, f_out, static_cast<cudaStream_t>(stream)));
  return PPS_OK;
}

int pps_stats(pps_table* t, pps_stats_t* out, void* stream) {
  if (int rc = check_table(t)) return rc;
  if (!out) return fail(PPS_EINVAL, "out is NULL");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  PPS_CUDA(cudaMemsetAsync(t->scratch_u64, 0, 2 * sizeof(unsigned long long), st));
  PPS_CUDA(pps::launch_count_nonzero(t->dev.slots, 8, 0, 8, t->T, t->scratch_u64, st));
  if (t->dev.hcells)
    PPS_CUDA(pps::launch_count_nonzero(t->dev.hcells, t->dev.hstride, t->dev.hfp_off, 4, t->Th,
                                       t->scratch_u64 + 1, st));
  pps::Ctrl c;
  unsigned long long occ[2] = {0, 0};
  PPS_CUDA(cudaMemcpyAsync(&c, t->dev.ctrl, sizeof(c), cudaMemcpyDeviceToHost, st));
  PPS_CUDA(cudaMemcpyAsync(occ, t->scratch_u64, sizeof(occ), cudaMemcpyDeviceToHost, st));
  PPS_CUDA(cudaStreamSynchronize(st));
  std::memset(out, 0, sizeof(*out));
  out->frame_cells = c.frame_cells;
  out->overflow_vertices = c.overflow_vertices;
  out->vertices = c.vertices;
  out->occupied_slots = occ[0];
  out->hist_occupied = occ[1];
  out->hist_overflow = c.hist_overflow;
  out->device_error = c.error;
  out->frame = t->kc.frame;
  if (c.error) {
    // clear the error word and the barrier state so the table stays usable
    PPS_CUDA(cudaMemsetAsync(&t->dev.ctrl->error, 0, 3 * sizeof(unsigned int), st));  // + barrier
    PPS_CUDA(cudaStreamSynchronize(st));
    return fail(PPS_EDEVICE, pps::device_error_text(c.error));
  }
  return PPS_OK;
}

int pps_table_dump(pps_table* t, uint32_t* fp_host, void* acc_host, void* stream) {
  if (int rc = check_table(t)) return rc;
  if (!fp_host) return fail(PPS_EINVAL, "fp_host is NULL");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t acc_b = t->dev.fixed ? 32 : 16;
  unsigned long long* slots =
      static_cast<unsigned long long*>(std::malloc(t->T * sizeof(unsigned long long)));
  unsigned char* acc = static_cast<unsigned char*>(std::malloc(t->D * acc_b));
  if (!slots || !acc) {
    std::free(slots);
    std::free(acc);
    return fail(PPS_ENOMEM, "pps_table_dump: host buffer");
  }
  const void* dacc = t->dev.fixed ? static_cast<const void*>(t->dev.acc64)
                                  : static_cast<const void*>(t->dev.acc);
  cudaError_t e = cudaMemcpyAsync(slots, t->dev.slots, t->T * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(acc, dacc, t->D * acc_b, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    std::free(slots);
    std::free(acc);
    return cuda_fail("pps_table_dump", e);
  }
  // per slot: the fingerprint, and the accumulator of the slot's cell
  for (size_t i = 0; i < t->T; ++i) {
    const unsigned long long w = slots[i];
    fp_host[i] = static_cast<uint32_t>(w);
    if (!acc_host) continue;
    unsigned char* dst = static_cast<unsigned char*>(acc_host) + i * acc_b;
    const size_t id = static_cast<size_t>(w >> 32);  // cell id + 1, 0 = empty
    if (id == 0 || id - 1 >= t->D)
      std::memset(dst, 0, acc_b);
    else
      std::memcpy(dst, acc + (id - 1) * acc_b, acc_b);
  }
  std::free(slots);
  std::free(acc);
  return PPS_OK;
}

}  // extern "C"
