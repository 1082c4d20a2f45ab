// Kernels of the hashed path space filter (sm_103a) and their launchers.
//
//  k_insert        key construction (Alg. 1) + probing insert + atomic
//                  accumulation (Sec. 3.2, 3.3.1); appends touched cells to the
//                  frame's dirty list.
//  k_blend         temporal blend over the dirty list (Sec. 3.4.1).
//  k_query         one lookup per vertex: cell average or blended value.
//  k_clear_dirty   empties the cells of the dirty list for the next frame.
//  k_fused         the whole frame in one persistent cooperative launch: the
//                  four steps above separated by grid barriers; each vertex's
//                  cell index stays in shared memory between the phases.
//
// Vertex streams are read four consecutive vertices per thread with 128-bit
// streaming loads (ld.global.cs) when the arrays are 16-byte aligned; table
// words are read at L2 (ld.global.cg) because they are written by atomics and
// by other CTAs.
#include <algorithm>

#include "pps_internal.h"

namespace pps {

namespace {

constexpr int kBlock = 256;        // split kernels
constexpr int kFusedBlock = 512;   // persistent kernel

__device__ __forceinline__ float4 load4(const float* p, size_t j, size_t end, bool vec) {
  if (vec && j + 4 <= end) return __ldcs(reinterpret_cast<const float4*>(p + j));
  float4 v;
  v.x = j < end ? __ldcs(p + j) : 0.f;
  v.y = j + 1 < end ? __ldcs(p + j + 1) : 0.f;
  v.z = j + 2 < end ? __ldcs(p + j + 2) : 0.f;
  v.w = j + 3 < end ? __ldcs(p + j + 3) : 0.f;
  return v;
}

__device__ __forceinline__ float comp(const float4& v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

__device__ __forceinline__ uint32_t vertex_id(const VertexPtrs& v, size_t j) {
  return v.id ? __ldcs(v.id + j) : v.id_base + static_cast<uint32_t>(j);
}

template <typename T>
__device__ __forceinline__ T block_sum(T x) {
  __shared__ T s_part[32];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) s_part[w] = x;
  __syncthreads();
  T tot = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (blockDim.x + 31) / 32; ++i) tot += s_part[i];
  return tot;  // valid in thread 0
}

// Insert the four vertices j..j+3 (those below `end`).  Returns their cell
// indices (kOverflowSlot on probe overflow) and which of them own their cell
// this frame (published its fingerprint).  Owners of a temporal table also
// link their cell to its history cell.
//
// The four vertices go through each step together so that their memory
// operations overlap: keys; merging of equal keys among the four (their
// contributions are summed in registers and sent with one atomic); the first
// probe of every distinct key (four compare-and-swaps in flight); the rare
// longer probes; the accumulating reds; and the owners' history probes.
struct Four {
  uint32_t slot[4];
  bool owner[4];
};

__device__ __forceinline__ Four insert_four(const KeyConst& kc, const TableDev& t,
                                            const VertexPtrs& v, size_t j, size_t end, bool vec,
                                            unsigned long long& n_ovf, unsigned long long& n_cells,
                                            unsigned long long& n_hovf) {
  const float4 PX = load4(v.px, j, end, vec), PY = load4(v.py, j, end, vec),
               PZ = load4(v.pz, j, end, vec);
  const float4 NX = load4(v.nx, j, end, vec), NY = load4(v.ny, j, end, vec),
               NZ = load4(v.nz, j, end, vec);
  uint32_t h1[4], f[4];
  bool lead[4];
  int of[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool valid = j + q < end;
    Key k{0u, 0u};
    if (valid)
      k = vertex_key(kc, comp(PX, q), comp(PY, q), comp(PZ, q), comp(NX, q), comp(NY, q),
                     comp(NZ, q), vertex_id(v, j + q), v.stream_id);
    h1[q] = k.h1;
    f[q] = k.fp;  // 0 marks an absent vertex (fingerprints are never 0)
    lead[q] = valid;
    of[q] = q;
  }
  // merge equal keys: a later vertex joins the first earlier one with its key
#pragma unroll
  for (int q = 1; q < 4; ++q) {
#pragma unroll
    for (int p = 0; p < q; ++p) {
      if (lead[q] && lead[p] && of[q] == q && h1[p] == h1[q] && f[p] == f[q]) {
        lead[q] = false;
        of[q] = p;
      }
    }
  }
  const float4 R = load4(v.r, j, end, vec), G = load4(v.g, j, end, vec),
               B = load4(v.b, j, end, vec);
  float sr[4], sg[4], sb[4];
  long long fr[4], fg[4], fb[4];
  uint32_t cnt[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    sr[q] = 0.f;
    sg[q] = 0.f;
    sb[q] = 0.f;
    fr[q] = fg[q] = fb[q] = 0;
    cnt[q] = 0u;
  }
  // (static indices only: both loops unroll completely)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool use = f[q] != 0u;
    const float r = use ? comp(R, q) : 0.f, g = use ? comp(G, q) : 0.f, b = use ? comp(B, q) : 0.f;
    long long xr = 0, xg = 0, xb = 0;
    if (t.fixed) {
      xr = to_fixed(r);
      xg = to_fixed(g);
      xb = to_fixed(b);
    }
#pragma unroll
    for (int p = 0; p <= q; ++p) {
      if (!use || of[q] != p) continue;
      sr[p] = __fadd_rn(sr[p], r);
      sg[p] = __fadd_rn(sg[p], g);
      sb[p] = __fadd_rn(sb[p], b);
      fr[p] += xr;
      fg[p] += xg;
      fb[p] += xb;
      ++cnt[p];
    }
  }
  // first probe of every distinct key, all in flight together
  const ProbeTable fpt = frame_probe(t);
  uint32_t old[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    old[q] = lead[q] ? atomicCAS(probe_fp(fpt, h1[q] & t.mask), 0u, f[q]) : 0u;
  uint32_t slot[4];
  bool claimed[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    slot[q] = kOverflowSlot;
    claimed[q] = false;
    if (!lead[q]) continue;
    if (old[q] == 0u || old[q] == f[q]) {
      slot[q] = h1[q] & t.mask;
      claimed[q] = old[q] == 0u;
    } else {
      bool c;
      slot[q] = probe_insert_from(fpt, h1[q] & t.mask, f[q], 1u, c);
      claimed[q] = c;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (lead[q] && slot[q] != kOverflowSlot)
      accumulate(t, slot[q], sr[q], sg[q], sb[q], fr[q], fg[q], fb[q], cnt[q]);
  // owners of a temporal table find or claim their history cell
  if (t.hist_mode) {
    const ProbeTable hpt = hist_probe(t);
    uint32_t hold[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      hold[q] = claimed[q] ? atomicCAS(probe_fp(hpt, h1[q] & t.hmask), 0u, f[q]) : 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!claimed[q]) continue;
      uint32_t h = h1[q] & t.hmask;
      if (hold[q] != 0u && hold[q] != f[q]) {
        bool hc;
        h = probe_insert_from(hpt, h1[q] & t.hmask, f[q], 1u, hc);
      }
      n_hovf += h == kOverflowSlot ? 1ull : 0ull;
      __stcg(frame_hslot(t, slot[q]), h);
    }
  }
  Four out;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t sl = slot[0];
#pragma unroll
    for (int p = 1; p <= q; ++p)
      if (of[q] == p) sl = slot[p];
    out.slot[q] = f[q] == 0u ? kOverflowSlot : sl;
    out.owner[q] = claimed[q];
    if (f[q] != 0u && out.slot[q] == kOverflowSlot) ++n_ovf;
    n_cells += claimed[q] ? 1ull : 0ull;
  }
  return out;
}

struct Result {
  float r, g, b;
  uint32_t n;
  uint8_t status;
};

// Look up the four cells s[0..3] (loads issued together) and resolve each
// vertex: cell average / blended value, or its own contribution on overflow.
__device__ __forceinline__ void resolve_four(const TableDev& t, const VertexPtrs& v, size_t j,
                                             size_t end, const uint32_t (&s)[4], bool blended,
                                             Result (&res)[4]) {
  AccRaw a[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (j + q < end && s[q] != kOverflowSlot) a[q] = load_value(t, s[q], blended);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    res[q] = Result{0.f, 0.f, 0.f, 0u, 0};
    if (j + q >= end) continue;
    if (s[q] == kOverflowSlot) {
      // probe limit exceeded: the unfiltered contribution of the vertex itself
      res[q].r = __ldcs(v.r + j + q);
      res[q].g = __ldcs(v.g + j + q);
      res[q].b = __ldcs(v.b + j + q);
      res[q].status = 2;
    } else {
      const CellMean m = value_of(t, a[q], blended);
      res[q].r = m.r;
      res[q].g = m.g;
      res[q].b = m.b;
      res[q].n = m.n;
      res[q].status = m.n < t.lowcount ? 1 : 0;
    }
  }
}

// Blend the owned cells among four stash entries, loads issued together.
__device__ __forceinline__ void blend_four(const TableDev& t, const uint32_t (&s)[4],
                                           const bool (&own)[4], float alpha) {
  AccRaw a[4];
  uint32_t h[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (!own[q]) continue;
    a[q] = load_acc(t, s[q]);
    h[q] = __ldcg(frame_hslot(t, s[q]));
  }
  HistRaw old[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    old[q] = HistRaw{0.f, 0.f, 0.f, 0u};
    if (own[q] && h[q] != kOverflowSlot) old[q] = load_hist(t, h[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (own[q]) blend_store(t, s[q], h[q], mean_of(t, a[q]), old[q], alpha);
}

__device__ __forceinline__ void store_four(const OutPtrs& o, size_t j, size_t end, bool vec,
                                           const Result (&res)[4]) {
  if (vec && j + 4 <= end) {
    __stcs(reinterpret_cast<float4*>(o.r + j), make_float4(res[0].r, res[1].r, res[2].r, res[3].r));
    __stcs(reinterpret_cast<float4*>(o.g + j), make_float4(res[0].g, res[1].g, res[2].g, res[3].g));
    __stcs(reinterpret_cast<float4*>(o.b + j), make_float4(res[0].b, res[1].b, res[2].b, res[3].b));
    if (o.count)
      __stcs(reinterpret_cast<uint4*>(o.count + j), make_uint4(res[0].n, res[1].n, res[2].n, res[3].n));
    if (o.status) {
      const uint32_t w = res[0].status | (res[1].status << 8) | (res[2].status << 16) |
                         (static_cast<uint32_t>(res[3].status) << 24);
      __stcs(reinterpret_cast<unsigned int*>(o.status + j), w);
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (j + q < end) {
      o.r[j + q] = res[q].r;
      o.g[j + q] = res[q].g;
      o.b[j + q] = res[q].b;
      if (o.count) o.count[j + q] = res[q].n;
      if (o.status) o.status[j + q] = res[q].status;
    }
  }
}

// ------------------------------------------------------------------ split path
__global__ void __launch_bounds__(kBlock) k_insert(KeyConst kc, TableDev t, VertexPtrs v,
                                                   size_t n, uint32_t* slot_out, int vec) {
  __shared__ uint32_t s_cells[kBlock * 4];
  __shared__ uint32_t s_count, s_base;
  unsigned long long n_ovf = 0, n_cells = 0, n_hovf = 0;
  const size_t ngroups = (n + 3) / 4;
  const size_t tiles = (ngroups + kBlock - 1) / kBlock;
  for (size_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const size_t j = (tile * kBlock + threadIdx.x) * 4;
    if (j < n) {
      const Four f = insert_four(kc, t, v, j, n, vec != 0, n_ovf, n_cells, n_hovf);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (f.owner[q]) s_cells[atomicAdd(&s_count, 1u)] = f.slot[q];
        if (slot_out && j + q < n) slot_out[j + q] = f.slot[q];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_base = s_count ? atomicAdd(&t.ctrl->dirty_count, s_count) : 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < s_count; i += kBlock) t.dirty[s_base + i] = s_cells[i];
    __syncthreads();
  }
  const unsigned long long a = block_sum(n_ovf);
  const unsigned long long c = block_sum(n_cells);
  const unsigned long long h = block_sum(n_hovf);
  if (threadIdx.x == 0) {
    if (a) atomicAdd(&t.ctrl->overflow_vertices, a);
    if (c) atomicAdd(&t.ctrl->frame_cells, c);
    if (h) atomicAdd(&t.ctrl->hist_overflow, h);
    if (blockIdx.x == 0) atomicAdd(&t.ctrl->vertices, static_cast<unsigned long long>(n));
  }
}

__global__ void __launch_bounds__(kBlock) k_query(KeyConst kc, TableDev t, VertexPtrs v, size_t n,
                                                  const uint32_t* slot_in, OutPtrs o, int vec,
                                                  int ovec, int blended) {
  const size_t ngroups = (n + 3) / 4;
  for (size_t gi = blockIdx.x * (size_t)blockDim.x + threadIdx.x; gi < ngroups;
       gi += (size_t)gridDim.x * blockDim.x) {
    const size_t j = gi * 4;
    uint32_t s[4];
    if (slot_in) {
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] = j + q < n ? __ldcs(slot_in + j + q) : kOverflowSlot;
    } else {
      const float4 PX = load4(v.px, j, n, vec), PY = load4(v.py, j, n, vec),
                   PZ = load4(v.pz, j, n, vec);
      const float4 NX = load4(v.nx, j, n, vec), NY = load4(v.ny, j, n, vec),
                   NZ = load4(v.nz, j, n, vec);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        s[q] = kOverflowSlot;
        if (j + q < n) {
          const Key k = vertex_key(kc, comp(PX, q), comp(PY, q), comp(PZ, q), comp(NX, q),
                                   comp(NY, q), comp(NZ, q), vertex_id(v, j + q), v.stream_id);
          s[q] = probe_find(t, k.h1 & t.mask, k.fp);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (s[q] != kOverflowSlot && s[q] > t.mask) {  // not a cell of this table
        atomicOr(&t.ctrl->error, kErrBadSlot);
        s[q] = kOverflowSlot;
      }
    }
    Result res[4];
    resolve_four(t, v, j, n, s, blended != 0, res);
    store_four(o, j, n, ovec != 0, res);
  }
}

__global__ void __launch_bounds__(kBlock) k_blend(TableDev t, float alpha) {
  const uint32_t cnt = t.ctrl->dirty_count;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    blend_cell(t, t.dirty[i], alpha);
}

__global__ void __launch_bounds__(kBlock) k_clear_dirty(TableDev t) {
  const uint32_t cnt = t.ctrl->dirty_count;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    clear_cell(t, t.dirty[i]);
}

__global__ void __launch_bounds__(kBlock) k_keys(KeyConst kc, VertexPtrs v, size_t n,
                                                 uint32_t* h_out, uint32_t* f_out) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n;
       j += (size_t)gridDim.x * blockDim.x) {
    const Key k = vertex_key(kc, __ldcs(v.px + j), __ldcs(v.py + j), __ldcs(v.pz + j),
                             __ldcs(v.nx + j), __ldcs(v.ny + j), __ldcs(v.nz + j),
                             vertex_id(v, j), v.stream_id);
    h_out[j] = k.h1;
    f_out[j] = k.fp;
  }
}

__global__ void __launch_bounds__(kBlock) k_count_occupied(const unsigned char* cells,
                                                           uint32_t stride, uint32_t fp_off,
                                                           uint32_t T, unsigned long long* out) {
  unsigned long long c = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < T; i += gridDim.x * blockDim.x)
    c += *reinterpret_cast<const uint32_t*>(cells + static_cast<size_t>(i) * stride + fp_off) != 0u;
  const unsigned long long s = block_sum(c);
  if (threadIdx.x == 0 && s) atomicAdd(out, s);
}

// ------------------------------------------------------------------ fused path
struct FusedArgs {
  KeyConst kc;
  TableDev t;
  VertexPtrs v;
  OutPtrs o;
  size_t n;
  size_t chunk;
  uint32_t* gstash;
  float alpha;
  int vec, ovec, blend;
};

template <bool TEMPORAL>
__global__ void __launch_bounds__(kFusedBlock, 1) k_fused(FusedArgs a) {
  extern __shared__ __align__(16) uint32_t s_stash[];
  const TableDev& t = a.t;
  const size_t beg = static_cast<size_t>(blockIdx.x) * a.chunk;
  const size_t end = min(a.n, beg + a.chunk);
  uint32_t* stash = a.gstash ? a.gstash + beg : s_stash;
  const bool vec = a.vec != 0;
  const size_t step = 4 * static_cast<size_t>(blockDim.x);

  // Phase A: keys, probing insert, accumulation.
  unsigned long long n_ovf = 0, n_cells = 0, n_hovf = 0;
  for (size_t j = beg + 4 * threadIdx.x; j < end; j += step) {
    const Four f = insert_four(a.kc, t, a.v, j, end, vec, n_ovf, n_cells, n_hovf);
    uint4 w;
    w.x = f.slot[0] == kOverflowSlot ? kStashOverflow : (f.slot[0] | (f.owner[0] ? kOwnerBit : 0u));
    w.y = f.slot[1] == kOverflowSlot ? kStashOverflow : (f.slot[1] | (f.owner[1] ? kOwnerBit : 0u));
    w.z = f.slot[2] == kOverflowSlot ? kStashOverflow : (f.slot[2] | (f.owner[2] ? kOwnerBit : 0u));
    w.w = f.slot[3] == kOverflowSlot ? kStashOverflow : (f.slot[3] | (f.owner[3] ? kOwnerBit : 0u));
    *reinterpret_cast<uint4*>(stash + (j - beg)) = w;
  }
  {
    const unsigned long long o = block_sum(n_ovf);
    const unsigned long long c = block_sum(n_cells);
    const unsigned long long h = block_sum(n_hovf);
    if (threadIdx.x == 0) {
      if (o) atomicAdd(&t.ctrl->overflow_vertices, o);
      if (c) atomicAdd(&t.ctrl->frame_cells, c);
      if (h) atomicAdd(&t.ctrl->hist_overflow, h);
      if (end > beg) atomicAdd(&t.ctrl->vertices, static_cast<unsigned long long>(end - beg));
    }
  }
  if (!grid_barrier(t.ctrl, gridDim.x)) return;

  // Phase B: temporal blend, once per touched cell by its owner.
  const bool blended = TEMPORAL && a.blend;
  if (blended) {
    for (size_t j = beg + 4 * threadIdx.x; j < end; j += step) {
      const uint4 w = *reinterpret_cast<const uint4*>(stash + (j - beg));
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
      uint32_t sl[4];
      bool own[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        own[q] = j + q < end && ws[q] != kStashOverflow && (ws[q] & kOwnerBit);
        sl[q] = ws[q] & ~kOwnerBit;
      }
      blend_four(t, sl, own, a.alpha);
    }
    if (!grid_barrier(t.ctrl, gridDim.x)) return;
  }

  // Phase C: one lookup per vertex.
  const bool ovec = a.ovec != 0;
  for (size_t j = beg + 4 * threadIdx.x; j < end; j += step) {
    const uint4 w = *reinterpret_cast<const uint4*>(stash + (j - beg));
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    uint32_t sl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) sl[q] = ws[q] == kStashOverflow ? kOverflowSlot : (ws[q] & ~kOwnerBit);
    Result res[4];
    resolve_four(t, a.v, j, end, sl, blended, res);
    store_four(a.o, j, end, ovec, res);
  }
  if (!grid_barrier(t.ctrl, gridDim.x)) return;

  // Phase D: owners empty their cells for the next frame.
  for (size_t j = beg + 4 * threadIdx.x; j < end; j += step) {
    const uint4 w = *reinterpret_cast<const uint4*>(stash + (j - beg));
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (j + q < end && ws[q] != kStashOverflow && (ws[q] & kOwnerBit))
        clear_cell(t, ws[q] & ~kOwnerBit);
  }
}

int sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  int c = 0;
  cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
  return c > 0 ? c : 1;
}

int split_grid(size_t work_items) {
  const size_t want = (work_items + kBlock - 1) / kBlock;
  const size_t cap = static_cast<size_t>(sm_count()) * 8;
  return static_cast<int>(std::max<size_t>(1, std::min(want, cap)));
}

}  // namespace

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static bool vec_inputs(const VertexPtrs& v) {
  return aligned16(v.px) && aligned16(v.py) && aligned16(v.pz) && aligned16(v.nx) &&
         aligned16(v.ny) && aligned16(v.nz) && aligned16(v.r) && aligned16(v.g) &&
         aligned16(v.b);
}

static bool vec_outputs(const OutPtrs& o) {
  return aligned16(o.r) && aligned16(o.g) && aligned16(o.b) && (!o.count || aligned16(o.count)) &&
         (!o.status || (reinterpret_cast<uintptr_t>(o.status) & 3u) == 0);
}

cudaError_t launch_insert(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                          uint32_t* slot_out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_insert<<<split_grid((n + 3) / 4), kBlock, 0, st>>>(kc, t, v, n, slot_out, vec_inputs(v) ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_query(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                         const uint32_t* slot_in, const OutPtrs& o, bool blended,
                         cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_query<<<split_grid((n + 3) / 4), kBlock, 0, st>>>(kc, t, v, n, slot_in, o,
                                                      vec_inputs(v) ? 1 : 0,
                                                      vec_outputs(o) ? 1 : 0, blended ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_keys(const KeyConst& kc, const VertexPtrs& v, size_t n, uint32_t* h_out,
                        uint32_t* f_out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_keys<<<split_grid(n), kBlock, 0, st>>>(kc, v, n, h_out, f_out);
  return cudaGetLastError();
}

cudaError_t launch_blend(const TableDev& t, float alpha, cudaStream_t st) {
  k_blend<<<sm_count() * 8, kBlock, 0, st>>>(t, alpha);
  return cudaGetLastError();
}

cudaError_t launch_clear_dirty(const TableDev& t, cudaStream_t st) {
  k_clear_dirty<<<sm_count() * 8, kBlock, 0, st>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_count_occupied(const unsigned char* cells, uint32_t stride, uint32_t fp_off,
                                  uint32_t T, unsigned long long* out, cudaStream_t st) {
  k_count_occupied<<<sm_count() * 4, kBlock, 0, st>>>(cells, stride, fp_off, T, out);
  return cudaGetLastError();
}

// Largest dynamic shared memory a k_fused CTA may request: the opt-in limit
// per block minus the kernel's static shared memory.
template <bool TEMPORAL>
static cudaError_t fused_dyn_smem_limit(size_t* limit) {
  static size_t cached = 0;
  if (!cached) {
    int dev = 0, maxopt = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_fused<TEMPORAL>);
    if (e != cudaSuccess) return e;
    const size_t lim = static_cast<size_t>(maxopt) - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(k_fused<TEMPORAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(lim));
    if (e != cudaSuccess) return e;
    cached = lim;
  }
  *limit = cached;
  return cudaSuccess;
}

template <bool TEMPORAL>
static cudaError_t fused_blocks_per_sm(size_t smem, int* nb) {
  size_t lim = 0;
  cudaError_t e = fused_dyn_smem_limit<TEMPORAL>(&lim);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_fused<TEMPORAL>, kFusedBlock, smem);
}

cudaError_t plan_fused(size_t n, bool temporal, FusedPlan* plan) {
  const int sms = sm_count();
  size_t maxdyn = 0;
  cudaError_t e = temporal ? fused_dyn_smem_limit<true>(&maxdyn) : fused_dyn_smem_limit<false>(&maxdyn);
  if (e != cudaSuccess) return e;
  int b0 = 0;
  e = temporal ? fused_blocks_per_sm<true>(0, &b0) : fused_blocks_per_sm<false>(0, &b0);
  if (e != cudaSuccess) return e;
  if (b0 < 1) return cudaErrorInvalidConfiguration;
  for (int b = b0; b >= 1; --b) {
    const int grid = sms * b;
    size_t chunk = (n + grid - 1) / grid;
    chunk = std::max<size_t>((chunk + 3) & ~static_cast<size_t>(3), 4);
    const size_t smem = chunk * sizeof(uint32_t);
    if (smem > maxdyn) continue;
    int nb = 0;
    e = temporal ? fused_blocks_per_sm<true>(smem, &nb) : fused_blocks_per_sm<false>(smem, &nb);
    if (e != cudaSuccess) return e;
    if (nb >= b) {
      plan->grid = grid;
      plan->block = kFusedBlock;
      plan->chunk = chunk;
      plan->smem = smem;
      plan->global_stash = false;
      return cudaSuccess;
    }
  }
  // The stash does not fit on chip: keep it in a global scratch buffer.
  const int grid = sms * b0;
  size_t chunk = (n + grid - 1) / grid;
  chunk = std::max<size_t>((chunk + 3) & ~static_cast<size_t>(3), 4);
  plan->grid = grid;
  plan->block = kFusedBlock;
  plan->chunk = chunk;
  plan->smem = 0;
  plan->global_stash = true;
  return cudaSuccess;
}

cudaError_t launch_fused(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                         const OutPtrs& o, bool temporal, bool blend, float alpha,
                         const FusedPlan& plan, uint32_t* gstash, cudaStream_t st) {
  FusedArgs a;
  a.kc = kc;
  a.t = t;
  a.v = v;
  a.o = o;
  a.n = n;
  a.chunk = plan.chunk;
  a.gstash = plan.global_stash ? gstash : nullptr;
  a.alpha = alpha;
  a.vec = vec_inputs(v) ? 1 : 0;
  a.ovec = vec_outputs(o) ? 1 : 0;
  a.blend = blend ? 1 : 0;
  void* args[] = {&a};
  const void* fn = temporal ? reinterpret_cast<const void*>(k_fused<true>)
                            : reinterpret_cast<const void*>(k_fused<false>);
  return cudaLaunchCooperativeKernel(fn, dim3(plan.grid), dim3(plan.block), args, plan.smem, st);
}

}  // namespace pps
