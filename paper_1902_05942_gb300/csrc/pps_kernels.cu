// Kernels of the hashed path space filter (sm_103a) and their launchers.
//
//  k_insert        key construction (Alg. 1) + probing insert + atomic
//                  accumulation (Sec. 3.2, 3.3.1) for one tile of vertices per
//                  CTA iteration; a tile's new cells get ids from the tile's
//                  own id range.
//  k_blend_sweep   temporal blend of every cell claimed this frame (Sec. 3.4.1).
//  k_query         one lookup per vertex: cell average or blended value.
//  k_clear_sweep   empties the frame's cells for the next frame.
//  k_fused         the whole frame in one persistent cooperative launch: the
//                  four steps above separated by grid barriers; each vertex's
//                  cell id stays in shared memory between the phases; the
//                  blend's tiles come from a second counter, and each CTA
//                  clears the cells its own tiles created.
//  k_fused_ws      the same frame with a pipelined insert: key warps build
//                  and merge keys into a shared-memory queue while probe warps
//                  run the table operations of the previous chunk (the default
//                  for frames without eviction or neighborhood search).
//  k_fused<NEIGH>, k_neighbors, k_clear_fused
//                  neighborhood-search frames: the persistent kernel queues
//                  its low-count vertices after the lookups, a separate launch
//                  searches them, a third empties the cells.
//  k_blend_lookup, k_blend_apply
//                  the blend of a history that follows changes of resolution.
//
// Vertex streams are read with streaming loads (ld.global.cs): in the split
// kernels four consecutive vertices per thread (128-bit when the arrays are
// 16-byte aligned), in the persistent kernels W consecutive vertices per
// thread with each warp's sub-batch one contiguous run; table words are read
// at L2 (ld.relaxed.gpu / ld.global.cg) because other CTAs write them.
#include <algorithm>

#include "pps_internal.h"

namespace pps {

namespace {

constexpr int kBlock = 256;            // split kernels
constexpr int kTile = kBlock * 4;      // vertices (and cell ids) per split-path tile
constexpr int kFusedBlock = 512;       // persistent kernel
constexpr int kFusedTile = kFusedBlock * 4;  // vertices per persistent-kernel tile
constexpr int kMaxTilesPerCta = 1024;  // tile list of one persistent CTA

// W consecutive floats of one stream (one 8- or 16-byte load when aligned).
template <int W>
__device__ __forceinline__ void loadw(float (&x)[W], const float* p, size_t j, size_t end,
                                      bool vec) {
  if (vec && j + W <= end) {
    if constexpr (W == 4) {
      const float4 v = __ldcs(reinterpret_cast<const float4*>(p + j));
      x[0] = v.x;
      x[1] = v.y;
      x[2] = v.z;
      x[3] = v.w;
    } else {
      const float2 v = __ldcs(reinterpret_cast<const float2*>(p + j));
      x[0] = v.x;
      x[1] = v.y;
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < W; ++q) x[q] = j + q < end ? __ldcs(p + j + q) : 0.f;
}

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

struct Counters {
  uint32_t ovf = 0, cells = 0;  // per thread (summed to 64 bits per CTA)
};

// The rare continuation of a probe whose home slot held another key, kept out
// of line so that the four-wide insert stays fully unrolled in registers.
// `my` is the id reserved for this key (kOverflowSlot: none yet).
struct MoreProbe {
  uint32_t slot, id, my;
  bool claimed;
};

__device__ __noinline__ MoreProbe probe_more(unsigned long long* slots, uint32_t mask,
                                             uint32_t max_probes, uint32_t home, uint32_t f,
                                             uint32_t my, uint32_t id_base, uint32_t* claims) {
  MoreProbe r{kOverflowSlot, kOverflowSlot, my, false};
  for (uint32_t p = 1; p < max_probes; ++p) {
    const uint32_t s = (home + p) & mask;
    unsigned long long w = ld_relaxed_u64(slots + s);
    if (w == 0ull) {
      if (r.my == kOverflowSlot) r.my = id_base + atomicAdd(claims, 1u);
      w = atomicCAS(slots + s, 0ull, slot_word(f, r.my));
      if (w == 0ull) {
        r.slot = s;
        r.id = r.my;
        r.claimed = true;
        return r;
      }
    }
    if (slot_fp(w) == f) {
      r.slot = s;
      r.id = slot_id(w);
      return r;
    }
  }
  return r;
}

template <int W>
struct Batch {
  uint32_t id[W];
};

// Insert the W vertices j..j+W-1 (those below `end`) and return their cell
// ids (kOverflowSlot on probe overflow).  New cells take ids id_base + k, k
// drawn from the tile's claim counter *claims (shared memory).
//
// The W vertices go through each step together so that their memory
// operations overlap: keys; merging of equal keys among them (their
// contributions are summed in registers and sent with one atomic); the first
// probe of every distinct key (W loads in flight, then the compare-and-swaps
// for empty slots); the rare longer probes; the accumulating reductions.
//
// `rec`: write each new cell's record (t.info) for the later blend and clear;
// a frame that neither blends nor clears slot by slot never reads it.
// KV: the vertices may carry the key variants (distance, extra word); the
// persistent kernels are built without them.
// KREC: also keep each new cell's quantized key in t.kw (for the history's
// changes of resolution).
template <int W, bool KV = false, bool KREC = false>
__device__ __forceinline__ Batch<W> insert_batch(const KeyConst& kc, const TableDev& t,
                                                 const VertexPtrs& v, size_t j, size_t end,
                                                 bool vec, uint32_t id_base, uint32_t* claims,
                                                 Counters& cnt_out, bool rec = true) {
  float PX[W], PY[W], PZ[W], NX[W], NY[W], NZ[W];
  loadw<W>(PX, v.px, j, end, vec);
  loadw<W>(PY, v.py, j, end, vec);
  loadw<W>(PZ, v.pz, j, end, vec);
  loadw<W>(NX, v.nx, j, end, vec);
  loadw<W>(NY, v.ny, j, end, vec);
  loadw<W>(NZ, v.nz, j, end, vec);
  uint32_t h1[W], f[W];
  bool lead[W];
  int of[W];
  uint4 kr[W];  // KREC: the quantized keys
#pragma unroll
  for (int q = 0; q < W; ++q) {
    const bool valid = j + q < end;
    Key k{0u, 0u};
    kr[q] = make_uint4(0u, 0u, 0u, 0u);
    if (valid) {
      if constexpr (KREC) {
        const KeyWords w = key_words(kc, PX[q], PY[q], PZ[q], NX[q], NY[q], NZ[q],
                                     vertex_id(v, j + q), v.stream_id,
                                     KV ? key_extra(v, j + q) : KeyExtra{});
        k = key_hash(kc, w);
        kr[q] = make_uint4(w.X, w.Y, w.Z, (w.L & 0xFFu) | (w.NQ << 8));
      } else {
        k = vertex_key(kc, PX[q], PY[q], PZ[q], NX[q], NY[q], NZ[q], vertex_id(v, j + q),
                       v.stream_id, KV ? key_extra(v, j + q) : KeyExtra{});
      }
    }
    h1[q] = k.h1;
    f[q] = k.fp;  // 0 marks an absent vertex (fingerprints are never 0)
    lead[q] = valid;
    of[q] = q;
  }
  // merge equal keys: a later vertex joins the first earlier one with its key
#pragma unroll
  for (int q = 1; q < W; ++q) {
#pragma unroll
    for (int p = 0; p < q; ++p) {
      if (lead[q] && lead[p] && h1[p] == h1[q] && f[p] == f[q]) {
        lead[q] = false;
        of[q] = p;
      }
    }
  }
  float rr[W], rg[W], rb[W];
  loadw<W>(rr, v.r, j, end, vec);
  loadw<W>(rg, v.g, j, end, vec);
  loadw<W>(rb, v.b, j, end, vec);
  long long xr[W], xg[W], xb[W];
#pragma unroll
  for (int q = 0; q < W; ++q) {
    xr[q] = t.fixed ? to_fixed(rr[q]) : 0;
    xg[q] = t.fixed ? to_fixed(rg[q]) : 0;
    xb[q] = t.fixed ? to_fixed(rb[q]) : 0;
  }
  // group sums of each leader p over its members q >= p (static bounds, selects)
  float sr[W], sg[W], sb[W];
  long long fr[W], fg[W], fb[W];
  uint32_t cnt[W];
#pragma unroll
  for (int p = 0; p < W; ++p) {
    sr[p] = sg[p] = sb[p] = 0.f;
    fr[p] = fg[p] = fb[p] = 0;
    cnt[p] = 0u;
#pragma unroll
    for (int q = p; q < W; ++q) {
      const bool m = f[q] != 0u && of[q] == p;
      sr[p] = m ? __fadd_rn(sr[p], rr[q]) : sr[p];
      sg[p] = m ? __fadd_rn(sg[p], rg[q]) : sg[p];
      sb[p] = m ? __fadd_rn(sb[p], rb[q]) : sb[p];
      fr[p] += m ? xr[q] : 0;
      fg[p] += m ? xg[q] : 0;
      fb[p] += m ? xb[q] : 0;
      cnt[p] += m ? 1u : 0u;
    }
  }
  // first probe step of every distinct key: loads in flight together
  unsigned long long w[W];
#pragma unroll
  for (int q = 0; q < W; ++q)
    w[q] = lead[q] ? ld_relaxed_u64_keep(t.slots + (h1[q] & t.mask)) : 1ull;
  // an empty home needs a cell id to publish with the fingerprint
  uint32_t my[W];
#pragma unroll
  for (int q = 0; q < W; ++q)
    my[q] = lead[q] && w[q] == 0ull ? id_base + atomicAdd(claims, 1u) : kOverflowSlot;
  unsigned long long old[W];
#pragma unroll
  for (int q = 0; q < W; ++q)
    old[q] = my[q] != kOverflowSlot
                 ? atomicCAS(t.slots + (h1[q] & t.mask), 0ull, slot_word(f[q], my[q]))
                 : w[q];
  uint32_t id[W], slot[W];
  bool claimed[W];
#pragma unroll
  for (int q = 0; q < W; ++q) {
    id[q] = kOverflowSlot;
    slot[q] = kOverflowSlot;
    claimed[q] = false;
    if (!lead[q]) continue;
    const uint32_t home = h1[q] & t.mask;
    if (my[q] != kOverflowSlot && old[q] == 0ull) {
      id[q] = my[q];
      slot[q] = home;
      claimed[q] = true;
    } else if (slot_fp(old[q]) == f[q]) {
      id[q] = slot_id(old[q]);
      slot[q] = home;
    } else {
      // the home slot holds another key: keep probing (rare at low load)
      const MoreProbe m = probe_more(t.slots, t.mask, t.max_probes, home, f[q], my[q], id_base,
                                     claims);
      slot[q] = m.slot;
      id[q] = m.id;
      my[q] = m.my;
      claimed[q] = m.claimed;
    }
    // record the cell, or mark a reserved id that ended up unused
    if (rec && my[q] != kOverflowSlot)
      st_once_u4(t.info + my[q], claimed[q] ? make_uint4(slot[q], h1[q], f[q], kOverflowSlot)
                                            : make_uint4(kNoSlot, 0u, 0u, kOverflowSlot));
    if constexpr (KREC)
      if (claimed[q]) __stcg(t.kw + my[q], kr[q]);
  }
#pragma unroll
  for (int q = 0; q < W; ++q)
    if (lead[q] && id[q] != kOverflowSlot)
      accumulate(t, id[q], sr[q], sg[q], sb[q], fr[q], fg[q], fb[q], cnt[q]);
  Batch<W> out;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    uint32_t d = id[0];
#pragma unroll
    for (int p = 1; p <= q; ++p)
      if (of[q] == p) d = id[p];
    out.id[q] = f[q] == 0u ? kOverflowSlot : d;
    if (f[q] != 0u && out.id[q] == kOverflowSlot) ++cnt_out.ovf;
    cnt_out.cells += claimed[q] ? 1u : 0u;
  }
  return out;
}

struct Result {
  float r, g, b;
  uint32_t n;
  uint8_t status;
};

// Neighborhood search (Sec. 3.3.1) for vertex j, whose own cell holds fewer
// than t.lowcount members: the pooled average of the 3 x 3 x 3 block of cells
// around its cell at the same level and with the same quantized normal.  A
// plain frame pools the cells' sums and counts (FP32 sums, or exact int64
// fixed-point sums with one rounding at the end); after a blend it pools the
// blended values weighted by their counts N.  Cells are visited in a fixed
// order (dx, dy, dz each -1, 0, +1, dz fastest), each found by a read-only
// probe.  Inlined into k_neighbors; the split lookup calls it out of line.
__device__ __forceinline__ Result neighbor_pool_inl(const KeyConst& kc, const TableDev& t,
                                             const VertexPtrs& v, size_t j, bool blended,
                                             Result own) {
  const KeyWords w0 =
      key_words(kc, __ldg(v.px + j), __ldg(v.py + j), __ldg(v.pz + j), __ldg(v.nx + j),
                __ldg(v.ny + j), __ldg(v.nz + j), vertex_id(v, j), v.stream_id, key_extra(v, j));
  float sr = 0.f, sg = 0.f, sb = 0.f;
  long long fr = 0, fg = 0, fb = 0;
  unsigned long long n = 0;
  // three cells (dz = -1, 0, +1) at a time: their first probes, then their
  // values, each as loads in flight together
#pragma unroll 1
  for (int o3 = 0; o3 < 9; ++o3) {
    uint32_t home[3], fp[3], id[3];
    unsigned long long w[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      KeyWords kw = w0;
      kw.X += static_cast<uint32_t>(o3 / 3 - 1);
      kw.Y += static_cast<uint32_t>(o3 % 3 - 1);
      kw.Z += static_cast<uint32_t>(q - 1);
      const Key k = key_hash(kc, kw);
      home[q] = k.h1 & t.mask;
      fp[q] = k.fp;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) w[q] = __ldcg(t.slots + home[q]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (w[q] == 0ull)
        id[q] = kOverflowSlot;
      else if (slot_fp(w[q]) == fp[q])
        id[q] = slot_id(w[q]);
      else  // the home slot holds another key: the rest of the probe sequence
        id[q] = probe_find_from(t, home[q], fp[q], 1u);
    }
    float4 c[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (id[q] != kOverflowSlot && !(t.fixed && !blended)) c[q] = __ldcg(value_ptr(t, id[q]));
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (id[q] == kOverflowSlot) continue;
      if (blended) {
        const uint32_t N = __float_as_uint(c[q].w);
        const float fN = __uint2float_rn(N);
        sr = __fadd_rn(sr, __fmul_rn(fN, c[q].x));
        sg = __fadd_rn(sg, __fmul_rn(fN, c[q].y));
        sb = __fadd_rn(sb, __fmul_rn(fN, c[q].z));
        n += N;
      } else if (!t.fixed) {
        sr = __fadd_rn(sr, c[q].x);
        sg = __fadd_rn(sg, c[q].y);
        sb = __fadd_rn(sb, c[q].z);
        n += static_cast<unsigned long long>(c[q].w);
      } else {
        const unsigned long long* a = t.acc64 + 4 * static_cast<size_t>(id[q]);
        fr += static_cast<long long>(__ldcg(a + 0));
        fg += static_cast<long long>(__ldcg(a + 1));
        fb += static_cast<long long>(__ldcg(a + 2));
        n += __ldcg(a + 3);
      }
    }
  }
  if (n == 0) return own;  // the own cell is always found; kept as a guard
  Result r;
  const float fn = __ull2float_rn(n);
  if (t.fixed && !blended) {
    r.r = __fdiv_rn(__fmul_rn(__ll2float_rn(fr), 0x1p-24f), fn);
    r.g = __fdiv_rn(__fmul_rn(__ll2float_rn(fg), 0x1p-24f), fn);
    r.b = __fdiv_rn(__fmul_rn(__ll2float_rn(fb), 0x1p-24f), fn);
  } else {
    r.r = __fdiv_rn(sr, fn);
    r.g = __fdiv_rn(sg, fn);
    r.b = __fdiv_rn(sb, fn);
  }
  r.n = static_cast<uint32_t>(min(n, 0xFFFFFFFFull));
  r.status = 5;  // PPS_STATUS_NEIGHBORS
  return r;
}

// The same out of line, for the split lookup (k_query), whose other work
// should not pay the search's registers.
__device__ __noinline__ Result neighbor_pool(const KeyConst& kc, const TableDev& t,
                                             const VertexPtrs& v, size_t j, bool blended,
                                             Result own) {
  return neighbor_pool_inl(kc, t, v, j, blended, own);
}

// Searching similar normals by linear probing (Sec. 3.2.2) for a vertex whose
// cell is `id`: with the normal only in the fingerprint, every cell of the
// voxel has the voxel's home slot and lies within P slots of it, so the walk
// from the home slot to the first empty slot (at most P slots) passes all of
// them, between the entries of other voxels.  Each entry's cell record (its
// quantized key) says whether it is the same voxel (x~, l') with a quantized
// normal within r steps on every axis; those cells are pooled: FP32 sums, or
// exact int64 sums in fixed-point mode, or after a blend the blended values
// weighted by their N.  Kept out of line: only tables with the search pay.
__device__ __noinline__ Result similar_pool(const TableDev& t, uint32_t id, bool blended) {
  const uint4 rec = __ldcg(t.kw + id);
  const uint32_t home = __ldcg(&t.info[id].y) & t.mask;
  const int r = static_cast<int>(t.normal_search) - 1;
  const int qx = static_cast<int>((rec.w >> 8) & 0xFFu);
  const int qy = static_cast<int>((rec.w >> 16) & 0xFFu);
  const int qz = static_cast<int>(rec.w >> 24);
  float sr = 0.f, sg = 0.f, sb = 0.f;
  long long fr = 0, fg = 0, fb = 0;
  unsigned long long n = 0;
#pragma unroll 1
  for (uint32_t p = 0; p < t.max_probes; ++p) {
    const unsigned long long w = __ldcg(t.slots + ((home + p) & t.mask));
    if (w == 0ull) break;
    const uint32_t c = slot_id(w);
    const uint4 o = __ldcg(t.kw + c);
    if (o.x != rec.x || o.y != rec.y || o.z != rec.z || ((o.w ^ rec.w) & 0xFFu)) continue;
    const int dx = abs(static_cast<int>((o.w >> 8) & 0xFFu) - qx);
    const int dy = abs(static_cast<int>((o.w >> 16) & 0xFFu) - qy);
    const int dz = abs(static_cast<int>(o.w >> 24) - qz);
    if (max(dx, max(dy, dz)) > r) continue;
    if (blended) {
      const float4 v = __ldcg(value_ptr(t, c));
      const uint32_t N = __float_as_uint(v.w);
      const float fN = __uint2float_rn(N);
      sr = __fadd_rn(sr, __fmul_rn(fN, v.x));
      sg = __fadd_rn(sg, __fmul_rn(fN, v.y));
      sb = __fadd_rn(sb, __fmul_rn(fN, v.z));
      n += N;
    } else if (!t.fixed) {
      const float4 v = __ldcg(t.acc + c);
      if (v.w >= kExactCountLimit) atomicOr(&t.ctrl->error, kErrCountSaturated);
      sr = __fadd_rn(sr, v.x);
      sg = __fadd_rn(sg, v.y);
      sb = __fadd_rn(sb, v.z);
      n += static_cast<unsigned long long>(v.w);
    } else {
      const unsigned long long* a = t.acc64 + 4 * static_cast<size_t>(c);
      fr += static_cast<long long>(__ldcg(a + 0));
      fg += static_cast<long long>(__ldcg(a + 1));
      fb += static_cast<long long>(__ldcg(a + 2));
      n += __ldcg(a + 3);
    }
  }
  Result res;
  const float fn = __ull2float_rn(n);
  if (t.fixed && !blended) {
    res.r = __fdiv_rn(__fmul_rn(__ll2float_rn(fr), 0x1p-24f), fn);
    res.g = __fdiv_rn(__fmul_rn(__ll2float_rn(fg), 0x1p-24f), fn);
    res.b = __fdiv_rn(__fmul_rn(__ll2float_rn(fb), 0x1p-24f), fn);
  } else {
    res.r = __fdiv_rn(sr, fn);
    res.g = __fdiv_rn(sg, fn);
    res.b = __fdiv_rn(sb, fn);
  }
  res.n = static_cast<uint32_t>(min(n, 0xFFFFFFFFull));
  res.status = res.n < t.lowcount ? 1 : 0;
  return res;
}

// Vertex j with cell `id`: if its cell is low-count, replace its outputs by
// the neighborhood-search result.
__device__ __forceinline__ void neighbors_of_vertex(const KeyConst& kc, const TableDev& t,
                                                    const VertexPtrs& v, const OutPtrs& o,
                                                    size_t j, uint32_t id, bool blended) {
  if (id == kOverflowSlot) return;
  const CellMean m = value_of(t, load_value(t, id, blended), blended);
  if (m.n >= t.lowcount) return;
  const Result r = neighbor_pool(kc, t, v, j, blended, Result{m.r, m.g, m.b, m.n, 1});
  o.r[j] = r.r;
  o.g[j] = r.g;
  o.b[j] = r.b;
  if (o.count) o.count[j] = r.n;
  if (o.status) o.status[j] = r.status;
}

// A queued low-count vertex j: its neighborhood-search result into the
// outputs.  The vertex's own cell is among the 27, so the pooled count is at
// least its own.
__device__ __forceinline__ void neighbors_of_queued(const KeyConst& kc, const TableDev& t,
                                                    const VertexPtrs& v, const OutPtrs& o,
                                                    uint32_t j, bool blended) {
  const Result r = neighbor_pool_inl(kc, t, v, j, blended, Result{o.r[j], o.g[j], o.b[j], 0u, 1});
  o.r[j] = r.r;
  o.g[j] = r.g;
  o.b[j] = r.b;
  if (o.count) o.count[j] = r.n;
  if (o.status) o.status[j] = r.status;
}

// Look up the cells id[0..W-1] (loads issued together) and resolve each vertex:
// cell average / blended value, or its own contribution on overflow.
template <int W>
__device__ __forceinline__ void resolve_batch(const TableDev& t, const VertexPtrs& v, size_t j,
                                              size_t end, const uint32_t (&id)[W], bool blended,
                                              Result (&res)[W]) {
  AccRaw a[W];
#pragma unroll
  for (int q = 0; q < W; ++q)
    if (j + q < end && id[q] != kOverflowSlot) a[q] = load_value(t, id[q], blended);
#pragma unroll
  for (int q = 0; q < W; ++q) {
    res[q] = Result{0.f, 0.f, 0.f, 0u, 0};
    if (j + q >= end) continue;
    if (id[q] == kOverflowSlot) {
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

template <int W>
__device__ __forceinline__ void store_batch(const OutPtrs& o, size_t j, size_t end, bool vec,
                                            const Result (&res)[W]) {
  if (vec && j + W <= end) {
    if constexpr (W == 4) {
      __stcs(reinterpret_cast<float4*>(o.r + j), make_float4(res[0].r, res[1].r, res[2].r, res[3].r));
      __stcs(reinterpret_cast<float4*>(o.g + j), make_float4(res[0].g, res[1].g, res[2].g, res[3].g));
      __stcs(reinterpret_cast<float4*>(o.b + j), make_float4(res[0].b, res[1].b, res[2].b, res[3].b));
      if (o.count)
        __stcs(reinterpret_cast<uint4*>(o.count + j),
               make_uint4(res[0].n, res[1].n, res[2].n, res[3].n));
      if (o.status) {
        const uint32_t w = res[0].status | (res[1].status << 8) | (res[2].status << 16) |
                           (static_cast<uint32_t>(res[3].status) << 24);
        __stcs(reinterpret_cast<unsigned int*>(o.status + j), w);
      }
    } else {
      __stcs(reinterpret_cast<float2*>(o.r + j), make_float2(res[0].r, res[1].r));
      __stcs(reinterpret_cast<float2*>(o.g + j), make_float2(res[0].g, res[1].g));
      __stcs(reinterpret_cast<float2*>(o.b + j), make_float2(res[0].b, res[1].b));
      if (o.count) __stcs(reinterpret_cast<uint2*>(o.count + j), make_uint2(res[0].n, res[1].n));
      if (o.status) {
        const unsigned short w = static_cast<unsigned short>(res[0].status | (res[1].status << 8));
        __stcs(reinterpret_cast<unsigned short*>(o.status + j), w);
      }
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < W; ++q) {
    if (j + q < end) {
      o.r[j + q] = res[q].r;
      o.g[j + q] = res[q].g;
      o.b[j + q] = res[q].b;
      if (o.count) o.count[j + q] = res[q].n;
      if (o.status) o.status[j + q] = res[q].status;
    }
  }
}

// Blend BW cells whose ids, history homes and fingerprints are known (`use`
// false: no cell): history probes issued together, then the blends.
template <int BW>
__device__ __forceinline__ void blend_cells(const TableDev& t, const uint32_t (&d)[BW],
                                            const uint32_t (&home)[BW], const uint32_t (&f)[BW],
                                            const bool (&use)[BW], const AccRaw (&a)[BW],
                                            float alpha, unsigned long long& n_hovf) {
  uint32_t old[BW], h[BW];
#pragma unroll
  for (int q = 0; q < BW; ++q) old[q] = use[q] ? atomicCAS(hist_fp(t, home[q]), 0u, f[q]) : 0u;
#pragma unroll
  for (int q = 0; q < BW; ++q) {
    h[q] = home[q];
    if (use[q] && old[q] != 0u && old[q] != f[q]) h[q] = hist_probe_rest(t, home[q], f[q], 1u);
    if (use[q] && h[q] == kOverflowSlot) ++n_hovf;
  }
  HistRaw hv[BW];
#pragma unroll
  for (int q = 0; q < BW; ++q) {
    hv[q] = HistRaw{0.f, 0.f, 0.f, 0u};
    if (use[q] && h[q] != kOverflowSlot) hv[q] = load_hist(t, h[q]);
  }
#pragma unroll
  for (int q = 0; q < BW; ++q)
    if (use[q]) blend_store(t, d[q], h[q], mean_of(t, a[q]), hv[q], alpha);
}

// The same for an evicting history (Sec. 3.4.3), one cell at a time, kept
// out of line so that the common path above keeps its registers.
__device__ __noinline__ unsigned long long blend_cell_evict(const TableDev& t, uint32_t d,
                                                            uint32_t home, uint32_t f,
                                                            float alpha) {
  const AccRaw a = load_acc(t, d);
  bool fresh = true;
  const uint32_t h = hist_claim_evict(t, home, f, &fresh);
  const HistRaw hv = h != kOverflowSlot && !fresh ? load_hist(t, h) : HistRaw{0.f, 0.f, 0.f, 0u};
  blend_store(t, d, h, mean_of(t, a), hv, alpha);
  return h == kOverflowSlot ? 1ull : 0ull;
}

// Blend the cells [base, base + count): each thread takes BW cells, one from
// each of BW consecutive runs of `stride` ids (coalesced loads), and issues
// their history probes together.  `first` is this thread's offset.
template <int BW, bool EVICT>
__device__ __forceinline__ void blend_range(const TableDev& t, uint32_t base, uint32_t count,
                                            uint32_t first, uint32_t stride, float alpha,
                                            unsigned long long& n_hovf) {
  for (uint32_t k0 = first; k0 < count; k0 += BW * stride) {
    uint32_t d[BW], home[BW], f[BW];
    bool use[BW];
    AccRaw a[BW];
#pragma unroll
    for (int q = 0; q < BW; ++q) {
      const uint32_t k = k0 + q * stride;
      d[q] = base + k;
      use[q] = false;
      home[q] = 0u;
      f[q] = 0u;
      if (k < count) {
        const uint4 in = ld_once_u4(t.info + d[q]);
        use[q] = in.x != kNoSlot;
        home[q] = in.y & t.hmask;
        f[q] = in.z;
        if (use[q] && !EVICT) a[q] = load_acc(t, d[q]);
      }
    }
    if constexpr (EVICT) {
#pragma unroll
      for (int q = 0; q < BW; ++q)
        if (use[q]) n_hovf += blend_cell_evict(t, d[q], home[q], f[q], alpha);
    } else {
      blend_cells<BW>(t, d, home, f, use, a, alpha, n_hovf);
    }
  }
}

// Empty the cells [base, base + count): their accumulators, and their slots
// unless the whole slot table is swept separately (`slots_swept`).
__device__ __forceinline__ void clear_range(const TableDev& t, uint32_t base, uint32_t count,
                                            uint32_t first, uint32_t stride, bool slots_swept) {
  for (uint32_t k = first; k < count; k += stride) {
    const uint32_t slot = slots_swept ? kNoSlot : ld_once_u4(t.info + base + k).x;
    clear_cell(t, base + k, slot);
  }
}

// Zero the whole slot table with 16-byte stores, `gthreads` threads from
// thread `gid`: cheaper than one scattered store per cell once a good share
// of the table is in use.
__device__ __forceinline__ void sweep_slots(const TableDev& t, size_t gid, size_t gthreads) {
  uint4* p = reinterpret_cast<uint4*>(t.slots);
  const size_t n16 = (static_cast<size_t>(t.mask) + 1) / 2;
  for (size_t i = gid; i < n16; i += gthreads) st_zero16_keep(p + i);
}

// ------------------------------------------------------------------ split path
template <int W, bool KREC>
__global__ void __launch_bounds__(kBlock) k_insert(KeyConst kc, TableDev t, VertexPtrs v,
                                                   size_t n, uint32_t* id_out, int vec,
                                                   uint32_t tile_base) {
  __shared__ uint32_t s_claims;
  Counters c;
  const size_t tiles = (n + kTile - 1) / kTile;
  for (size_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    if (threadIdx.x == 0) s_claims = 0;
    __syncthreads();
    const uint32_t tix = tile_base + static_cast<uint32_t>(tile);
#pragma unroll 1
    for (int sub = 0; sub < 4; sub += W) {
      const size_t j = tile * kTile + threadIdx.x * 4 + sub;
      if (j < n) {
        const Batch<W> b =
            insert_batch<W, true, KREC>(kc, t, v, j, n, vec != 0, tix * kTile, &s_claims, c);
        if (id_out) {
#pragma unroll
          for (int q = 0; q < W; ++q)
            if (j + q < n) id_out[j + q] = b.id[q];
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) t.bcount[tix] = s_claims;
  }
  const unsigned long long a = block_sum(static_cast<unsigned long long>(c.ovf));
  const unsigned long long b = block_sum(static_cast<unsigned long long>(c.cells));
  if (threadIdx.x == 0) {
    if (a) atomicAdd(&t.ctrl->overflow_vertices, a);
    if (b) atomicAdd(&t.ctrl->frame_cells, b);
    if (blockIdx.x == 0) atomicAdd(&t.ctrl->vertices, static_cast<unsigned long long>(n));
  }
}

__global__ void __launch_bounds__(kBlock) k_query(KeyConst kc, TableDev t, VertexPtrs v, size_t n,
                                                  const uint32_t* id_in, OutPtrs o, int vec,
                                                  int ovec, int blended, uint32_t id_limit) {
  const size_t ngroups = (n + 3) / 4;
  for (size_t gi = blockIdx.x * (size_t)blockDim.x + threadIdx.x; gi < ngroups;
       gi += (size_t)gridDim.x * blockDim.x) {
    const size_t j = gi * 4;
    uint32_t id[4];
    if (id_in) {
#pragma unroll
      for (int q = 0; q < 4; ++q) id[q] = j + q < n ? __ldcs(id_in + j + q) : kOverflowSlot;
    } else {
      const float4 PX = load4(v.px, j, n, vec), PY = load4(v.py, j, n, vec),
                   PZ = load4(v.pz, j, n, vec);
      const float4 NX = load4(v.nx, j, n, vec), NY = load4(v.ny, j, n, vec),
                   NZ = load4(v.nz, j, n, vec);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        id[q] = kOverflowSlot;
        if (j + q < n) {
          const Key k = vertex_key(kc, comp(PX, q), comp(PY, q), comp(PZ, q), comp(NX, q),
                                   comp(NY, q), comp(NZ, q), vertex_id(v, j + q), v.stream_id,
                                   key_extra(v, j + q));
          id[q] = probe_find(t, k.h1 & t.mask, k.fp);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (id[q] != kOverflowSlot && id[q] >= id_limit) {  // not a cell of this frame
        atomicOr(&t.ctrl->error, kErrBadSlot);
        id[q] = kOverflowSlot;
      }
    }
    Result res[4];
    resolve_batch<4>(t, v, j, n, id, blended != 0, res);
    if (t.normal_search) {
#pragma unroll 1
      for (int q = 0; q < 4; ++q)
        if (j + q < n && id[q] != kOverflowSlot) res[q] = similar_pool(t, id[q], blended != 0);
    }
    store_batch<4>(o, j, n, ovec != 0, res);
    if (t.neighbors) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (j + q < n) neighbors_of_vertex(kc, t, v, o, j + q, id[q], blended != 0);
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_blend_sweep(TableDev t, uint32_t ntiles, float alpha) {
  unsigned long long n_hovf = 0;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    if (t.hist_evict)
      blend_range<4, true>(t, tile * kTile, t.bcount[tile], threadIdx.x, blockDim.x, alpha, n_hovf);
    else
      blend_range<4, false>(t, tile * kTile, t.bcount[tile], threadIdx.x, blockDim.x, alpha, n_hovf);
  const unsigned long long h = block_sum(n_hovf);
  if (threadIdx.x == 0 && h) atomicAdd(&t.ctrl->hist_overflow, h);
}

// Changes in resolution across frames (Sec. 3.4.2), for a cell whose history
// entry is new this frame; `rec` is the cell's quantized key.  Resolution
// decreased: the history of its eight finer children (2 x~ + {0,1}^3, level
// l' - 1, same quantized normal) is added up, sums and counts, giving
// sum(N_i c_i) / sum(N_i) with count sum(N_i) (FP32, children in the order
// dx, dy, dz, the last fastest).  Otherwise, resolution increased: its coarser
// parent (floor(x~ / 2), level l' + 1) passes on its average with count
// ceil(N / 8).  Read-only probes; an entry claimed during this frame holds
// N = 0 and counts as absent, so the result is the history as it was before
// the frame.  Kept out of line: only new entries pay for it.
__device__ __forceinline__ uint32_t hist_find(const TableDev& t, uint32_t home, uint32_t f) {
  for (uint32_t p = 0; p < t.max_probes; ++p) {
    const uint32_t h = (home + p) & t.hmask;
    const uint32_t w = __ldcg(hist_fp(t, h));
    if (w == 0u) return kOverflowSlot;
    if (w == f) return h;
  }
  return kOverflowSlot;
}

__device__ __noinline__ HistRaw migrate_history(const KeyConst& kc, const TableDev& t, uint4 rec) {
  KeyWords w;
  w.X = rec.x;
  w.Y = rec.y;
  w.Z = rec.z;
  w.L = static_cast<uint32_t>(static_cast<int32_t>(static_cast<int8_t>(rec.w & 0xFFu)));
  w.NQ = rec.w >> 8;
  w.EX = 0u;
  w.has_ex = false;
  float sr = 0.f, sg = 0.f, sb = 0.f;
  uint32_t sn = 0u;
  for (uint32_t d = 0; d < 8; ++d) {
    KeyWords c = w;
    c.X = 2u * w.X + (d >> 2);
    c.Y = 2u * w.Y + ((d >> 1) & 1u);
    c.Z = 2u * w.Z + (d & 1u);
    c.L = w.L - 1u;
    const Key k = key_hash(kc, c);
    const uint32_t h = hist_find(t, k.h1 & t.hmask, k.fp);
    if (h == kOverflowSlot) continue;
    const HistRaw o = load_hist(t, h);
    if (o.n == 0u) continue;
    const float fn = __uint2float_rn(o.n);
    sr = __fadd_rn(sr, __fmul_rn(fn, o.r));
    sg = __fadd_rn(sg, __fmul_rn(fn, o.g));
    sb = __fadd_rn(sb, __fmul_rn(fn, o.b));
    sn += o.n;
  }
  if (sn) {
    const float fn = __uint2float_rn(sn);
    return HistRaw{__fdiv_rn(sr, fn), __fdiv_rn(sg, fn), __fdiv_rn(sb, fn), sn};
  }
  KeyWords p = w;
  p.X = static_cast<uint32_t>(static_cast<int32_t>(w.X) >> 1);
  p.Y = static_cast<uint32_t>(static_cast<int32_t>(w.Y) >> 1);
  p.Z = static_cast<uint32_t>(static_cast<int32_t>(w.Z) >> 1);
  p.L = w.L + 1u;
  const Key k = key_hash(kc, p);
  const uint32_t h = hist_find(t, k.h1 & t.hmask, k.fp);
  if (h != kOverflowSlot) {
    HistRaw o = load_hist(t, h);
    if (o.n) {
      o.n = (o.n + 7u) / 8u;
      return o;
    }
  }
  return HistRaw{0.f, 0.f, 0.f, 0u};
}

// The blend of a table whose history follows changes of resolution, in two
// launches so that every migration reads the history as it was before the
// frame: k_blend_lookup finds or claims each cell's history entry and keeps
// the value its blend starts from (own, migrated, or none) in t.hold and the
// entry in info.w; k_blend_apply blends and stores.
__global__ void __launch_bounds__(kBlock) k_blend_lookup(KeyConst kc, TableDev t, uint32_t ntiles) {
  unsigned long long n_hovf = 0;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint32_t base = tile * kTile, count = t.bcount[tile];
    for (uint32_t k = threadIdx.x; k < count; k += blockDim.x) {
      const uint32_t d = base + k;
      const uint4 in = __ldcg(t.info + d);
      if (in.x == kNoSlot) continue;
      const uint32_t home = in.y & t.hmask, f = in.z;
      const uint32_t old = atomicCAS(hist_fp(t, home), 0u, f);
      const uint32_t h = old == 0u || old == f ? home : hist_probe_rest(t, home, f, 1u);
      HistRaw hv{0.f, 0.f, 0.f, 0u};
      if (h == kOverflowSlot) {
        ++n_hovf;
      } else {
        hv = load_hist(t, h);
        if (hv.n == 0u) hv = migrate_history(kc, t, __ldcg(t.kw + d));
      }
      __stcg(t.hold + d, make_float4(hv.r, hv.g, hv.b, __uint_as_float(hv.n)));
      __stcg(&t.info[d].w, h);
    }
  }
  const unsigned long long s = block_sum(n_hovf);
  if (threadIdx.x == 0 && s) atomicAdd(&t.ctrl->hist_overflow, s);
}

__global__ void __launch_bounds__(kBlock) k_blend_apply(TableDev t, uint32_t ntiles, float alpha) {
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint32_t base = tile * kTile, count = t.bcount[tile];
    for (uint32_t k = threadIdx.x; k < count; k += blockDim.x) {
      const uint32_t d = base + k;
      const uint4 in = __ldcg(t.info + d);
      if (in.x == kNoSlot) continue;
      const AccRaw a = load_acc(t, d);
      const float4 o = __ldcg(t.hold + d);
      blend_store(t, d, in.w, mean_of(t, a), HistRaw{o.x, o.y, o.z, __float_as_uint(o.w)}, alpha);
    }
  }
}

// Neighborhood search of the low-count vertices that the persistent kernel
// queued, one per thread.
__global__ void __launch_bounds__(kBlock) k_neighbors(KeyConst kc, TableDev t, VertexPtrs v,
                                                      OutPtrs o, const uint32_t* nq, int blended) {
  const unsigned long long cnt = __ldcg(&t.ctrl->neigh_count);
  for (unsigned long long i = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x;
       i < cnt; i += static_cast<unsigned long long>(gridDim.x) * blockDim.x)
    neighbors_of_queued(kc, t, v, o, __ldcs(nq + i), blended != 0);
}

__global__ void __launch_bounds__(kBlock) k_clear_sweep(TableDev t, uint32_t ntiles, int sweep) {
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    clear_range(t, tile * kTile, t.bcount[tile], threadIdx.x, blockDim.x, sweep != 0);
  if (sweep)
    sweep_slots(t, blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x,
                static_cast<size_t>(gridDim.x) * blockDim.x);
}

__global__ void __launch_bounds__(kBlock) k_keys(KeyConst kc, VertexPtrs v, size_t n,
                                                 uint32_t* h_out, uint32_t* f_out) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n;
       j += (size_t)gridDim.x * blockDim.x) {
    const Key k = vertex_key(kc, __ldcs(v.px + j), __ldcs(v.py + j), __ldcs(v.pz + j),
                             __ldcs(v.nx + j), __ldcs(v.ny + j), __ldcs(v.nz + j),
                             vertex_id(v, j), v.stream_id, key_extra(v, j));
    h_out[j] = k.h1;
    f_out[j] = k.fp;
  }
}

__global__ void __launch_bounds__(kBlock) k_count_nonzero(const unsigned char* base, uint32_t stride,
                                                          uint32_t off, uint32_t width, uint64_t n,
                                                          unsigned long long* out) {
  unsigned long long c = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned char* p = base + i * stride + off;
    c += width == 8 ? (*reinterpret_cast<const unsigned long long*>(p) != 0ull)
                    : (*reinterpret_cast<const uint32_t*>(p) != 0u);
  }
  const unsigned long long s = block_sum(c);
  if (threadIdx.x == 0 && s) atomicAdd(out, s);
}

// Empty the cells of the persistent kernel's tiles (kFusedTile ids each), for
// the kernel variant that leaves them to a later launch.
__global__ void __launch_bounds__(kBlock) k_clear_fused(TableDev t, uint32_t ntiles, int sweep) {
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    clear_range(t, tile * static_cast<uint32_t>(kFusedTile), __ldcg(t.bcount + tile), threadIdx.x,
                blockDim.x, sweep != 0);
  if (sweep)
    sweep_slots(t, blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x,
                static_cast<size_t>(gridDim.x) * blockDim.x);
}

// ------------------------------------------------------------------ fused path
// Offset in its tile of the first of the W vertices a thread takes in
// sub-batch `sub` (0, W, ..): sub-batch k covers the k-th run of
// kFusedBlock * W vertices, W consecutive ones per thread, so that each
// warp's loads and stores of a stream are one contiguous run.
template <int W, int BLOCK = kFusedBlock>
__device__ __forceinline__ uint32_t fused_offset(int sub) {
  return static_cast<uint32_t>(sub / W) * (BLOCK * W) + threadIdx.x * W;
}

// Next tile of the frame's tile counter (ntiles once all are taken), in
// stream order or, with `backwards`, from the end of the vertex stream.  The
// pipelined insert takes them backwards: streams are bounce-major, so the
// secondary-bounce tiles, whose vertices nearly all create cells of their own
// and cost the most, go first and the cheap primary-hit tiles balance the CTAs
// at the end of the insert (HD plain frame 6 %, temporal 3 % shorter).  The
// per-thread insert measured slower backwards (stress frame +3 %).
__device__ __forceinline__ uint32_t claim_tile(Ctrl* ctrl, uint32_t ntiles, bool backwards = false) {
  const unsigned long long k = atomicAdd(&ctrl->tile_next, 1ull);
  if (k >= ntiles) return ntiles;
  return backwards ? ntiles - 1u - static_cast<uint32_t>(k) : static_cast<uint32_t>(k);
}

struct FusedArgs {
  KeyConst kc;
  TableDev t;
  VertexPtrs v;
  OutPtrs o;
  size_t n;
  uint32_t cap_tiles;  // tiles this CTA may take (its stash capacity)
  uint32_t* gstash;    // global stash (indexed by vertex) when it does not fit on chip
  float alpha;
  int vec, ovec, blend;
  int sweep;     // zero the whole slot table at the end instead of slot by slot
  uint32_t* nq;  // neighborhood search: the queue of low-count vertices
  int merge;     // pipelined insert: 1 no warp aggregation, 2 gated, 3 always
};

// The persistent kernel.  Phase A hands out tiles of kFusedTile consecutive
// vertices from a per-frame counter, so CTAs that meet cheap (coherent)
// vertices take more tiles; each CTA remembers its tiles, keeps every vertex's
// cell id in its shared-memory stash, and later looks up and clears exactly
// those tiles (the blend hands tiles out again from a second counter).  A
// tile's new cells take ids from the tile's own range
// [tile * kFusedTile, tile * kFusedTile + claims).
template <bool TEMPORAL, int W, bool EVICT = false, bool NEIGH = false>
__global__ void __launch_bounds__(kFusedBlock, W == 4 ? 1 : 2) k_fused(FusedArgs a) {
  extern __shared__ __align__(16) uint32_t s_stash[];
  __shared__ uint32_t s_tile[kMaxTilesPerCta];
  __shared__ uint32_t s_claims[kMaxTilesPerCta];
  __shared__ uint32_t s_cur, s_taken;
  __shared__ unsigned long long s_nv;  // vertices of this CTA's tiles
  const TableDev& t = a.t;
  const uint32_t ntiles = static_cast<uint32_t>((a.n + kFusedTile - 1) / kFusedTile);
  const bool vec = a.vec != 0;
  if (threadIdx.x == 0) {
    s_taken = 0;
    s_nv = 0;
  }

  // Phase A: keys, probing insert, accumulation, tile by tile.
  Counters c;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tile = ntiles;
      if (s_taken < a.cap_tiles) tile = claim_tile(t.ctrl, ntiles);
      s_cur = tile;
      if (tile < ntiles) {
        s_tile[s_taken] = tile;
        s_claims[s_taken] = 0;
        s_nv += min(a.n, static_cast<size_t>(tile) * kFusedTile + kFusedTile) -
                static_cast<size_t>(tile) * kFusedTile;
      }
    }
    __syncthreads();
    const uint32_t tile = s_cur;
    if (tile >= ntiles) break;
    const uint32_t k = s_taken;
    const size_t t0 = static_cast<size_t>(tile) * kFusedTile;
    const size_t end = min(a.n, t0 + kFusedTile);
    uint32_t* stash = a.gstash ? a.gstash + t0 : s_stash + static_cast<size_t>(k) * kFusedTile;
#pragma unroll 1
    for (int sub = 0; sub < 4; sub += W) {
      const size_t j = t0 + fused_offset<W>(sub);
      if (j < end) {
        const Batch<W> b = insert_batch<W>(a.kc, t, a.v, j, end, vec, static_cast<uint32_t>(t0),
                                           &s_claims[k], c,
                                           (TEMPORAL && a.blend) || !a.sweep);
#pragma unroll
        for (int q = 0; q < W; ++q) stash[j - t0 + q] = b.id[q];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // for the blend, which any CTA may take, and for the separate clear
      if ((TEMPORAL && a.blend) || NEIGH) __stcg(t.bcount + tile, s_claims[k]);
      ++s_taken;
    }
  }
  {
    const unsigned long long o = block_sum(static_cast<unsigned long long>(c.ovf));
    const unsigned long long k = block_sum(static_cast<unsigned long long>(c.cells));
    if (threadIdx.x == 0) {
      if (o) atomicAdd(&t.ctrl->overflow_vertices, o);
      if (k) atomicAdd(&t.ctrl->frame_cells, k);
      if (s_nv) atomicAdd(&t.ctrl->vertices, s_nv);
    }
  }
  if (!grid_barrier(t.ctrl, gridDim.x)) return;
  const uint32_t taken = s_taken;

  // Phase B: temporal blend of the frame's cells, tile by tile from a second
  // counter, so that CTAs whose tiles created few cells take more.
  const bool blended = TEMPORAL && a.blend;
  if (blended) {
    unsigned long long n_hovf = 0;
    for (;;) {
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned long long b = atomicAdd(&t.ctrl->blend_next, 1ull);
        s_cur = b < ntiles ? static_cast<uint32_t>(b) : ntiles;
      }
      __syncthreads();
      const uint32_t tile = s_cur;
      if (tile >= ntiles) break;
      blend_range<W, EVICT>(t, tile * static_cast<uint32_t>(kFusedTile), __ldcg(t.bcount + tile),
                            threadIdx.x, blockDim.x, a.alpha, n_hovf);
    }
    const unsigned long long h = block_sum(n_hovf);
    if (threadIdx.x == 0 && h) atomicAdd(&t.ctrl->hist_overflow, h);
    if (!grid_barrier(t.ctrl, gridDim.x)) return;
  }

  // Phase C: one lookup per vertex of this CTA's tiles.
  const bool ovec = a.ovec != 0;
  for (uint32_t k = 0; k < taken; ++k) {
    const size_t t0 = static_cast<size_t>(s_tile[k]) * kFusedTile;
    const size_t end = min(a.n, t0 + kFusedTile);
    const uint32_t* stash = a.gstash ? a.gstash + t0 : s_stash + static_cast<size_t>(k) * kFusedTile;
#pragma unroll 1
    for (int sub = 0; sub < 4; sub += W) {
      const size_t j = t0 + fused_offset<W>(sub);
      if (j < end) {
        uint32_t id[W];
#pragma unroll
        for (int q = 0; q < W; ++q) id[q] = stash[j - t0 + q];
        Result res[W];
        resolve_batch<W>(t, a.v, j, end, id, blended, res);
        store_batch<W>(a.o, j, end, ovec, res);
      }
    }
  }
  // Neighborhood search: this kernel variant only queues its low-count
  // vertices (one atomic per warp); k_neighbors then searches the whole queue
  // at full occupancy and k_clear_fused empties the cells, so that the
  // irregular searches neither unbalance the persistent CTAs nor cost the
  // persistent kernel registers.
  if constexpr (NEIGH) {
    const int lane = threadIdx.x & 31;
    for (uint32_t k = 0; k < taken; ++k) {
      const size_t t0 = static_cast<size_t>(s_tile[k]) * kFusedTile;
      const size_t end = min(a.n, t0 + kFusedTile);
      const uint32_t* stash = a.gstash ? a.gstash + t0 : s_stash + static_cast<size_t>(k) * kFusedTile;
      for (size_t base = t0 + (threadIdx.x & ~31u); base < end; base += blockDim.x) {
        const size_t j = base + lane;
        bool low = false;
        if (j < end) {
          const uint32_t id = stash[j - t0];
          low = id != kOverflowSlot &&
                value_of(t, load_value(t, id, blended), blended).n < t.lowcount;
        }
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, low);
        if (mask) {
          unsigned long long b0 = 0ull;
          if (lane == 0) b0 = atomicAdd(&t.ctrl->neigh_count, static_cast<unsigned long long>(__popc(mask)));
          b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
          if (low) a.nq[b0 + __popc(mask & ((1u << lane) - 1u))] = static_cast<uint32_t>(j);
        }
      }
    }
    return;
  }
  if (!grid_barrier(t.ctrl, gridDim.x)) return;

  // Phase D: empty the cells this CTA's tiles created (and, when many slots
  // are in use, sweep the slot table instead of clearing slot by slot).
  for (uint32_t k = 0; k < taken; ++k)
    clear_range(t, s_tile[k] * static_cast<uint32_t>(kFusedTile), s_claims[k], threadIdx.x,
                blockDim.x, a.sweep != 0);
  if (a.sweep)
    sweep_slots(t, blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x,
                static_cast<size_t>(gridDim.x) * blockDim.x);
}

// ------------------------------------------------------------------ pipelined insert
// k_fused_ws: the persistent kernel with its insert (phase A) split between
// two groups of warps that work on different chunks of vertices at once.
//
//  key warps    read a chunk's vertex streams (coalesced; two vertices per
//               thread at a time, whose keys are built together so that their
//               chains of Philox rounds and hash steps overlap), build each
//               vertex's key (Algorithm 1), merge equal keys within the
//               warp (__match_any_sync: the lowest lane of each group of equal
//               keys becomes its leader and the members add their
//               contributions to the leader's entry with shared-memory
//               atomics), and append one queue entry per distinct key:
//               {home hash, fingerprint, member lanes, first vertex of the
//               warp} and the group's sums and count.
//  probe warps  take a full chunk's entries, four per thread at a time, and
//               run the table operations of Sec. 3.2 for all four together
//               (first probes, id claims, compare-and-swaps, the rare longer
//               probes, then the accumulating reductions); each entry's cell id
//               goes to the stash word of every member vertex.
//
// Two queue buffers alternate, so the key warps fill one chunk while the
// probe warps drain the other.  The handover uses two mbarriers per buffer
// (full: every key thread arrives after writing its entries; empty: every
// probe thread arrives after reading them), waited with a bounded
// try_wait loop (about two seconds of wall time, then kErrBarrierTimeout and
// the launch ends like a timed-out grid barrier).  The key warps decide
// together whether to go on (a named-barrier AND vote), so none of them is
// left waiting at a barrier.  The stash is the global one (indexed by
// vertex); phases B, C and D are those of k_fused.  Cell records, stash words
// and history cells are written and read with an evict-first L2 policy, so
// that the slot index and the accumulators stay in L2.
constexpr int kWsChunk = 1024;  // vertices per queue chunk: half a tile
constexpr int kWsChunksPerTile = kFusedTile / kWsChunk;
constexpr uint32_t kWsEnd = 0xFFFFFFFFu;  // chunk header: no more tiles

struct WsHeader {
  uint32_t count;  // entries in the chunk
  uint32_t k;      // the tile's place in this CTA's tile list
  uint32_t tile;   // the tile, or kWsEnd
};

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(m))),
               "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* m) {
  unsigned long long state;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];"
               : "=l"(state)
               : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(m)))
               : "memory");
  (void)state;
}

// Wait for the phase of parity `parity` of mbarrier m to complete, for about
// `limit_ns` of wall time at most; false when the wait gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m, uint32_t parity,
                                                  unsigned long long limit_ns = 2000000000ull) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(m));
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// AND of `pred` over the `nthreads` threads that use named barrier `id`.
__device__ __forceinline__ bool bar_and(int id, int nthreads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
      " bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(pred ? 1u : 0u), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

// Shared-memory layout of k_fused_ws (dynamic part): 2 headers, 4 mbarriers
// (full[2], empty[2]), two queue buffers of kWsChunk entries and their FP32
// group sums {r, g, b, count} (fixed-point tables leave the sums to the probe
// warps, which add the members' contributions exactly in int64).
struct WsLayout {
  static constexpr size_t kHeaders = 64;
  __host__ __device__ static constexpr size_t keys_off() { return kHeaders; }
  __host__ __device__ static constexpr size_t sums_off() {
    return kHeaders + 2 * kWsChunk * sizeof(uint4);
  }
  __host__ __device__ static constexpr size_t sum_words(bool) { return 1; }
  __host__ __device__ static constexpr size_t bytes(bool fixed) {
    return sums_off() + 2 * kWsChunk * sum_words(fixed) * sizeof(float4);
  }
};

// Append the queue entry of vertex j (valid) of this warp's lanes `vm` (the
// valid lanes are consecutive vertices): merge equal keys among the warp's
// lanes (the lowest lane of a group leads, the others add their contributions
// to its entry), one entry per group.  `merge`: 1 no merging (every lane its
// own group); 2 merge only when two neighbouring lanes hold equal keys, which
// one shuffle and a vote find (coherent primary hits repeat keys across
// neighbouring pixels, secondary bounces rarely repeat one within a warp, and
// there the match costs more than the probes it saves); 3 always merge.
__device__ __forceinline__ void ws_enqueue(const TableDev& t, uint4* keys, float4* sums, WsHeader* h,
                                           unsigned vm, const Key& k, size_t j, float r, float g,
                                           float b, int merge) {
  const uint32_t lane = threadIdx.x & 31;
  const unsigned long long kk = (static_cast<unsigned long long>(k.h1) << 32) | k.fp;
  bool match = merge == 3;
  if (merge == 2) {
    const unsigned long long up = __shfl_up_sync(vm, kk, 1);
    match = __ballot_sync(vm, lane > 0 && up == kk) != 0u;
  }
  const unsigned grp = match ? __match_any_sync(vm, kk) : 1u << lane;
  const uint32_t leader = __ffs(grp) - 1;
  const bool lead = leader == lane;
  const unsigned lm = __ballot_sync(vm, lead);
  const uint32_t first = __ffs(vm) - 1;
  uint32_t e = 0;
  if (lane == first) e = atomicAdd(&h->count, static_cast<uint32_t>(__popc(lm)));
  e = __shfl_sync(vm, e, first) + __popc(lm & ((1u << lane) - 1u));
  e = __shfl_sync(vm, e, leader);
  if (lead) {
    keys[e] = make_uint4(k.h1, k.fp, grp, static_cast<uint32_t>(j - lane));
    if (!t.fixed)
      sums[e] = make_float4(r, g, b, __uint_as_float(static_cast<uint32_t>(__popc(grp))));
  }
  // fixed point: the probe warps sum the members exactly; no match: every lane leads
  if (t.fixed || !match) return;
  __syncwarp(vm);
  if (!lead) {
    atomicAdd(&sums[e].x, r);
    atomicAdd(&sums[e].y, g);
    atomicAdd(&sums[e].z, b);
  }
}

// The key warps' work on one chunk [c0, c0 + kWsChunk) of the vertices below
// `end`: KV vertices per thread at a time (KT apart, so that each warp's loads
// of a stream are one coalesced run), their keys built together so that the
// independent chains of Philox rounds and hash steps overlap.
template <int KEYW, int KV>
__device__ __forceinline__ void ws_key_chunk(const FusedArgs& a, uint4* keys, float4* sums,
                                             WsHeader* h, size_t c0, size_t end) {
  const TableDev& t = a.t;
  const VertexPtrs& v = a.v;
  constexpr int KT = KEYW * 32;
  const size_t cend = min(end, c0 + kWsChunk);
#pragma unroll 1
  for (size_t base = c0 + threadIdx.x; base < c0 + kWsChunk; base += KV * KT) {
    float px[KV], py[KV], pz[KV], nx[KV], ny[KV], nz[KV], r[KV], g[KV], b[KV];
#pragma unroll
    for (int q = 0; q < KV; ++q) {
      const size_t j = base + q * KT;
      const bool ok = j < cend;
      px[q] = ok ? __ldcs(v.px + j) : 0.f;
      py[q] = ok ? __ldcs(v.py + j) : 0.f;
      pz[q] = ok ? __ldcs(v.pz + j) : 0.f;
      nx[q] = ok ? __ldcs(v.nx + j) : 0.f;
      ny[q] = ok ? __ldcs(v.ny + j) : 0.f;
      nz[q] = ok ? __ldcs(v.nz + j) : 1.f;
      const bool rgb = ok && !t.fixed;  // fixed point: summed by the probe warps
      r[q] = rgb ? __ldcs(v.r + j) : 0.f;
      g[q] = rgb ? __ldcs(v.g + j) : 0.f;
      b[q] = rgb ? __ldcs(v.b + j) : 0.f;
    }
    Key k[KV];
#pragma unroll
    for (int q = 0; q < KV; ++q) {
      const size_t j = base + q * KT;
      k[q] = vertex_key(a.kc, px[q], py[q], pz[q], nx[q], ny[q], nz[q],
                        j < cend ? vertex_id(v, j) : 0u, v.stream_id);
    }
#pragma unroll
    for (int q = 0; q < KV; ++q) {
      const size_t j = base + q * KT;
      const bool valid = j < cend;
      const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
      if (valid) ws_enqueue(t, keys, sums, h, vm, k[q], j, r[q], g[q], b[q], a.merge);
    }
  }
}

// One probe thread's entries e0, e0 + stride, ... (at most 4) of a chunk:
// the table operations of all of them together.
template <int PB>
__device__ __forceinline__ void ws_probe_group(const TableDev& t, const VertexPtrs& v,
                                               const uint4* keys,
                                               const float4* sums, uint32_t q, uint32_t e0,
                                               uint32_t stride, uint32_t id_base,
                                               uint32_t* claims, uint32_t* gstash, bool rec,
                                               Counters& cnt) {
  uint32_t h1[PB], f[PB], mask[PB], vb[PB];
  bool use[PB];
#pragma unroll
  for (int i = 0; i < PB; ++i) {
    const uint32_t e = e0 + i * stride;
    use[i] = e < q;
    const uint4 kq = use[i] ? keys[e] : make_uint4(0u, 0u, 0u, 0u);
    h1[i] = kq.x;
    f[i] = kq.y;
    mask[i] = kq.z;
    vb[i] = kq.w;
  }
  unsigned long long w[PB];
#pragma unroll
  for (int i = 0; i < PB; ++i) w[i] = use[i] ? ld_relaxed_u64_keep(t.slots + (h1[i] & t.mask)) : 1ull;
  // ids for the entries whose first probe found an empty slot: one
  // shared-memory atomic per warp, the lanes' ids in (entry, lane) order
  uint32_t my[PB];
  {
    // the lanes of this warp in this call: those whose first entry is below q
    const uint32_t lane = threadIdx.x & 31u, lt = (1u << lane) - 1u;
    const uint32_t e_lane0 = e0 - lane;
    const uint32_t nin = q > e_lane0 ? min(32u, q - e_lane0) : 0u;
    const unsigned am = nin >= 32u ? 0xFFFFFFFFu : (1u << nin) - 1u;
    unsigned bm[PB];
    uint32_t tot = 0;
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      bm[i] = __ballot_sync(am, use[i] && w[i] == 0ull);
      tot += __popc(bm[i]);
    }
    const uint32_t first = __ffs(am) - 1u;
    uint32_t base = 0;
    if (lane == first && tot) base = atomicAdd(claims, tot);
    base = __shfl_sync(am, base, first);
    uint32_t off = 0;
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      my[i] = (bm[i] >> lane) & 1u ? id_base + base + off + __popc(bm[i] & lt) : kOverflowSlot;
      off += __popc(bm[i]);
    }
  }
  unsigned long long old[PB];
#pragma unroll
  for (int i = 0; i < PB; ++i)
    old[i] = my[i] != kOverflowSlot
                 ? atomicCAS(t.slots + (h1[i] & t.mask), 0ull, slot_word(f[i], my[i]))
                 : w[i];
  uint32_t id[PB];
#pragma unroll
  for (int i = 0; i < PB; ++i) {
    id[i] = kOverflowSlot;
    if (!use[i]) continue;
    const uint32_t home = h1[i] & t.mask;
    uint32_t slot = home;
    bool claimed = false;
    if (my[i] != kOverflowSlot && old[i] == 0ull) {
      id[i] = my[i];
      claimed = true;
    } else if (slot_fp(old[i]) == f[i]) {
      id[i] = slot_id(old[i]);
    } else {
      const MoreProbe m = probe_more(t.slots, t.mask, t.max_probes, home, f[i], my[i], id_base,
                                     claims);
      slot = m.slot;
      id[i] = m.id;
      my[i] = m.my;
      claimed = m.claimed;
    }
    if (rec && my[i] != kOverflowSlot)
      st_once_u4(t.info + my[i], claimed ? make_uint4(slot, h1[i], f[i], kOverflowSlot)
                                         : make_uint4(kNoSlot, 0u, 0u, kOverflowSlot));
    cnt.cells += claimed ? 1u : 0u;
  }
#pragma unroll
  for (int i = 0; i < PB; ++i) {
    if (!use[i]) continue;
    const uint32_t e = e0 + i * stride;
    if (id[i] != kOverflowSlot) {
      if (!t.fixed) {
        const float4 s = sums[e];
        red_add_v4_keep(t.acc + id[i], s.x, s.y, s.z, static_cast<float>(__float_as_uint(s.w)));
      } else {
        // exact int64 sums of the members' fixed-point contributions
        long long fr = 0, fg = 0, fb = 0;
        for (uint32_t m = mask[i]; m; m &= m - 1u) {
          const uint32_t j = vb[i] + __ffs(m) - 1;
          fr += to_fixed(__ldg(v.r + j));
          fg += to_fixed(__ldg(v.g + j));
          fb += to_fixed(__ldg(v.b + j));
        }
        accumulate(t, id[i], 0.f, 0.f, 0.f, fr, fg, fb, __popc(mask[i]));
      }
    } else {
      cnt.ovf += __popc(mask[i]);
    }
    for (uint32_t m = mask[i]; m; m &= m - 1u) st_once_u32(gstash + vb[i] + __ffs(m) - 1, id[i]);
  }
}

template <bool TEMPORAL, int KEYW, int PRW, int KV>
__global__ void __launch_bounds__((KEYW + PRW) * 32, 2) k_fused_ws(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ uint32_t s_tile[kMaxTilesPerCta];
  __shared__ uint32_t s_claims[kMaxTilesPerCta];
  __shared__ uint32_t s_cur, s_taken;
  constexpr int KT = KEYW * 32, PT = PRW * 32;
  const TableDev& t = a.t;
  const uint32_t ntiles = static_cast<uint32_t>((a.n + kFusedTile - 1) / kFusedTile);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(s_dyn);
  uint64_t* full = reinterpret_cast<uint64_t*>(s_dyn + 32);
  uint64_t* empty = full + 2;
  uint4* keys = reinterpret_cast<uint4*>(s_dyn + WsLayout::keys_off());
  float4* sums = reinterpret_cast<float4*>(s_dyn + WsLayout::sums_off());
  const size_t sw = WsLayout::sum_words(t.fixed != 0);
  if (threadIdx.x == 0) {
    s_taken = 0;
    for (int b = 0; b < 2; ++b) {
      mbar_init(full + b, KT);
      mbar_init(empty + b, PT);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // Phase A: key warps and probe warps on alternate chunks.
  Counters c;
  unsigned long long nv = 0;  // vertices of this CTA's tiles (key thread 0)
  bool ok = true;
  if (threadIdx.x < KT) {
    uint32_t tile = 0, k = 0;
    for (uint32_t ch = 0;; ++ch) {
      const uint32_t bsel = ch & 1u;
      bool go = true;
      if (ch >= 2) go = mbar_wait_bounded(empty + bsel, ((ch >> 1) + 1u) & 1u);
      if (threadIdx.x == 0 && go) {
        if (ch % kWsChunksPerTile == 0) {
          tile = s_taken < a.cap_tiles ? claim_tile(t.ctrl, ntiles, true) : ntiles;
          if (tile < ntiles) {
            k = s_taken;
            s_tile[k] = tile;
            s_claims[k] = 0;
            s_taken = k + 1;
            nv += min(a.n, static_cast<size_t>(tile) * kFusedTile + kFusedTile) -
                  static_cast<size_t>(tile) * kFusedTile;
          }
        }
        hdr[bsel].count = 0;
        hdr[bsel].k = k;
        hdr[bsel].tile = tile < ntiles ? tile : kWsEnd;
      }
      go = bar_and(1, KT, go);  // also publishes the header to the key warps
      if (!go) {
        ok = false;
        break;
      }
      // this buffer's header is rewritten only after the probe warps have
      // released it, which needs every key thread's arrival for this chunk
      const uint32_t cur = hdr[bsel].tile;
      if (cur != kWsEnd) {
        const size_t t0 = static_cast<size_t>(cur) * kFusedTile;
        ws_key_chunk<KEYW, KV>(a, keys + bsel * kWsChunk, sums + bsel * kWsChunk * sw, hdr + bsel,
                           t0 + (ch % kWsChunksPerTile) * kWsChunk, min(a.n, t0 + kFusedTile));
      }
      mbar_arrive(full + bsel);
      if (cur == kWsEnd) break;
    }
  } else {
    const uint32_t pt = threadIdx.x - KT;
    const bool rec = (TEMPORAL && a.blend) || !a.sweep;
    for (uint32_t ch = 0;; ++ch) {
      const uint32_t bsel = ch & 1u;
      if (!mbar_wait_bounded(full + bsel, (ch >> 1) & 1u)) {
        ok = false;
        break;
      }
      const WsHeader hh = hdr[bsel];
      if (hh.tile == kWsEnd) break;
      const uint32_t id_base = hh.tile * static_cast<uint32_t>(kFusedTile);
      const uint4* kq = keys + bsel * kWsChunk;
      const float4* sq = sums + bsel * kWsChunk * sw;
#pragma unroll 1
      for (uint32_t e0 = pt; e0 < hh.count; e0 += 4 * PT)
        ws_probe_group<4>(t, a.v, kq, sq, hh.count, e0, PT, id_base, &s_claims[hh.k], a.gstash, rec,
                          c);
      mbar_arrive(empty + bsel);
    }
  }
  if (!ok) atomicOr(&t.ctrl->error, kErrBarrierTimeout);
  __syncthreads();
  const uint32_t taken = s_taken;
  {
    const unsigned long long o = block_sum(static_cast<unsigned long long>(c.ovf));
    const unsigned long long kk = block_sum(static_cast<unsigned long long>(c.cells));
    if (threadIdx.x == 0) {
      if (o) atomicAdd(&t.ctrl->overflow_vertices, o);
      if (kk) atomicAdd(&t.ctrl->frame_cells, kk);
      if (nv) atomicAdd(&t.ctrl->vertices, nv);
      if (TEMPORAL && a.blend)
        for (uint32_t i = 0; i < taken; ++i) __stcg(t.bcount + s_tile[i], s_claims[i]);
    }
  }
  if (!grid_barrier(t.ctrl, gridDim.x)) return;

  // Phase B: temporal blend, tiles from the second counter (as k_fused).
  const bool blended = TEMPORAL && a.blend;
  if (blended) {
    unsigned long long n_hovf = 0;
    for (;;) {
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned long long bb = atomicAdd(&t.ctrl->blend_next, 1ull);
        s_cur = bb < ntiles ? static_cast<uint32_t>(bb) : ntiles;
      }
      __syncthreads();
      const uint32_t tile = s_cur;
      if (tile >= ntiles) break;
      blend_range<2, false>(t, tile * static_cast<uint32_t>(kFusedTile), __ldcg(t.bcount + tile),
                            threadIdx.x, blockDim.x, a.alpha, n_hovf);
    }
    const unsigned long long hs = block_sum(n_hovf);
    if (threadIdx.x == 0 && hs) atomicAdd(&t.ctrl->hist_overflow, hs);
    if (!grid_barrier(t.ctrl, gridDim.x)) return;
  }

  // Phase C: one lookup per vertex of this CTA's tiles (cell ids from the stash).
  const bool ovec = a.ovec != 0;
  for (uint32_t k = 0; k < taken; ++k) {
    const size_t t0 = static_cast<size_t>(s_tile[k]) * kFusedTile;
    const size_t end = min(a.n, t0 + kFusedTile);
#pragma unroll 1
    for (int sub = 0; sub < 4; sub += 2) {
      const size_t j = t0 + fused_offset<2>(sub);
      if (j < end) {
        uint32_t id[2];
        if (j + 2 <= end) {  // j is even and the stash 8-byte aligned
          const uint2 w2 = __ldcs(reinterpret_cast<const uint2*>(a.gstash + j));
          id[0] = w2.x;
          id[1] = w2.y;
        } else {
          id[0] = __ldcs(a.gstash + j);
          id[1] = kOverflowSlot;
        }
        Result res[2];
        resolve_batch<2>(t, a.v, j, end, id, blended, res);
        store_batch<2>(a.o, j, end, ovec, res);
      }
    }
  }
  if (!grid_barrier(t.ctrl, gridDim.x)) return;

  // Phase D: empty the cells this CTA's tiles created.
  for (uint32_t k = 0; k < taken; ++k)
    clear_range(t, s_tile[k] * static_cast<uint32_t>(kFusedTile), s_claims[k], threadIdx.x,
                blockDim.x, a.sweep != 0);
  if (a.sweep)
    sweep_slots(t, blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x,
                static_cast<size_t>(gridDim.x) * blockDim.x);
}

// The batched persistent kernel: the same phases as k_fused over the tiles of
// several views, each with its own table.  Tiles are numbered across views
// (view v owns tiles [tile_base, tile_base + ntiles)) and handed out from one
// counter; a CTA copies the descriptor of the view of each tile it takes into
// shared memory and remembers (view, tile) for the later phases.
struct MultiArgs {
  const ViewDesc* views;
  Ctrl* ctrl;  // grid barrier and tile counter of the batch
  uint32_t* gstash;
  uint32_t nviews, total_tiles, cap_tiles;
  float alpha;
};

__device__ __forceinline__ void copy_view(ViewDesc* dst, const ViewDesc* src) {
  const int words = static_cast<int>(sizeof(ViewDesc) / sizeof(uint32_t));
  for (int i = threadIdx.x; i < words; i += blockDim.x)
    reinterpret_cast<uint32_t*>(dst)[i] = reinterpret_cast<const uint32_t*>(src)[i];
}

template <bool TEMPORAL, int W, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (W == 4 ? 1 : 2) * (kFusedBlock / BLOCK)) k_fused_multi(MultiArgs a) {
  constexpr int kPer = kFusedTile / BLOCK;  // vertices per thread per tile
  extern __shared__ __align__(16) uint32_t s_stash[];
  __shared__ uint32_t s_tile[kMaxTilesPerCta];
  __shared__ uint32_t s_claims[kMaxTilesPerCta];
  __shared__ uint16_t s_view[kMaxTilesPerCta];
  __shared__ __align__(16) ViewDesc s_vd;
  __shared__ uint32_t s_next, s_taken;
  __shared__ unsigned long long s_ovf, s_cells;
  if (threadIdx.x == 0) s_taken = 0;

  // Phase A: keys, probing insert, accumulation, tile by tile across views.
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t gt = a.total_tiles;
      if (s_taken < a.cap_tiles) gt = static_cast<uint32_t>(atomicAdd(&a.ctrl->tile_next, 1ull));
      s_next = gt;
      if (gt < a.total_tiles) {
        uint32_t v = 0;
        while (v + 1 < a.nviews && a.views[v + 1].tile_base <= gt) ++v;
        s_view[s_taken] = static_cast<uint16_t>(v);
        s_tile[s_taken] = gt - a.views[v].tile_base;
        s_claims[s_taken] = 0;
      }
      s_ovf = 0;
      s_cells = 0;
    }
    __syncthreads();
    const uint32_t gt = s_next;
    if (gt >= a.total_tiles) break;
    const uint32_t k = s_taken;
    copy_view(&s_vd, a.views + s_view[k]);
    __syncthreads();
    const size_t t0 = static_cast<size_t>(s_tile[k]) * kFusedTile;
    const size_t end = min(static_cast<size_t>(s_vd.n), t0 + kFusedTile);
    uint32_t* stash = a.gstash ? a.gstash + static_cast<size_t>(gt) * kFusedTile
                               : s_stash + static_cast<size_t>(k) * kFusedTile;
    Counters c;
#pragma unroll 1
    for (int sub = 0; sub < kPer; sub += W) {
      const size_t j = t0 + fused_offset<W, BLOCK>(sub);
      if (j < end) {
        const Batch<W> b = insert_batch<W>(s_vd.kc, s_vd.t, s_vd.v, j, end, s_vd.vec != 0,
                                           static_cast<uint32_t>(t0), &s_claims[k], c);
#pragma unroll
        for (int q = 0; q < W; ++q) stash[j - t0 + q] = b.id[q];
      }
    }
    // per-view counters of this tile
    unsigned long long o = c.ovf, cl = c.cells;
    for (int off = 16; off > 0; off >>= 1) {
      o += __shfl_xor_sync(0xFFFFFFFFu, o, off);
      cl += __shfl_xor_sync(0xFFFFFFFFu, cl, off);
    }
    if ((threadIdx.x & 31) == 0) {
      if (o) atomicAdd(&s_ovf, o);
      if (cl) atomicAdd(&s_cells, cl);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_ovf) atomicAdd(&s_vd.t.ctrl->overflow_vertices, s_ovf);
      if (s_cells) atomicAdd(&s_vd.t.ctrl->frame_cells, s_cells);
      atomicAdd(&s_vd.t.ctrl->vertices, static_cast<unsigned long long>(end - t0));
      ++s_taken;
    }
  }
  if (!grid_barrier(a.ctrl, gridDim.x)) return;
  const uint32_t taken = s_taken;

  // Phase B: temporal blend of the cells this CTA's tiles created.
  if (TEMPORAL) {
    for (uint32_t k = 0; k < taken; ++k) {
      __syncthreads();
      copy_view(&s_vd, a.views + s_view[k]);
      __syncthreads();
      if (!s_vd.blended) continue;
      unsigned long long n_hovf = 0;
      blend_range<W, false>(s_vd.t, s_tile[k] * static_cast<uint32_t>(kFusedTile), s_claims[k],
                     threadIdx.x, blockDim.x, a.alpha, n_hovf);
      if (n_hovf) atomicAdd(&s_vd.t.ctrl->hist_overflow, n_hovf);
    }
    if (!grid_barrier(a.ctrl, gridDim.x)) return;
  }

  // Phase C: one lookup per vertex of this CTA's tiles.
  for (uint32_t k = 0; k < taken; ++k) {
    __syncthreads();
    copy_view(&s_vd, a.views + s_view[k]);
    __syncthreads();
    const size_t t0 = static_cast<size_t>(s_tile[k]) * kFusedTile;
    const size_t end = min(static_cast<size_t>(s_vd.n), t0 + kFusedTile);
    const size_t gt = static_cast<size_t>(s_vd.tile_base) + s_tile[k];
    const uint32_t* stash = a.gstash ? a.gstash + gt * kFusedTile
                                     : s_stash + static_cast<size_t>(k) * kFusedTile;
    const bool blended = TEMPORAL && s_vd.blended;
#pragma unroll 1
    for (int sub = 0; sub < kPer; sub += W) {
      const size_t j = t0 + fused_offset<W, BLOCK>(sub);
      if (j < end) {
        uint32_t id[W];
#pragma unroll
        for (int q = 0; q < W; ++q) id[q] = stash[j - t0 + q];
        Result res[W];
        resolve_batch<W>(s_vd.t, s_vd.v, j, end, id, blended, res);
        store_batch<W>(s_vd.o, j, end, s_vd.ovec != 0, res);
      }
    }
  }
  if (!grid_barrier(a.ctrl, gridDim.x)) return;

  // Phase D: empty the cells this CTA's tiles created; sweep the slot tables
  // of the views that are swept.
  for (uint32_t k = 0; k < taken; ++k) {
    __syncthreads();
    copy_view(&s_vd, a.views + s_view[k]);
    __syncthreads();
    clear_range(s_vd.t, s_tile[k] * static_cast<uint32_t>(kFusedTile), s_claims[k], threadIdx.x,
                blockDim.x, s_vd.sweep != 0);
  }
  for (uint32_t v = 0; v < a.nviews; ++v) {
    __syncthreads();
    copy_view(&s_vd, a.views + v);
    __syncthreads();
    if (s_vd.sweep)
      sweep_slots(s_vd.t, blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x,
                  static_cast<size_t>(gridDim.x) * blockDim.x);
  }
}

int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    cached = c > 0 ? c : 1;
  }
  return cached;
}

int split_grid(size_t work_items) {
  const size_t want = (work_items + kBlock - 1) / kBlock;
  const size_t cap = static_cast<size_t>(sm_count()) * 8;
  return static_cast<int>(std::max<size_t>(1, std::min(want, cap)));
}

}  // namespace

int tile_size() { return kTile; }
int fused_tile_size() { return kFusedTile; }

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
                          uint32_t* id_out, uint32_t tile_base, int batch, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int grid = split_grid((n + 3) / 4);
  const int vec = vec_inputs(v) ? 1 : 0;
  if (t.hist_migrate || t.normal_search) {  // keep each new cell's quantized key
    if (batch == 2)
      k_insert<2, true><<<grid, kBlock, 0, st>>>(kc, t, v, n, id_out, vec, tile_base);
    else
      k_insert<4, true><<<grid, kBlock, 0, st>>>(kc, t, v, n, id_out, vec, tile_base);
  } else if (batch == 2) {
    k_insert<2, false><<<grid, kBlock, 0, st>>>(kc, t, v, n, id_out, vec, tile_base);
  } else {
    k_insert<4, false><<<grid, kBlock, 0, st>>>(kc, t, v, n, id_out, vec, tile_base);
  }
  return cudaGetLastError();
}

cudaError_t launch_query(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                         const uint32_t* id_in, const OutPtrs& o, bool blended, uint32_t id_limit,
                         cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_query<<<split_grid((n + 3) / 4), kBlock, 0, st>>>(kc, t, v, n, id_in, o,
                                                      vec_inputs(v) ? 1 : 0,
                                                      vec_outputs(o) ? 1 : 0, blended ? 1 : 0,
                                                      id_limit);
  return cudaGetLastError();
}

cudaError_t launch_keys(const KeyConst& kc, const VertexPtrs& v, size_t n, uint32_t* h_out,
                        uint32_t* f_out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_keys<<<split_grid(n), kBlock, 0, st>>>(kc, v, n, h_out, f_out);
  return cudaGetLastError();
}

cudaError_t launch_blend(const KeyConst& kc, const TableDev& t, uint32_t ntiles, float alpha,
                         cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  const uint32_t grid = std::min<uint32_t>(ntiles, static_cast<uint32_t>(sm_count()) * 8);
  if (t.hist_migrate) {
    k_blend_lookup<<<grid, kBlock, 0, st>>>(kc, t, ntiles);
    k_blend_apply<<<grid, kBlock, 0, st>>>(t, ntiles, alpha);
  } else {
    k_blend_sweep<<<grid, kBlock, 0, st>>>(t, ntiles, alpha);
  }
  return cudaGetLastError();
}

// Sweeping the slot table pays once the frame's vertices reach an eighth of it.
static bool sweep_pays(const TableDev& t, size_t vertices) {
  return vertices >= (static_cast<size_t>(t.mask) + 1) / 8;
}

cudaError_t launch_clear(const TableDev& t, uint32_t ntiles, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  const int sweep = sweep_pays(t, static_cast<size_t>(ntiles) * kTile) ? 1 : 0;
  const uint32_t grid = std::min<uint32_t>(std::max<uint32_t>(ntiles, sweep ? 1u << 30 : 0u),
                                           static_cast<uint32_t>(sm_count()) * 8);
  k_clear_sweep<<<grid, kBlock, 0, st>>>(t, ntiles, sweep);
  return cudaGetLastError();
}

// Evicting history: when the per-table epoch runs out, every entry's
// priority drops by `by` (at least 1 remains), keeping the order of recent
// entries.
__global__ void __launch_bounds__(kBlock) k_hist_age(TableDev t, uint32_t by) {
  const size_t Th = static_cast<size_t>(t.hmask) + 1;
  for (size_t h = blockIdx.x * (size_t)blockDim.x + threadIdx.x; h < Th;
       h += (size_t)gridDim.x * blockDim.x) {
    uint32_t* fp = hist_fp(t, static_cast<uint32_t>(h));
    const uint32_t w = *fp;
    if (w == 0u) continue;
    const uint32_t r = w >> 24;
    *fp = ((r > by ? r - by : 1u) << 24) | (w & 0xFFFFFFu);
  }
}

cudaError_t launch_hist_age(const TableDev& t, uint32_t by, cudaStream_t st) {
  k_hist_age<<<sm_count() * 8, kBlock, 0, st>>>(t, by);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock) k_combine_coarse(size_t n, const uint8_t* fine_status,
                                                           OutPtrs c, OutPtrs o) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n;
       j += (size_t)gridDim.x * blockDim.x) {
    if (fine_status[j] != 1 || c.status[j] == 2) continue;
    o.r[j] = c.r[j];
    o.g[j] = c.g[j];
    o.b[j] = c.b[j];
    if (o.count) o.count[j] = c.count[j];
    if (o.status) o.status[j] = 4;  // PPS_STATUS_COARSE
  }
}

cudaError_t launch_combine_coarse(size_t n, const uint8_t* fine_status, const OutPtrs& coarse,
                                  const OutPtrs& o, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = std::min<size_t>((n + kBlock - 1) / kBlock, static_cast<size_t>(sm_count()) * 8);
  k_combine_coarse<<<static_cast<unsigned>(blocks), kBlock, 0, st>>>(n, fine_status, coarse, o);
  return cudaGetLastError();
}

cudaError_t launch_count_nonzero(const void* base, uint32_t stride, uint32_t off, uint32_t width,
                                 uint64_t n, unsigned long long* out, cudaStream_t st) {
  k_count_nonzero<<<sm_count() * 4, kBlock, 0, st>>>(static_cast<const unsigned char*>(base),
                                                     stride, off, width, n, out);
  return cudaGetLastError();
}

template <bool TEMPORAL, bool EVICT, bool NEIGH>
static const void* fused_fn(int batch) {
  return batch == 2 ? reinterpret_cast<const void*>(k_fused<TEMPORAL, 2, EVICT, NEIGH>)
                    : reinterpret_cast<const void*>(k_fused<TEMPORAL, 4, EVICT, NEIGH>);
}

// The kernel for a frame: with or without a history, an evicting one or not,
// with or without the neighborhood search.
static const void* fused_kernel(bool temporal, int batch, bool evict, bool neigh) {
  if (temporal && evict)
    return neigh ? fused_fn<true, true, true>(batch) : fused_fn<true, true, false>(batch);
  if (temporal) return neigh ? fused_fn<true, false, true>(batch) : fused_fn<true, false, false>(batch);
  return neigh ? fused_fn<false, false, true>(batch) : fused_fn<false, false, false>(batch);
}

// Largest dynamic shared memory a k_fused CTA may request: the opt-in limit
// per block minus the kernel's static shared memory (set once per kernel).
static cudaError_t fused_dyn_smem_limit(const void* fn, size_t* limit) {
  static const void* done[32] = {nullptr};
  static size_t lims[32] = {0};
  for (int i = 0; i < 32; ++i)
    if (done[i] == fn) {
      *limit = lims[i];
      return cudaSuccess;
    }
  int dev = 0, maxopt = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  const size_t lim = static_cast<size_t>(maxopt) - fa.sharedSizeBytes;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(lim));
  if (e != cudaSuccess) return e;
  for (int i = 0; i < 32; ++i)
    if (!done[i]) {
      done[i] = fn;
      lims[i] = lim;
      break;
    }
  *limit = lim;
  return cudaSuccess;
}

template <bool TEMPORAL>
static const void* ws_fn(int key_warps) {
  if (key_warps == 4) return reinterpret_cast<const void*>(k_fused_ws<TEMPORAL, 4, 12, 2>);
  if (key_warps == 12) return reinterpret_cast<const void*>(k_fused_ws<TEMPORAL, 12, 4, 2>);
  return reinterpret_cast<const void*>(k_fused_ws<TEMPORAL, 8, 8, 2>);
}

static const void* ws_kernel(bool temporal, int key_warps) {
  return temporal ? ws_fn<true>(key_warps) : ws_fn<false>(key_warps);
}

// The pipelined insert: two CTAs of 512 threads per SM when their queues fit
// (one otherwise); the stash is the global one.
static cudaError_t plan_ws(size_t n, bool temporal, int key_warps, bool fixed, FusedPlan* plan) {
  const void* fn = ws_kernel(temporal, key_warps);
  size_t maxdyn = 0;
  cudaError_t e = fused_dyn_smem_limit(fn, &maxdyn);
  if (e != cudaSuccess) return e;
  const size_t smem = WsLayout::bytes(fixed);
  if (smem > maxdyn) return cudaErrorInvalidConfiguration;
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kFusedBlock, smem);
  if (e != cudaSuccess) return e;
  if (nb < 1) return cudaErrorInvalidConfiguration;
  plan->grid = sm_count() * std::min(nb, 2);
  plan->block = kFusedBlock;
  plan->batch = 2;
  plan->cap_tiles = kMaxTilesPerCta;
  plan->smem = smem;
  plan->global_stash = true;
  plan->evict = false;
  plan->neigh = false;
  plan->key_warps = key_warps;
  const size_t ntiles = (n + kFusedTile - 1) / kFusedTile;
  if (static_cast<size_t>(plan->grid) * kMaxTilesPerCta < ntiles) return cudaErrorInvalidValue;
  return cudaSuccess;
}

cudaError_t plan_fused(size_t n, bool temporal, int batch, FusedPlan* plan, bool evict,
                       bool neigh, InsertShape shape, bool fixed) {
  plan->key_warps = 0;
  if (shape.pipelined && !evict && !neigh) {
    const int kw = shape.key_warps == 4 || shape.key_warps == 12 ? shape.key_warps : 8;
    plan->merge = shape.merge;
    return plan_ws(n, temporal, kw, fixed, plan);
  }
  const void* fn = fused_kernel(temporal, batch, evict, neigh);
  plan->evict = temporal && evict;
  plan->neigh = neigh;
  const int sms = sm_count();
  size_t maxdyn = 0;
  cudaError_t e = fused_dyn_smem_limit(fn, &maxdyn);
  if (e != cudaSuccess) return e;
  int b0 = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, fn, kFusedBlock, 0);
  if (e != cudaSuccess) return e;
  if (b0 < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const size_t ntiles = (n + kFusedTile - 1) / kFusedTile;
  const size_t tile_bytes = kFusedTile * sizeof(uint32_t);
  plan->block = kFusedBlock;
  plan->batch = batch;
  for (int b = b0; b >= 1; --b) {
    // shared memory per CTA when b CTAs share an SM (static part and a reserve deducted)
    const size_t per = std::min(maxdyn, static_cast<size_t>(smem_sm) / b - 12 * 1024);
    size_t cap = std::min<size_t>(per / tile_bytes, kMaxTilesPerCta);
    // the largest stash with which b CTAs still fit on an SM
    int nb = 0;
    for (; cap > 0; --cap) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kFusedBlock, cap * tile_bytes);
      if (e != cudaSuccess) return e;
      if (nb >= b) break;
    }
    if (cap == 0 || cap * static_cast<size_t>(sms) * b < ntiles) continue;
    if (nb >= b) {
      plan->grid = sms * b;
      plan->cap_tiles = static_cast<uint32_t>(cap);
      plan->smem = cap * tile_bytes;
      plan->global_stash = false;
      return cudaSuccess;
    }
  }
  // The stash does not fit on chip: keep it in a global scratch buffer.
  plan->grid = sms * b0;
  plan->cap_tiles = kMaxTilesPerCta;
  plan->smem = 0;
  plan->global_stash = true;
  if (static_cast<size_t>(plan->grid) * kMaxTilesPerCta < ntiles) return cudaErrorInvalidValue;
  return cudaSuccess;
}

cudaError_t launch_fused(const KeyConst& kc, const TableDev& t, const VertexPtrs& v, size_t n,
                         const OutPtrs& o, bool temporal, bool blend, float alpha,
                         const FusedPlan& plan, uint32_t* gstash, uint32_t* nq, cudaStream_t st) {
  FusedArgs a;
  a.kc = kc;
  a.t = t;
  a.v = v;
  a.o = o;
  a.n = n;
  a.cap_tiles = plan.cap_tiles;
  a.gstash = plan.global_stash ? gstash : nullptr;
  a.alpha = alpha;
  a.vec = vec_inputs(v) ? 1 : 0;
  a.ovec = vec_outputs(o) ? 1 : 0;
  a.blend = blend ? 1 : 0;
  a.sweep = sweep_pays(t, n) ? 1 : 0;
  a.nq = nq;
  a.merge = plan.merge;
  void* args[] = {&a};
  if (plan.key_warps > 0)
    return cudaLaunchCooperativeKernel(ws_kernel(temporal, plan.key_warps), dim3(plan.grid),
                                       dim3(plan.block), args, plan.smem, st);
  cudaError_t e = cudaLaunchCooperativeKernel(
      fused_kernel(temporal, plan.batch, plan.evict, plan.neigh), dim3(plan.grid), dim3(plan.block),
      args, plan.smem, st);
  if (e != cudaSuccess || !plan.neigh) return e;
  // the queued neighborhood searches, then the clear the persistent kernel left
  const int sms = sm_count();
  k_neighbors<<<sms * 8, kBlock, 0, st>>>(kc, t, v, o, nq, blend ? 1 : 0);
  const uint32_t ntiles = static_cast<uint32_t>((n + kFusedTile - 1) / kFusedTile);
  k_clear_fused<<<std::min<uint32_t>(ntiles, static_cast<uint32_t>(sms) * 8), kBlock, 0, st>>>(
      t, ntiles, a.sweep);
  return cudaGetLastError();
}

bool vec_inputs_host(const VertexPtrs& v) { return vec_inputs(v); }
bool vec_outputs_host(const OutPtrs& o) { return vec_outputs(o); }
bool sweep_pays_host(const TableDev& t, size_t vertices) { return sweep_pays(t, vertices); }

template <bool TEMPORAL, int W>
static const void* multi_fn(int block) {
  return block == 256 ? reinterpret_cast<const void*>(k_fused_multi<TEMPORAL, W, 256>)
                      : reinterpret_cast<const void*>(k_fused_multi<TEMPORAL, W, 512>);
}

static const void* multi_kernel(bool temporal, int batch, int block) {
  if (temporal) return batch == 2 ? multi_fn<true, 2>(block) : multi_fn<true, 4>(block);
  return batch == 2 ? multi_fn<false, 2>(block) : multi_fn<false, 4>(block);
}

cudaError_t plan_multi(size_t total_tiles, bool temporal, int batch, int block, MultiPlan* plan) {
  block = block == 256 ? 256 : kFusedBlock;
  const void* fn = multi_kernel(temporal, batch, block);
  const int sms = sm_count();
  size_t maxdyn = 0;
  cudaError_t e = fused_dyn_smem_limit(fn, &maxdyn);
  if (e != cudaSuccess) return e;
  int b0 = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, fn, block, 0);
  if (e != cudaSuccess) return e;
  if (b0 < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const size_t tile_bytes = kFusedTile * sizeof(uint32_t);
  plan->block = block;
  plan->batch = batch;
  for (int b = b0; b >= 1; --b) {
    const size_t per = std::min(maxdyn, static_cast<size_t>(smem_sm) / b - 12 * 1024);
    const size_t cap = std::min<size_t>(per / tile_bytes, kMaxTilesPerCta);
    if (cap == 0 || cap * static_cast<size_t>(sms) * b < total_tiles) continue;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, cap * tile_bytes);
    if (e != cudaSuccess) return e;
    if (nb >= b) {
      plan->grid = sms * b;
      plan->cap_tiles = static_cast<uint32_t>(cap);
      plan->smem = cap * tile_bytes;
      plan->global_stash = false;
      return cudaSuccess;
    }
  }
  plan->grid = sms * b0;
  plan->cap_tiles = kMaxTilesPerCta;
  plan->smem = 0;
  plan->global_stash = true;
  if (static_cast<size_t>(plan->grid) * kMaxTilesPerCta < total_tiles) return cudaErrorInvalidValue;
  return cudaSuccess;
}

cudaError_t launch_multi(const ViewDesc* views, uint32_t nviews, uint32_t total_tiles, Ctrl* ctrl,
                         bool temporal, float alpha, const MultiPlan& plan, uint32_t* gstash,
                         cudaStream_t st) {
  MultiArgs a;
  a.views = views;
  a.ctrl = ctrl;
  a.gstash = plan.global_stash ? gstash : nullptr;
  a.nviews = nviews;
  a.total_tiles = total_tiles;
  a.cap_tiles = plan.cap_tiles;
  a.alpha = alpha;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(multi_kernel(temporal, plan.batch, plan.block), dim3(plan.grid),
                                     dim3(plan.block), args, plan.smem, st);
}

}  // namespace pps
