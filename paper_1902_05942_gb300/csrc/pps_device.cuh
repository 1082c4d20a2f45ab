// Device-side building blocks of the hashed path space filter (sm_103a).
//
// Key construction follows Algorithm 1; the table follows Sec. 3.2 (open
// addressing, linear probing with a step limit) and Sec. 3.2.1 (32-bit
// fingerprints, 0 = empty); accumulation is the scatter form of Sec. 3.2 (one
// atomic add per component plus a counter, Sec. 3.3.1); temporal blending is
// Sec. 3.4.1.
//
// Every floating-point step of key construction uses an explicitly rounded
// intrinsic (__fadd_rn, __fmul_rn, __fdiv_rn, __fsqrt_rn), so nothing is
// contracted into an FMA and the integer keys are reproducible bit for bit by
// any IEEE-754 implementation that performs the same operations in the same
// order.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace pps {

constexpr uint32_t kOverflowSlot = 0xFFFFFFFFu;  // slot_out value on probe overflow
constexpr uint32_t kOwnerBit = 0x80000000u;      // stash word: this vertex owns its cell
constexpr uint32_t kStashOverflow = 0x7FFFFFFFu; // stash word: probe overflow

// ---------------------------------------------------------------- parameters
struct KeyConst {
  float cam[3];
  float k;  // fl32(voxel_scale * pixel_angle)
  uint32_t seed, frame;
  uint32_t hseed_home, hseed_fp;
  uint32_t mask;  // T - 1
  uint32_t max_probes;
  int32_t lod_min, lod_max;
  uint32_t jitter, nih;  // jitter on/off, normal in home hash
  // Philox4x32-10 key of rounds 1..9 for the jitter draw (seed and frame
  // bumped by the Weyl constants; set_round_keys): the same for every vertex
  // of a frame, so the kernels read them from their parameters
  uint32_t rk0[9], rk1[9];
};

// Fill kc.rk0 / kc.rk1 from kc.seed and kc.frame; call whenever either changes.
__host__ __device__ inline void set_round_keys(KeyConst& kc) {
  uint32_t k0 = kc.seed, k1 = kc.frame;
  for (int r = 0; r < 9; ++r) {
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
    kc.rk0[r] = k0;
    kc.rk1[r] = k1;
  }
}

// Per-frame and lifetime counters plus the device error word and the state of
// the grid barrier used by the persistent filter kernel.
struct Ctrl {
  unsigned long long frame_cells;
  unsigned long long overflow_vertices;
  unsigned long long vertices;
  unsigned long long hist_overflow;
  unsigned long long tile_next;   // persistent kernel: next vertex tile to hand out
  unsigned long long blend_next;  // persistent kernel: next tile whose cells to blend
  unsigned long long neigh_count;  // persistent kernel: low-count vertices queued for the search
  unsigned int error;
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned int pad[1];
};
constexpr size_t kCtrlFrameBytes = 7 * sizeof(unsigned long long);  // reset per frame

enum : unsigned int {
  kErrBarrierTimeout = 1u,
  kErrBadSlot = 2u,
  // FP32 accumulation: a cell reached 2^24 members, past which adding 1.0f to
  // its FP32 count no longer changes it, so its count and average are not
  // exact (fixed-point accumulation counts in 64 bits and has no such limit)
  kErrCountSaturated = 4u,
};

constexpr float kExactCountLimit = 16777216.0f;  // 2^24

// Table layout.
//
// The hashed table of Sec. 3.2 holds, per slot, only the key's 32-bit
// fingerprint and the id of its cell: slot = (id + 1) << 32 | fingerprint, 0 =
// empty.  At 8 bytes a slot, a table of 2^23 slots (64 MB) stays in L2, where
// the probing compare-and-swaps run several times faster than on DRAM-backed
// lines.  The cells themselves live in dense arrays indexed by the cell id:
//   acc   {sum r, sum g, sum b, count} FP32 (16 B), or int64 sums (32 B, fixed)
//   info  {slot, home hash, fingerprint, history cell} (16 B)
//   kw    the cell's quantized key {x~x, x~y, x~z, l' & 0xFF | q(n) << 8}
//         (16 B, tables whose history follows changes of resolution)
//   hold  the old value {c r, c g, c b, N} the cell's blend starts from
//         (16 B, same tables)
// Ids are handed out per block of vertices: a CTA (or a tile of the split
// path) owns the id range [block * B, block * B + count[block]), where B is its
// vertex count, so a frame's cells occupy a few contiguous runs and the
// per-cell passes (blend, clear) are coalesced sweeps over them.
//
// History cell, FP32 (32 B): [0,16) {c r, c g, c b, N}, [16,20) fingerprint.
// History cell, FP16 (16 B): [0,8) {half r, half g, half b, uint16 N}, [8,12) fp.
// After the blend the cell's acc holds the blended value {c r, c g, c b, N}.
struct TableDev {
  unsigned long long* slots;  // [T] index of the hashed table
  float4* acc;                // [D] FP32 accumulators (FP32 mode)
  unsigned long long* acc64;  // [D][4] fixed-point accumulators (fixed mode)
  uint4* info;                // [D] {slot, h1, fingerprint, history cell}
  uint4* kw;                  // [D] quantized keys (hist_migrate)
  float4* hold;               // [D] old values of the blend (hist_migrate)
  uint32_t* bcount;           // [blocks] cells claimed per id block
  unsigned char* hcells;      // [Th] history cells (temporal tables)
  Ctrl* ctrl;
  uint32_t hstride;           // bytes per history cell: 32 or 16
  uint32_t hfp_off;           // fingerprint offset in a history cell: 16 or 8
  uint32_t mask;              // T - 1
  uint32_t hmask;             // Th - 1
  uint32_t max_probes;
  uint32_t lowcount;
  int fixed;                  // accumulation mode
  int hist_mode;              // 0 none, 1 FP32, 2 FP16
  int neighbors;              // low-count vertices take the 3x3x3 pooled average
  int hist_evict;             // history fingerprints carry a priority (evicting table)
  int hist_migrate;           // history follows changes of resolution (Sec. 3.4.2)
  uint32_t hist_rank;         // evicting table: this frame's priority (blend epoch)
  uint32_t normal_search;     // 0 off; r + 1: lookups pool the voxel's normals within r steps
};

constexpr uint32_t kNoSlot = 0xFFFFFFFFu;  // info.x of an id reserved but not used

struct VertexPtrs {
  const float *px, *py, *pz, *nx, *ny, *nz, *r, *g, *b;
  const uint32_t* id;
  uint32_t id_base;
  uint32_t stream_id;
  const float* dist;       // optional distance for the level of detail
  const uint32_t* extra;   // optional extra key word
};

struct OutPtrs {
  float *r, *g, *b;
  uint32_t* count;
  uint8_t* status;
};

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds of two 32x32->64 multiplies; the key is
// bumped by the Weyl constants between rounds.
// The first two output words of one draw, the round keys taken from the key
// constants (round 0: seed and frame; rounds 1..9: kc.rk0 / kc.rk1).
__device__ __forceinline__ uint2 philox_first2_rk(uint32_t c0, uint32_t c1, const KeyConst& kc) {
  uint32_t x0 = c0, x1 = c1, x2 = 0u, x3 = 0u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t k0 = r ? kc.rk0[r - 1] : kc.seed, k1 = r ? kc.rk1[r - 1] : kc.frame;
    const uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
    const uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
    const uint32_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
    x0 = n0;
    x1 = lo1;
    x2 = n2;
    x3 = lo0;
  }
  return make_uint2(x0, x1);
}

// ---------------------------------------------------------------- MurmurHash3_x86_32
__device__ __forceinline__ uint32_t mm_body(uint32_t h, uint32_t k) {
  k *= 0xCC9E2D51u;
  k = __funnelshift_l(k, k, 15);
  k *= 0x1B873593u;
  h ^= k;
  h = __funnelshift_l(h, h, 13);
  return h * 5u + 0xE6546B64u;
}

__device__ __forceinline__ uint32_t mm_final(uint32_t h, uint32_t nbytes) {
  h ^= nbytes;
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// ---------------------------------------------------------------- Algorithm 1
__device__ __forceinline__ float pow2_int(int l) {
  return __uint_as_float(static_cast<uint32_t>(l + 127) << 23);
}

// |p_cam - x| in FP32, one rounding per operation.
__device__ __forceinline__ float camera_distance(const KeyConst& kc, float x, float y, float z) {
  const float dx = __fsub_rn(kc.cam[0], x);
  const float dy = __fsub_rn(kc.cam[1], y);
  const float dz = __fsub_rn(kc.cam[2], z);
  return __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)));
}

// floor(log2(k * d)) from the exponent bits of the FP32 product.
__device__ __forceinline__ int level_at(const KeyConst& kc, float d) {
  const float F = __fmul_rn(kc.k, d);
  const int e = static_cast<int>((__float_as_uint(F) >> 23) & 0xFFu) - 127;
  return min(max(e, kc.lod_min), kc.lod_max);
}

// Algorithm 1's level_of_detail(|p_cam - x|).
__device__ __forceinline__ int level_of_detail(const KeyConst& kc, float x, float y, float z) {
  return level_at(kc, camera_distance(kc, x, y, z));
}

__device__ __forceinline__ int32_t quantize_coord(float v, float inv) {
  float q = floorf(__fmul_rn(v, inv));
  q = fminf(fmaxf(q, -2147483648.0f), 2147483520.0f);
  return __float2int_rz(q);
}

__device__ __forceinline__ uint32_t quantize_normal(float c) {
  float q = floorf(__fmul_rn(__fadd_rn(c, 1.0f), 128.0f));
  q = fminf(fmaxf(q, 0.0f), 255.0f);
  return static_cast<uint32_t>(q);
}

struct Key {
  uint32_t h1;  // full 32-bit home hash; the home index is h1 & (T - 1)
  uint32_t fp;
};

// The words a key is hashed from: the quantized position x~ (three int32 as
// bits), the level l', the packed quantized normal and, if given, an extra
// word.
struct KeyWords {
  uint32_t X, Y, Z, L, NQ, EX;
  bool has_ex;
};

// Where the optional per-vertex inputs of the key variants are: a distance
// for the level of detail and an extra key word of vertex j (read where they
// are used, so that a frame without them carries nothing extra).
struct KeyExtra {
  const float* dist = nullptr;
  const uint32_t* extra = nullptr;
  size_t j = 0;
};

__device__ __forceinline__ KeyExtra key_extra(const VertexPtrs& v, size_t j) {
  KeyExtra e;
  e.dist = v.dist;
  e.extra = v.extra;
  e.j = j;
  return e;
}

__device__ __forceinline__ KeyWords key_words(const KeyConst& kc, float px, float py, float pz,
                                              float nx, float ny, float nz, uint32_t id,
                                              uint32_t stream_id, const KeyExtra& ke = KeyExtra{}) {
  const int l0 = ke.dist ? level_at(kc, __ldg(ke.dist + ke.j)) : level_of_detail(kc, px, py, pz);
  float xj = px, yj = py, zj = pz;
  int l1 = l0;
  if (kc.jitter) {
    // jitter(n): a point of the tangent plane, (u, w) uniform in [-0.5, 0.5)
    const uint2 rnd = philox_first2_rk(id, stream_id, kc);
    const float u = __fsub_rn(__fmul_rn(__uint2float_rn(rnd.x >> 8), 0x1p-24f), 0.5f);
    const float w = __fsub_rn(__fmul_rn(__uint2float_rn(rnd.y >> 8), 0x1p-24f), 0.5f);
    // tangent frame after Duff et al. (JCGT 2017)
    const float s = copysignf(1.0f, nz);
    const float a = -__frcp_rn(__fadd_rn(s, nz));  // = -1 / (s + nz), correctly rounded
    const float q = __fmul_rn(__fmul_rn(nx, ny), a);
    const float tx = __fadd_rn(1.0f, __fmul_rn(s, __fmul_rn(__fmul_rn(nx, nx), a)));
    const float ty = __fmul_rn(s, q);
    const float tz = -__fmul_rn(s, nx);
    const float bx = q;
    const float by = __fadd_rn(s, __fmul_rn(__fmul_rn(ny, ny), a));
    const float bz = -ny;
    const float E = pow2_int(l0);  // voxel edge at the pre-jitter level
    xj = __fadd_rn(px, __fmul_rn(__fadd_rn(__fmul_rn(u, tx), __fmul_rn(w, bx)), E));
    yj = __fadd_rn(py, __fmul_rn(__fadd_rn(__fmul_rn(u, ty), __fmul_rn(w, by)), E));
    zj = __fadd_rn(pz, __fmul_rn(__fadd_rn(__fmul_rn(u, tz), __fmul_rn(w, bz)), E));
    l1 = ke.dist ? level_at(kc, __fadd_rn(__fsub_rn(__ldg(ke.dist + ke.j),
                                                    camera_distance(kc, px, py, pz)),
                                          camera_distance(kc, xj, yj, zj)))
                 : level_of_detail(kc, xj, yj, zj);
  }
  const float inv = pow2_int(-l1);
  KeyWords kw;
  kw.X = static_cast<uint32_t>(quantize_coord(xj, inv));
  kw.Y = static_cast<uint32_t>(quantize_coord(yj, inv));
  kw.Z = static_cast<uint32_t>(quantize_coord(zj, inv));
  kw.L = static_cast<uint32_t>(l1);
  kw.NQ = quantize_normal(nx) | (quantize_normal(ny) << 8) | (quantize_normal(nz) << 16);
  kw.has_ex = ke.extra != nullptr;
  kw.EX = kw.has_ex ? __ldg(ke.extra + ke.j) : 0u;
  return kw;
}

// hash (home) and hash2 (fingerprint, 0 remapped to 1) of the key words.
__device__ __forceinline__ Key key_hash(const KeyConst& kc, const KeyWords& kw) {
  uint32_t h = kc.hseed_home;
  h = mm_body(h, kw.X);
  h = mm_body(h, kw.Y);
  h = mm_body(h, kw.Z);
  h = mm_body(h, kw.L);
  uint32_t hbytes = 16u;
  if (kc.nih) {
    h = mm_body(h, kw.NQ);
    hbytes = 20u;
  }
  uint32_t f = kc.hseed_fp;
  f = mm_body(f, kw.X);
  f = mm_body(f, kw.Y);
  f = mm_body(f, kw.Z);
  f = mm_body(f, kw.L);
  f = mm_body(f, kw.NQ);
  uint32_t fbytes = 20u;
  if (kw.has_ex) {
    h = mm_body(h, kw.EX);
    f = mm_body(f, kw.EX);
    hbytes += 4u;
    fbytes += 4u;
  }
  h = mm_final(h, hbytes);
  f = mm_final(f, fbytes);
  return Key{h, f ? f : 1u};
}

__device__ __forceinline__ Key vertex_key(const KeyConst& kc, float px, float py, float pz,
                                          float nx, float ny, float nz, uint32_t id,
                                          uint32_t stream_id, const KeyExtra& ke = KeyExtra{}) {
  return key_hash(kc, key_words(kc, px, py, pz, nx, ny, nz, id, stream_id, ke));
}

// ---------------------------------------------------------------- memory helpers
// L2 eviction priority "evict last" for the lines the next frame touches
// again (slot index, accumulators): the vertex streams and outputs pass
// through L2 with evict-first loads and stores (.cs), these stay behind them.
__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// L2 eviction priority "evict first" for data a frame touches once and the
// next frame does not need in L2 (cell records, history cells, the stash):
// they should not push the slot index and the accumulators out.  Loads of such
// data written by other CTAs of the same launch bypass L1 (.cg).
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ uint4 ld_once_u4(const void* p) {
  uint4 v;
  asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(l2_evict_first())
               : "memory");
  return v;
}

__device__ __forceinline__ uint2 ld_once_u2(const void* p) {
  uint2 v;
  asm volatile("ld.global.cg.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
               : "=r"(v.x), "=r"(v.y)
               : "l"(p), "l"(l2_evict_first())
               : "memory");
  return v;
}

__device__ __forceinline__ void st_once_u4(void* p, uint4 v) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x),
               "r"(v.y), "r"(v.z), "r"(v.w), "l"(l2_evict_first())
               : "memory");
}

__device__ __forceinline__ void st_once_u2(void* p, uint2 v) {
  asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.x), "r"(v.y),
               "l"(l2_evict_first())
               : "memory");
}

__device__ __forceinline__ void st_once_u32(void* p, uint32_t v) {
  asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(l2_evict_first())
               : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64_keep(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.L2::cache_hint.u64 %0, [%1], %2;"
               : "=l"(v)
               : "l"(p), "l"(l2_evict_last())
               : "memory");
  return v;
}

__device__ __forceinline__ void red_add_v4_keep(float4* p, float a, float b, float c, float d) {
  asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p),
               "f"(a), "f"(b), "f"(c), "f"(d), "l"(l2_evict_last())
               : "memory");
}

__device__ __forceinline__ void st_zero16_keep(void* p) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %1, %1, %1}, %2;" ::"l"(p), "r"(0u),
               "l"(l2_evict_last())
               : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ long long to_fixed(float v) {
  return __float2ll_rn(__fmul_rn(v, 16777216.0f));  // round(v * 2^24), exact product
}

__device__ __forceinline__ unsigned long long slot_word(uint32_t f, uint32_t id) {
  return (static_cast<unsigned long long>(id + 1u) << 32) | f;
}
__device__ __forceinline__ uint32_t slot_fp(unsigned long long w) {
  return static_cast<uint32_t>(w);
}
__device__ __forceinline__ uint32_t slot_id(unsigned long long w) {
  return static_cast<uint32_t>(w >> 32) - 1u;
}

// One probe step in the hashed table (Sec. 3.2, linear probing on the
// fingerprint): `w` is the word read at the slot.  A slot holding f is a hit; an
// empty slot is claimed with one 64-bit compare-and-swap that publishes the
// fingerprint and the cell id together (so a reader never sees a fingerprint
// without its cell); a slot holding another key moves the probe on.  Words are
// only ever published, never changed, within a frame, so a key present in the
// window is met before any empty slot.
enum ProbeOutcome { kHit, kClaimed, kNext };

__device__ __forceinline__ ProbeOutcome probe_step(unsigned long long* slot, unsigned long long w,
                                                   uint32_t f, uint32_t my_id, uint32_t& id) {
  if (w != 0ull) {
    if (slot_fp(w) == f) {
      id = slot_id(w);
      return kHit;
    }
    return kNext;
  }
  const unsigned long long old = atomicCAS(slot, 0ull, slot_word(f, my_id));
  if (old == 0ull) {
    id = my_id;
    return kClaimed;
  }
  if (slot_fp(old) == f) {
    id = slot_id(old);
    return kHit;
  }
  return kNext;
}

// The rest of a probe sequence, one step at a time, from step p0.  Returns the
// slot (kOverflowSlot after P steps) and the cell id through `id`.
__device__ __forceinline__ uint32_t probe_rest(const TableDev& t, uint32_t home, uint32_t f,
                                               uint32_t p0, uint32_t my_id, uint32_t& id,
                                               bool& claimed) {
  claimed = false;
  for (uint32_t p = p0; p < t.max_probes; ++p) {
    const uint32_t s = (home + p) & t.mask;
    const ProbeOutcome o = probe_step(t.slots + s, ld_relaxed_u64(t.slots + s), f, my_id, id);
    if (o == kNext) continue;
    claimed = o == kClaimed;
    return s;
  }
  return kOverflowSlot;
}

// Read-only lookup of a key's cell id (query without a stored id), from
// probe step p0 on.
__device__ __forceinline__ uint32_t probe_find_from(const TableDev& t, uint32_t home, uint32_t f,
                                                    uint32_t p0) {
  for (uint32_t p = p0; p < t.max_probes; ++p) {
    const unsigned long long w = __ldcg(t.slots + ((home + p) & t.mask));
    if (w == 0ull) return kOverflowSlot;
    if (slot_fp(w) == f) return slot_id(w);
  }
  return kOverflowSlot;
}

__device__ __forceinline__ uint32_t probe_find(const TableDev& t, uint32_t home, uint32_t f) {
  return probe_find_from(t, home, f, 0u);
}

// History table probing: 32-bit compare-and-swap on the history fingerprint.
__device__ __forceinline__ uint32_t* hist_fp(const TableDev& t, uint32_t h) {
  return reinterpret_cast<uint32_t*>(t.hcells + static_cast<size_t>(h) * t.hstride + t.hfp_off);
}

__device__ __forceinline__ uint32_t hist_probe_rest(const TableDev& t, uint32_t home, uint32_t f,
                                                    uint32_t p0) {
  for (uint32_t p = p0; p < t.max_probes; ++p) {
    const uint32_t h = (home + p) & t.hmask;
    const uint32_t old = atomicCAS(hist_fp(t, h), 0u, f);
    if (old == 0u || old == f) return h;
  }
  return kOverflowSlot;
}

// Evicting history table (Sec. 3.4.3): fingerprint word = priority << 24 |
// low 24 bits of the fingerprint, 0 = empty.  Find the cell's entry in its
// window (refreshing its priority to this frame's), or claim the first empty
// cell, or -- with the window full -- replace the smallest word if its
// priority is older than this frame's.  `fresh`: the entry holds no history
// of this cell.  Compare-and-swaps on the whole word keep a concurrent
// claim, refresh or replacement from being lost; a few retries, then none.
static __device__ __noinline__ uint32_t hist_claim_evict(const TableDev& t, uint32_t home,
                                                         uint32_t f, bool* fresh) {
  const uint32_t f24 = f & 0xFFFFFFu;
  const uint32_t nw = (t.hist_rank << 24) | f24;
  for (int attempt = 0; attempt < 4; ++attempt) {
    uint32_t victim = kOverflowSlot, vword = 0xFFFFFFFFu;
    bool retry = false;
    for (uint32_t p = 0; p < t.max_probes; ++p) {
      const uint32_t h = (home + p) & t.hmask;
      uint32_t* fp = hist_fp(t, h);
      uint32_t w = __ldcg(fp);
      if (w == 0u) {
        w = atomicCAS(fp, 0u, nw);
        if (w == 0u) {
          *fresh = true;
          return h;
        }
      }
      if ((w & 0xFFFFFFu) == f24) {
        if (w != nw) {
          const uint32_t o = atomicCAS(fp, w, nw);
          if (o != w && (o & 0xFFFFFFu) != f24) {
            retry = true;  // replaced under us: scan again
            break;
          }
        }
        *fresh = false;
        return h;
      }
      if (w < vword) {
        vword = w;
        victim = h;
      }
    }
    if (retry) continue;
    if ((vword >> 24) >= t.hist_rank) return kOverflowSlot;  // all entries are this frame's
    if (atomicCAS(hist_fp(t, victim), vword, nw) == vword) {
      *fresh = true;
      return victim;
    }
  }
  return kOverflowSlot;
}

// Accumulate a group of `cnt` contributions (sums r, g, b) into cell `id`.
__device__ __forceinline__ void accumulate(const TableDev& t, uint32_t id, float r, float g, float b,
                                           long long fr, long long fg, long long fb, uint32_t cnt) {
  if (!t.fixed) {
    red_add_v4_keep(t.acc + id, r, g, b, static_cast<float>(cnt));
    return;
  }
  unsigned long long* a = t.acc64 + 4 * static_cast<size_t>(id);
  atomicAdd(a + 0, static_cast<unsigned long long>(fr));
  atomicAdd(a + 1, static_cast<unsigned long long>(fg));
  atomicAdd(a + 2, static_cast<unsigned long long>(fb));
  atomicAdd(a + 3, static_cast<unsigned long long>(cnt));
}

// Cell average of this frame: sum / count, one FP32 round-to-nearest division
// (fixed mode: fl32(sum) * 2^-24 / fl32(count)).
struct CellMean {
  float r, g, b;
  uint32_t n;
};

// The raw accumulator of a cell as loaded from memory (both modes).
struct AccRaw {
  float4 lo;  // FP32 sums, or int64 sums r, g as bits (fixed)
  float4 hi;  // fixed mode: int64 sum b and count as bits
};

__device__ __forceinline__ float4* value_ptr(const TableDev& t, uint32_t id) {
  return t.fixed ? reinterpret_cast<float4*>(t.acc64 + 4 * static_cast<size_t>(id)) : t.acc + id;
}

__device__ __forceinline__ AccRaw load_acc(const TableDev& t, uint32_t id) {
  AccRaw a;
  const float4* p = value_ptr(t, id);
  a.lo = __ldcg(p);
  a.hi = t.fixed ? __ldcg(p + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
  return a;
}

__device__ __forceinline__ long long bits64(float x, float y) {
  return static_cast<long long>((static_cast<unsigned long long>(__float_as_uint(y)) << 32) |
                                __float_as_uint(x));
}

__device__ __forceinline__ CellMean mean_of(const TableDev& t, const AccRaw& a) {
  CellMean m;
  if (!t.fixed) {
    if (a.lo.w >= kExactCountLimit) atomicOr(&t.ctrl->error, kErrCountSaturated);
    m.r = __fdiv_rn(a.lo.x, a.lo.w);
    m.g = __fdiv_rn(a.lo.y, a.lo.w);
    m.b = __fdiv_rn(a.lo.z, a.lo.w);
    m.n = static_cast<uint32_t>(a.lo.w);
  } else {
    const long long sr = bits64(a.lo.x, a.lo.y), sg = bits64(a.lo.z, a.lo.w);
    const long long sb = bits64(a.hi.x, a.hi.y);
    const unsigned long long n = static_cast<unsigned long long>(bits64(a.hi.z, a.hi.w));
    const float fn = __ull2float_rn(n);
    m.r = __fdiv_rn(__fmul_rn(__ll2float_rn(sr), 0x1p-24f), fn);
    m.g = __fdiv_rn(__fmul_rn(__ll2float_rn(sg), 0x1p-24f), fn);
    m.b = __fdiv_rn(__fmul_rn(__ll2float_rn(sb), 0x1p-24f), fn);
    m.n = static_cast<uint32_t>(n);
  }
  return m;
}

// History value as loaded from memory.
struct HistRaw {
  float r, g, b;
  uint32_t n;
};

__device__ __forceinline__ HistRaw load_hist(const TableDev& t, uint32_t h) {
  HistRaw o;
  const unsigned char* c = t.hcells + static_cast<size_t>(h) * t.hstride;
  if (t.hist_mode == 1) {
    const uint4 v = ld_once_u4(c);
    o.r = __uint_as_float(v.x);
    o.g = __uint_as_float(v.y);
    o.b = __uint_as_float(v.z);
    o.n = v.w;
  } else {
    const uint2 v = ld_once_u2(c);
    const float2 rg = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    o.r = rg.x;
    o.g = rg.y;
    o.b = __half2float(__ushort_as_half(static_cast<unsigned short>(v.y & 0xFFFFu)));
    o.n = v.y >> 16;
  }
  return o;
}

// Temporal filtering / integration of one cell (Sec. 3.4.1):
// c = alpha c_old + (1 - alpha) c_new, alpha < 0 meaning alpha = N_old / (N_old +
// N_new); no history -> c = c_new.  The history cell h is updated (h ==
// kOverflowSlot: the history window was full; the cell keeps c_new and
// N = N_new) and the result replaces the cell's accumulator for the lookups.
__device__ __forceinline__ void blend_store(const TableDev& t, uint32_t id, uint32_t h,
                                            const CellMean& m, const HistRaw& old, float alpha) {
  float cr = m.r, cg = m.g, cb = m.b;
  uint32_t N = m.n;
  if (h != kOverflowSlot) {
    if (old.n != 0u) {
      const float a =
          alpha >= 0.0f ? alpha
                        : __fdiv_rn(__uint2float_rn(old.n),
                                    __fadd_rn(__uint2float_rn(old.n), __uint2float_rn(m.n)));
      const float a1 = __fsub_rn(1.0f, a);
      cr = __fadd_rn(__fmul_rn(a, old.r), __fmul_rn(a1, cr));
      cg = __fadd_rn(__fmul_rn(a, old.g), __fmul_rn(a1, cg));
      cb = __fadd_rn(__fmul_rn(a, old.b), __fmul_rn(a1, cb));
    }
    unsigned char* c = t.hcells + static_cast<size_t>(h) * t.hstride;
    if (t.hist_mode == 1) {
      N = old.n + m.n;
      st_once_u4(c, make_uint4(__float_as_uint(cr), __float_as_uint(cg), __float_as_uint(cb), N));
    } else {
      N = min(old.n + m.n, 65535u);
      const __half2 rg = __floats2half2_rn(cr, cg);
      const __half hb = __float2half_rn(cb);
      const uint32_t lo = *reinterpret_cast<const uint32_t*>(&rg);
      const uint32_t hi = static_cast<uint32_t>(__half_as_ushort(hb)) | (N << 16);
      st_once_u2(c, make_uint2(lo, hi));
      // lookups see what the history stores
      const float2 back = __half22float2(rg);
      cr = back.x;
      cg = back.y;
      cb = __half2float(hb);
    }
  }
  __stcg(value_ptr(t, id), make_float4(cr, cg, cb, __uint_as_float(N)));
}

// Value returned for cell `id`: the cell average, or the blended value.
__device__ __forceinline__ CellMean value_of(const TableDev& t, const AccRaw& a, bool blended) {
  if (!blended) return mean_of(t, a);
  CellMean m;
  m.r = a.lo.x;
  m.g = a.lo.y;
  m.b = a.lo.z;
  m.n = __float_as_uint(a.lo.w);
  return m;
}

__device__ __forceinline__ AccRaw load_value(const TableDev& t, uint32_t id, bool blended) {
  if (!blended) return load_acc(t, id);
  AccRaw a;
  a.lo = __ldcg(value_ptr(t, id));
  a.hi = make_float4(0.f, 0.f, 0.f, 0.f);
  return a;
}

// Empty cell `id` (its accumulator and its slot) for the next frame.
__device__ __forceinline__ void clear_cell(const TableDev& t, uint32_t id, uint32_t slot) {
  float4* p = value_ptr(t, id);
  st_zero16_keep(p);
  if (t.fixed) st_zero16_keep(p + 1);
  if (slot != kNoSlot) __stcg(t.slots + slot, 0ull);
}

// ---------------------------------------------------------------- grid barrier
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier over all CTAs of a cooperative launch.  Thread 0 of each CTA
// arrives on a counter; the last arrival resets it and bumps the generation;
// the others wait for the generation to change.  The wait is bounded (about
// two seconds of wall time): on timeout the CTA raises kErrBarrierTimeout in
// the device error word and every CTA returns false, so the launch ends.
__device__ __forceinline__ bool grid_barrier(Ctrl* c, unsigned int nblocks,
                                             unsigned long long limit_ns = 2000000000ull) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int gen = ld_acquire_u32(&c->bar_gen);
    __threadfence();
    const unsigned int arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == nblocks - 1u) {
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      while (ld_acquire_u32(&c->bar_gen) == gen) {
        if (ld_acquire_u32(&c->error) & kErrBarrierTimeout) {
          ok = 0;
          break;
        }
        if (globaltimer_ns() - t0 > limit_ns) {
          atomicOr(&c->error, kErrBarrierTimeout);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace pps
