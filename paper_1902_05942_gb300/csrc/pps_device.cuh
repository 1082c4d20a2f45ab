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
};

// Per-frame and lifetime counters plus the device error word and the state of
// the grid barrier used by the persistent filter kernel.
struct Ctrl {
  unsigned long long frame_cells;
  unsigned long long overflow_vertices;
  unsigned long long vertices;
  unsigned long long hist_overflow;
  unsigned int dirty_count;
  unsigned int error;
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned int pad[4];
};
constexpr size_t kCtrlFrameBytes = 4 * sizeof(unsigned long long);  // reset per frame

enum : unsigned int {
  kErrBarrierTimeout = 1u,
  kErrBadSlot = 2u,
};

// Fixed-point accumulator of one cell: sums of round(v * 2^24) and the count.
struct __align__(32) AccFixed {
  long long r, g, b;
  unsigned long long n;
};

// The frame table (fp, acc) is emptied every frame.  Temporal state lives in a
// separate history table (hfp, hist / hist16) whose fingerprints persist across
// frames; the owner of a frame cell links it to its history cell (hslot).
struct TableDev {
  uint32_t* fp;       // [T] fingerprints, 0 = empty
  float4* acc;        // [T] FP32 {sum r, sum g, sum b, count} (FP32 mode)
  AccFixed* acc64;    // [T] fixed-point accumulators (fixed mode)
  uint32_t* dirty;    // [T] cells claimed this frame (split path)
  uint32_t* hslot;    // [T] history cell of each claimed frame cell
  uint32_t* hfp;      // [Th] history fingerprints
  float4* hist;       // [Th] FP32 history {c r, c g, c b, N bits} (hist FP32)
  uint2* hist16;      // [Th] FP16 history {half2(r,g), half b | u16 N << 16}
  Ctrl* ctrl;
  uint32_t mask;      // T - 1
  uint32_t hmask;     // Th - 1
  uint32_t max_probes;
  uint32_t lowcount;
  int fixed;          // accumulation mode
  int hist_mode;      // 0 none, 1 FP32, 2 FP16
};

struct VertexPtrs {
  const float *px, *py, *pz, *nx, *ny, *nz, *r, *g, *b;
  const uint32_t* id;
  uint32_t id_base;
  uint32_t stream_id;
};

struct OutPtrs {
  float *r, *g, *b;
  uint32_t* count;
  uint8_t* status;
};

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds of two 32x32->64 multiplies; the key is
// bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint2 philox_first2(uint32_t c0, uint32_t c1, uint32_t k0,
                                               uint32_t k1) {
  uint32_t x0 = c0, x1 = c1, x2 = 0u, x3 = 0u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
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

// floor(log2(k * |p_cam - x|)) from the exponent bits of the FP32 product.
__device__ __forceinline__ int level_of_detail(const KeyConst& kc, float x, float y, float z) {
  const float dx = __fsub_rn(kc.cam[0], x);
  const float dy = __fsub_rn(kc.cam[1], y);
  const float dz = __fsub_rn(kc.cam[2], z);
  const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  const float F = __fmul_rn(kc.k, __fsqrt_rn(d2));
  const int e = static_cast<int>((__float_as_uint(F) >> 23) & 0xFFu) - 127;
  return min(max(e, kc.lod_min), kc.lod_max);
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

__device__ __forceinline__ Key vertex_key(const KeyConst& kc, float px, float py, float pz,
                                          float nx, float ny, float nz, uint32_t id,
                                          uint32_t stream_id) {
  const int l0 = level_of_detail(kc, px, py, pz);
  float xj = px, yj = py, zj = pz;
  int l1 = l0;
  if (kc.jitter) {
    // jitter(n): a point of the tangent plane, (u, w) uniform in [-0.5, 0.5)
    const uint2 rnd = philox_first2(id, stream_id, kc.seed, kc.frame);
    const float u = __fsub_rn(__fmul_rn(__uint2float_rn(rnd.x >> 8), 0x1p-24f), 0.5f);
    const float w = __fsub_rn(__fmul_rn(__uint2float_rn(rnd.y >> 8), 0x1p-24f), 0.5f);
    // tangent frame after Duff et al. (JCGT 2017)
    const float s = copysignf(1.0f, nz);
    const float a = __fdiv_rn(-1.0f, __fadd_rn(s, nz));
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
    l1 = level_of_detail(kc, xj, yj, zj);
  }
  const float inv = pow2_int(-l1);
  const uint32_t X = static_cast<uint32_t>(quantize_coord(xj, inv));
  const uint32_t Y = static_cast<uint32_t>(quantize_coord(yj, inv));
  const uint32_t Z = static_cast<uint32_t>(quantize_coord(zj, inv));
  const uint32_t L = static_cast<uint32_t>(l1);
  const uint32_t NQ = quantize_normal(nx) | (quantize_normal(ny) << 8) | (quantize_normal(nz) << 16);
  uint32_t h = kc.hseed_home;
  h = mm_body(h, X);
  h = mm_body(h, Y);
  h = mm_body(h, Z);
  h = mm_body(h, L);
  if (kc.nih) {
    h = mm_body(h, NQ);
    h = mm_final(h, 20u);
  } else {
    h = mm_final(h, 16u);
  }
  uint32_t f = kc.hseed_fp;
  f = mm_body(f, X);
  f = mm_body(f, Y);
  f = mm_body(f, Z);
  f = mm_body(f, L);
  f = mm_body(f, NQ);
  f = mm_final(f, 20u);
  return Key{h, f ? f : 1u};
}

// ---------------------------------------------------------------- memory helpers
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_add_v4(float4* p, float a, float b, float c, float d) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a),
               "f"(b), "f"(c), "f"(d)
               : "memory");
}

__device__ __forceinline__ float4 atom_add_v4(float4* p, float a, float b, float c, float d) {
  float4 o;
  asm volatile("atom.relaxed.gpu.global.add.v4.f32 {%0, %1, %2, %3}, [%4], {%5, %6, %7, %8};"
               : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w)
               : "l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
  return o;
}

__device__ __forceinline__ long long to_fixed(float v) {
  return __float2ll_rn(__fmul_rn(v, 16777216.0f));  // round(v * 2^24), exact product
}

// Linear probing on the fingerprint word (Sec. 3.2): a slot holding f is a hit,
// an empty slot is claimed with one compare-and-swap, anything else is skipped.
// Fingerprints are only ever published, never moved, so a key that exists in
// the window is found before any empty slot.  Returns kOverflowSlot after P
// steps.  `claimed` is set when this call published f.
__device__ __forceinline__ uint32_t probe_insert(uint32_t* fp, uint32_t mask, uint32_t P,
                                                 uint32_t home, uint32_t f, bool& claimed) {
  claimed = false;
  for (uint32_t p = 0; p < P; ++p) {
    const uint32_t s = (home + p) & mask;
    const uint32_t cur = ld_relaxed(fp + s);
    if (cur == f) return s;
    if (cur == 0u) {
      const uint32_t old = atomicCAS(fp + s, 0u, f);
      if (old == 0u) {
        claimed = true;
        return s;
      }
      if (old == f) return s;
    }
  }
  return kOverflowSlot;
}

// Read-only probe (query without a stored slot index).
__device__ __forceinline__ uint32_t probe_find(const uint32_t* fp, uint32_t mask, uint32_t P,
                                               uint32_t home, uint32_t f) {
  for (uint32_t p = 0; p < P; ++p) {
    const uint32_t s = (home + p) & mask;
    const uint32_t cur = __ldcg(fp + s);
    if (cur == f) return s;
    if (cur == 0u) return kOverflowSlot;
  }
  return kOverflowSlot;
}

// Accumulate one contribution (or a group of `cnt` combined ones) into cell s.
__device__ __forceinline__ void accumulate(const TableDev& t, uint32_t s, float r, float g, float b,
                                           long long fr, long long fg, long long fb, uint32_t cnt) {
  if (!t.fixed) {
    red_add_v4(t.acc + s, r, g, b, static_cast<float>(cnt));
    return;
  }
  AccFixed* a = t.acc64 + s;
  atomicAdd(reinterpret_cast<unsigned long long*>(&a->r), static_cast<unsigned long long>(fr));
  atomicAdd(reinterpret_cast<unsigned long long*>(&a->g), static_cast<unsigned long long>(fg));
  atomicAdd(reinterpret_cast<unsigned long long*>(&a->b), static_cast<unsigned long long>(fb));
  atomicAdd(&a->n, static_cast<unsigned long long>(cnt));
}

// The owner (claimer) of frame cell s finds or claims the key's history cell
// and records it in hslot[s] (kOverflowSlot when the history window is full).
__device__ __forceinline__ void link_history(const TableDev& t, uint32_t s, uint32_t h1, uint32_t f,
                                             unsigned long long& n_hovf) {
  bool claimed;
  const uint32_t hs = probe_insert(t.hfp, t.hmask, t.max_probes, h1 & t.hmask, f, claimed);
  n_hovf += hs == kOverflowSlot ? 1ull : 0ull;
  __stcg(t.hslot + s, hs);
}

// Cell average of this frame: sum / count, one FP32 round-to-nearest division
// (fixed mode: fl32(sum) * 2^-24 / fl32(count)).
struct CellMean {
  float r, g, b;
  uint32_t n;
};

__device__ __forceinline__ CellMean cell_mean(const TableDev& t, uint32_t s) {
  CellMean m;
  if (!t.fixed) {
    const float4 a = __ldcg(t.acc + s);
    m.r = __fdiv_rn(a.x, a.w);
    m.g = __fdiv_rn(a.y, a.w);
    m.b = __fdiv_rn(a.z, a.w);
    m.n = static_cast<uint32_t>(a.w);
  } else {
    const AccFixed* a = t.acc64 + s;
    const long long sr = __ldcg(&a->r), sg = __ldcg(&a->g), sb = __ldcg(&a->b);
    const unsigned long long n = __ldcg(&a->n);
    const float fn = __ull2float_rn(n);
    m.r = __fdiv_rn(__fmul_rn(__ll2float_rn(sr), 0x1p-24f), fn);
    m.g = __fdiv_rn(__fmul_rn(__ll2float_rn(sg), 0x1p-24f), fn);
    m.b = __fdiv_rn(__fmul_rn(__ll2float_rn(sb), 0x1p-24f), fn);
    m.n = static_cast<uint32_t>(n);
  }
  return m;
}

// The blended value of a frame cell replaces its accumulator: 16 bytes
// {c r, c g, c b, N bits} at the start of the cell's accumulator (both modes).
__device__ __forceinline__ float4* blended_slot(const TableDev& t, uint32_t s) {
  return t.fixed ? reinterpret_cast<float4*>(t.acc64 + s) : t.acc + s;
}

// Temporal filtering / integration of one cell (Sec. 3.4.1), run once per
// claimed frame cell by its owner: c = alpha c_old + (1 - alpha) c_new, where
// alpha < 0 means alpha = N_old / (N_old + N_new); no history -> c = c_new.
// The history cell is updated and the result is left in the frame cell for
// the lookups of this frame.  A cell whose history window was full keeps
// c_new and N = N_new.
__device__ __forceinline__ void blend_cell(const TableDev& t, uint32_t s, float alpha) {
  const CellMean m = cell_mean(t, s);
  float cr = m.r, cg = m.g, cb = m.b;
  uint32_t N = m.n;
  const uint32_t hs = __ldcg(t.hslot + s);
  if (hs != kOverflowSlot) {
    uint32_t n_old;
    float or_, og, ob;
    if (t.hist_mode == 1) {
      const float4 h = __ldcg(t.hist + hs);
      or_ = h.x;
      og = h.y;
      ob = h.z;
      n_old = __float_as_uint(h.w);
    } else {
      const uint2 h = __ldcg(t.hist16 + hs);
      const float2 rg = __half22float2(*reinterpret_cast<const __half2*>(&h.x));
      or_ = rg.x;
      og = rg.y;
      ob = __half2float(__ushort_as_half(static_cast<unsigned short>(h.y & 0xFFFFu)));
      n_old = h.y >> 16;
    }
    if (n_old != 0u) {
      const float a =
          alpha >= 0.0f ? alpha
                        : __fdiv_rn(__uint2float_rn(n_old),
                                    __fadd_rn(__uint2float_rn(n_old), __uint2float_rn(m.n)));
      const float a1 = __fsub_rn(1.0f, a);
      cr = __fadd_rn(__fmul_rn(a, or_), __fmul_rn(a1, cr));
      cg = __fadd_rn(__fmul_rn(a, og), __fmul_rn(a1, cg));
      cb = __fadd_rn(__fmul_rn(a, ob), __fmul_rn(a1, cb));
    }
    if (t.hist_mode == 1) {
      N = n_old + m.n;
      __stcg(t.hist + hs, make_float4(cr, cg, cb, __uint_as_float(N)));
    } else {
      N = min(n_old + m.n, 65535u);
      const __half2 rg = __floats2half2_rn(cr, cg);
      const __half hb = __float2half_rn(cb);
      const uint32_t lo = *reinterpret_cast<const uint32_t*>(&rg);
      const uint32_t hi = static_cast<uint32_t>(__half_as_ushort(hb)) | (N << 16);
      __stcg(t.hist16 + hs, make_uint2(lo, hi));
      // lookups see what the history stores
      const float2 back = __half22float2(rg);
      cr = back.x;
      cg = back.y;
      cb = __half2float(hb);
    }
  }
  __stcg(blended_slot(t, s), make_float4(cr, cg, cb, __uint_as_float(N)));
}

// Value returned for a vertex of cell s: the cell average, or the blended
// value left in the cell by blend_cell.
__device__ __forceinline__ CellMean cell_value(const TableDev& t, uint32_t s, bool blended) {
  if (!blended) return cell_mean(t, s);
  const float4 h = __ldcg(blended_slot(t, s));
  CellMean m;
  m.r = h.x;
  m.g = h.y;
  m.b = h.z;
  m.n = __float_as_uint(h.w);
  return m;
}

// Empty a frame cell (fingerprint and accumulator) for the next frame.
__device__ __forceinline__ void clear_cell(const TableDev& t, uint32_t s) {
  if (!t.fixed) {
    __stcg(t.acc + s, make_float4(0.f, 0.f, 0.f, 0.f));
  } else {
    float4* p = reinterpret_cast<float4*>(t.acc64 + s);
    __stcg(p, make_float4(0.f, 0.f, 0.f, 0.f));
    __stcg(p + 1, make_float4(0.f, 0.f, 0.f, 0.f));
  }
  __stcg(t.fp + s, 0u);
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
__device__ __forceinline__ bool grid_barrier(Ctrl* c, unsigned int nblocks) {
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
        if (globaltimer_ns() - t0 > 2000000000ull) {
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
