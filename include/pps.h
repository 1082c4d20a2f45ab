/*
 * pps.h -- C ABI of the GB300 hashed path space filtering library.
 *
 * The operation is the second phase of the method of Binder, Fricke and Keller,
 * "Massively Parallel Path Space Filtering" (2019), Sec. 3: the input is a set
 * of path vertices with their descriptors (position, normal) and their
 * contributions L_i f_i cos (Eq. 9); every vertex receives the average of the
 * contributions of all vertices whose quantized key equals its own (Eq. 7,
 * Eq. 8/9 with w = 1), optionally blended across frames (Sec. 3.4.1).
 *
 * Conventions (all entry points):
 *  - Every function is extern "C", returns int: PPS_OK (0) or a PPS_E* code;
 *    pps_last_error() returns the message of the calling thread's last error.
 *    No C++ exception crosses this boundary.
 *  - Array arguments are DEVICE pointers owned by the caller unless the name
 *    says _host.  The library owns only what pps_create allocates (the table,
 *    its control block and, on demand, its scratch buffers) and frees it in
 *    pps_destroy.
 *  - Work is enqueued on the cudaStream_t passed as `void* stream` (NULL = the
 *    legacy default stream) and runs asynchronously; only pps_stats,
 *    pps_table_dump and pps_filter_host synchronize that stream.
 *  - A table is bound to the device that was current at pps_create; call it
 *    with that device current.  A table must not be used from two host threads
 *    at once, and calls on one table must be ordered (same stream, or streams
 *    ordered by events).
 *  - Float inputs must be finite; normals must be unit length.
 */
#ifndef PPS_H
#define PPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define PPS_OK 0
#define PPS_EINVAL 1  /* bad argument (NULL, size, alignment, range)          */
#define PPS_ENOMEM 2  /* device or host allocation failed                      */
#define PPS_ECUDA 3   /* a CUDA runtime call failed (message has the name)     */
#define PPS_EDEVICE 4 /* a kernel raised the table's device error word         */
#define PPS_ESTATE 5  /* call out of order for the table's frame state         */

/* ---- bits of the device error word (pps_stats_t.device_error) ----------- */
#define PPS_DEVERR_BARRIER_TIMEOUT 1u  /* a grid-barrier wait gave up (~2 s);   */
                                       /* the launch ended early                */
#define PPS_DEVERR_BAD_SLOT 2u         /* a lookup got a cell id that is not    */
                                       /* one of this frame's                   */
#define PPS_DEVERR_COUNT_SATURATED 4u  /* FP32 accumulation: a cell reached     */
                                       /* 2^24 members, past which its FP32     */
                                       /* count (and so its average) is not     */
                                       /* exact; PPS_ACCUM_FIXED has no limit   */

/* ---- per-vertex status written by pps_query / pps_filter ---------------- */
#define PPS_STATUS_OK 0       /* cell average returned                         */
#define PPS_STATUS_LOWCOUNT 1 /* average returned, count < lowcount_threshold  */
#define PPS_STATUS_OVERFLOW 2 /* probe limit exceeded: the vertex's own,       */
                              /* unfiltered contribution returned (Sec. 3.2)   */
#define PPS_STATUS_MLP 3      /* low count: the learned fallback's prediction  */
#define PPS_STATUS_COARSE 4   /* low count: the next coarser resolution's cell */
                              /* average (multi-level accumulation, 3.3.2)     */
#define PPS_STATUS_NEIGHBORS 5 /* low count: pooled average of the 3x3x3 block */
                              /* of cells around the vertex's (Sec. 3.3.1)     */

/* ---- modes -------------------------------------------------------------- */
#define PPS_ACCUM_FP32 0  /* FP32 sums, FP32 count lane: red.add.v4.f32; counts */
                          /* exact below 2^24 members per cell (see above)      */
#define PPS_ACCUM_FIXED 1 /* int64 sums of round(v * 2^24): order-free, exact   */
#define PPS_HIST_NONE 0   /* no temporal state: every frame starts empty        */
#define PPS_HIST_FP32 1   /* history average FP32, count uint32                 */
#define PPS_HIST_FP16 2   /* history average binary16, count uint16 saturating  */
#define PPS_FALLBACK_NONE 0      /* low-count vertices keep their cell average  */
#define PPS_FALLBACK_COARSE 1    /* multi-level accumulation (Sec. 3.3.2)       */
#define PPS_FALLBACK_NEIGHBORS 2 /* neighborhood search (Sec. 3.3.1)            */

/*
 * Table and key parameters (Algorithm 1; Sec. 3.1.1, 3.2, 3.2.1; Sec. 4).
 *
 *  log2_slots         T = 2^log2_slots cells, 4 <= log2_slots <= 30.  The index
 *                     is hash & (T - 1) ("modulo", Sec. 3.2).
 *  max_probes         P, linear-probing limit, 1 <= P <= min(T, 4096).  A vertex
 *                     that finds neither its fingerprint nor an empty cell in
 *                     P steps keeps its own contribution (Sec. 3.2).
 *  voxel_scale        s > 0: the voxel edge is s times the projected size of a
 *                     pixel at the vertex's camera distance (Sec. 4), snapped
 *                     down to a power of two: 2^floor(log2(s * pixel_angle * d)).
 *  pixel_angle        theta_px > 0 = 2 tan(fov_y / 2) / image height.
 *  jitter             1: jitter positions in the tangent plane before
 *                     quantization (Sec. 3.1.4, Alg. 1); 0: plain quantization.
 *  seed               jitter key word 0 (word 1 is the frame number).
 *  hash_seed_home     seed of hash  (MurmurHash3_x86_32) -> home index i.
 *  hash_seed_fp       seed of hash2 (MurmurHash3_x86_32) -> fingerprint f; the
 *                     sentinel 0 marks an empty cell and is remapped to 1
 *                     (Sec. 3.2.1).
 *  normal_in_home_hash 0: the quantized normal enters only hash2, exactly as
 *                     Algorithm 1 prints it; 1: it enters both hashes
 *                     ("the arguments ... may be extended", Alg. 1 caption).
 *                     Cell membership is the same either way.
 *  lod_min, lod_max   clamp of the level of detail, -126 < lod_min <= lod_max < 127.
 *  accum_mode         PPS_ACCUM_FP32 or PPS_ACCUM_FIXED.
 *  hist_mode          PPS_HIST_NONE, PPS_HIST_FP32 or PPS_HIST_FP16: the
 *                     temporal state of Sec. 3.4.1 in a second open-addressed
 *                     table whose fingerprints persist across frames.
 *  lowcount_threshold a returned count below it is flagged LOWCOUNT (Sec. 3.3).
 *  log2_hist_slots    history table size Th = 2^log2_hist_slots (0: same as T),
 *                     4..30; probed with the same limit P.
 *  fallback           what a vertex whose cell holds fewer than
 *                     lowcount_threshold members (after a blend: N) receives
 *                     instead of its cell's average (Sec. 3.3):
 *                     PPS_FALLBACK_NONE       the cell average, status LOWCOUNT;
 *                     PPS_FALLBACK_COARSE     multi-level accumulation (3.3.2):
 *                        the table keeps a second table for the next coarser
 *                        resolution (voxel_scale doubled, so every level of
 *                        detail grows by exactly one; same T, P, seeds, modes
 *                        and its own history), every vertex is inserted into
 *                        both, and a low-count vertex gets the coarser cell's
 *                        value and count, status COARSE (unless its coarse
 *                        insert overflowed: then LOWCOUNT as before);
 *                     PPS_FALLBACK_NEIGHBORS  neighborhood search (3.3.1): a
 *                        low-count vertex gets the pooled average of the
 *                        3 x 3 x 3 block of cells around its own (same level,
 *                        same quantized normal): the block's summed sums over
 *                        its summed counts, or after a blend the blended values
 *                        weighted by their N; count = the block's members,
 *                        status NEIGHBORS.
 *                     Fallback tables work with pps_filter and the split calls;
 *                     pps_batch_create and pps_filter_noalloc reject them, and
 *                     pps_stats / pps_table_dump / pps_keys describe the
 *                     table's own (finest) resolution.
 *  hist_evict         1: the history table evicts (Sec. 3.4.3).  Its 32-bit
 *                     fingerprint words hold a priority in the top 8 bits --
 *                     the blend epoch of the entry's last use (1..255, counted
 *                     per table; when it runs out every priority drops by 128)
 *                     -- over the fingerprint's low 24 bits.  A cell that finds
 *                     neither its entry nor an empty cell in its P-cell window
 *                     replaces the entry with the smallest word (least recently
 *                     used) if that entry is older than this frame, and starts
 *                     afresh there (no history).  Entries found are refreshed
 *                     to this epoch.  Needs hist_mode != NONE.  0: no eviction
 *                     (history entries live as long as the table).
 *  hist_migrate       1: history follows changes of resolution across frames
 *                     (Sec. 3.4.2).  A cell whose history entry is new this
 *                     frame takes as its old value the history of its eight
 *                     finer children (2 x~ + {0,1}^3 at level l' - 1, same
 *                     quantized normal) added up -- sum(N_i c_i) / sum(N_i)
 *                     with count sum(N_i) -- or, with no such child, the
 *                     average of its coarser parent (floor(x~ / 2) at level
 *                     l' + 1) with count ceil(N_parent / 8).  The lookups read
 *                     the history as it was before this frame's blend.  Needs
 *                     hist_mode != NONE and hist_evict = 0; frames run through
 *                     the split kernels (pps_filter does so itself), which then
 *                     keep each cell's quantized key (16 B per cell); no extra
 *                     key word (pps_vertices.extra) is accepted; pps_batch_create
 *                     and pps_filter_noalloc reject such tables.
 *  normal_search      searching similar normals by linear probing (Sec. 3.2.2):
 *                     0 = off; r + 1 (r = 0 .. 255) = every lookup returns the
 *                     pooled average of the cells of its voxel (same x~ and
 *                     l') whose quantized normal lies within r steps of its
 *                     own on every axis (max over axes |q - q'| <= r): the
 *                     pooled sums over the pooled counts (fixed point: exact
 *                     int64 sums), or after a blend the blended values
 *                     weighted by their N; count = the pooled count, status
 *                     OK or LOWCOUNT by it.  Needs normal_in_home_hash = 0
 *                     (so a voxel's normals share a home slot and lie within
 *                     its P-slot window, which the lookup walks past
 *                     mismatching entries) and fallback NONE; no extra key
 *                     word.  Frames run through the split kernels, which keep
 *                     each cell's quantized key (16 B per cell) for the test;
 *                     pps_batch_create and pps_filter_noalloc reject such
 *                     tables.  r = 0 gives the plain lookup.
 */
typedef struct pps_params {
  uint32_t log2_slots;
  uint32_t max_probes;
  float voxel_scale;
  float pixel_angle;
  uint32_t jitter;
  uint32_t seed;
  uint32_t hash_seed_home;
  uint32_t hash_seed_fp;
  uint32_t normal_in_home_hash;
  int32_t lod_min;
  int32_t lod_max;
  uint32_t accum_mode;
  uint32_t hist_mode;
  uint32_t lowcount_threshold;
  uint32_t log2_hist_slots;
  uint32_t fallback;
  uint32_t hist_evict;
  uint32_t hist_migrate;
  uint32_t normal_search;
} pps_params;

/* Camera position p_cam of Algorithm 1 (world space). */
typedef struct pps_camera {
  float pos[3];
} pps_camera;

/*
 * One batch of path vertices, structure of arrays, n entries each (device).
 *  px,py,pz   position x;  nx,ny,nz unit normal n;  r,g,b contribution.
 *  id         optional per-vertex jitter counter (NULL: id_base + index).
 *  stream_id  second jitter counter word (e.g. a view index).
 *  dist       optional per-vertex distance for the level of detail (e.g. the
 *             length of the path to the vertex, Sec. 3.1.1) in place of the
 *             camera distance: l = level(dist); after the jitter,
 *             l' = level((dist - |p_cam - x|) + |p_cam - x'|), FP32 with one
 *             rounding per operation (so dist = |p_cam - x| gives Algorithm 1
 *             exactly).  NULL: Algorithm 1.
 *  extra      optional per-vertex 32-bit key word (a material or layer id, a
 *             quantized incident direction, ...; Sec. 3.1.2 and the caption of
 *             Algorithm 1) hashed last into both hashes: vertices share a cell
 *             only if their extra words are equal.  NULL: none.  Use the same
 *             choice for every call on a table in a frame.
 * pps_filter runs frames with dist or extra through the split kernels (the
 * persistent launch is built without them); pps_batch_create,
 * pps_filter_noalloc and the host-buffer calls reject them.
 * All nine float arrays are required.  16-byte-aligned arrays are read with
 * 128-bit loads; other alignments take a scalar path.
 */
typedef struct pps_vertices {
  const float *px, *py, *pz;
  const float *nx, *ny, *nz;
  const float *r, *g, *b;
  const uint32_t *id;
  uint32_t id_base;
  uint32_t stream_id;
  const float *dist;
  const uint32_t *extra;
} pps_vertices;

/*
 * Per-vertex results (device), n entries each.
 *  r,g,b   filtered contribution: the cell average (or the blended history
 *          value with a history), or the own contribution on OVERFLOW.
 *  count   optional: vertices behind the returned value (this frame's cell
 *          count; N_old + N_new with a history; 0 on OVERFLOW).
 *  status  optional: PPS_STATUS_* per vertex.
 */
typedef struct pps_output {
  float *r, *g, *b;
  uint32_t *count;
  uint8_t *status;
} pps_output;

/* Counters of the last frame (filled by pps_stats). */
typedef struct pps_stats_t {
  uint64_t frame_cells;       /* cells claimed this frame                      */
  uint64_t overflow_vertices; /* vertices that hit the probe limit this frame  */
  uint64_t occupied_slots;    /* frame-table slots holding a fingerprint now   */
  uint64_t vertices;          /* vertices inserted this frame                  */
  uint64_t hist_overflow;     /* cells whose history window was full           */
  uint64_t hist_occupied;     /* history slots holding a fingerprint           */
  uint32_t device_error;      /* device error word (0 = none)                  */
  uint32_t frame;             /* frame number of the last pps_build/pps_filter */
} pps_stats_t;

/*
 * Launch shape of a table's kernels (no effect on results up to the order of
 * FP32 additions; fixed-point results are identical).
 *  batch      per-thread insert: vertices each thread carries through one
 *             insert step together (their probes and atomics overlap): 2 or 4;
 *             0 = library default (2).  Also used by the split kernels and the
 *             batched launch.
 *  insert     how pps_filter's persistent launch inserts: 0 = library default
 *             (pipelined while the slot index fits in L2, T <= 2^23; per
 *             thread for larger tables), 1 = per thread (each thread builds its vertices'
 *             keys, then probes and accumulates them), 2 = pipelined (key
 *             warps build keys, merge equal ones within the warp as `merge`
 *             says and queue one entry per group in shared memory; probe
 *             warps run the table operations of four queued keys per thread
 *             at once).  Frames
 *             with an evicting history or the neighborhood fallback always
 *             insert per thread.
 *  key_warps  pipelined insert: key warps of the 16 warps of a CTA (the rest
 *             probe): 4, 8 or 12; 0 = library default (8).
 *  block      batched launch (taken from the first view's table): threads
 *             per CTA, 256 or 512; 0 = library default (512).  Each CTA
 *             takes tiles of 2,048 vertices, 2048 / block per thread.
 *  merge      pipelined insert: warp aggregation of equal keys before they are
 *             queued: 0 = library default (2); 1 = none, one queue entry per
 *             vertex; 2 = merge with __match_any_sync (the lowest lane of each
 *             group of equal keys leads, the others add their contributions
 *             to its entry) in the warps where two neighbouring lanes hold
 *             equal keys, and skip the match elsewhere (coherent primary hits
 *             repeat keys across neighbouring pixels; secondary bounces
 *             rarely repeat one within a warp); 3 = merge in every warp.
 *  reserved   must be zero.
 */
typedef struct pps_tuning {
  uint32_t batch;
  uint32_t insert;
  uint32_t key_warps;
  uint32_t block;
  uint32_t merge;
  uint32_t reserved[3];
} pps_tuning;

typedef struct pps_table pps_table;

/* Library version string (static storage). */
const char *pps_version(void);

/* Copies the calling thread's last error message into buf (NUL-terminated,
 * truncated to len).  Returns PPS_OK. */
int pps_last_error(char *buf, size_t len);

/*
 * pps_create: allocate a table for `p` on the current device and clear it.
 * The frame table's cells (Sec. 3.2) are separate arrays: fingerprints (4 B
 * per cell) and accumulators (16 B FP32 / 32 B fixed).  With a history, a
 * second table holds fingerprints (4 B) and history values (16 B FP32 / 8 B
 * FP16) per history cell, plus 4 B per frame cell linking it to its history
 * cell.  *out receives the handle.
 * Errors: PPS_EINVAL (bad parameters), PPS_ENOMEM, PPS_ECUDA.
 */
int pps_create(pps_table **out, const pps_params *p);

/* pps_destroy: synchronize the device and free everything pps_create and
 * later calls allocated.  NULL is accepted. */
int pps_destroy(pps_table *t);

/*
 * pps_build: begin a frame (Sec. 3, second phase): record the camera and the
 * frame number (jitter key word 1) and empty the frame-table cells of the
 * previous frame (the history is kept).
 * Errors: PPS_EINVAL.
 */
int pps_build(pps_table *t, const pps_camera *cam, uint32_t frame, void *stream);

/*
 * pps_insert: for each of the n vertices compute its key (Algorithm 1), find
 * or claim its cell by linear probing on the fingerprint word (Sec. 3.2,
 * 3.2.1) and add its contribution and a count of one atomically (Sec. 3.2,
 * Sec. 3.3.1).  The vertex that claims a cell also finds or claims the key's
 * history cell when the table keeps a history.  slot_out (nullable, n entries): the vertex's cell index, or 0xFFFFFFFF when
 * the probe limit was exceeded; pass it to pps_query to skip re-probing.
 * May be called several times per frame.  Errors: PPS_EINVAL, PPS_ESTATE
 * (no pps_build since the last pps_blend).
 */
int pps_insert(pps_table *t, const pps_vertices *v, size_t n, uint32_t *slot_out,
               void *stream);

/*
 * pps_blend: temporal filtering / integration (Sec. 3.4.1) over every cell
 * touched this frame: c = alpha * c_old + (1 - alpha) * c_new, where c_new is
 * the cell's average this frame and c_old its history; alpha < 0 selects
 * alpha = N_old / (N_old + N_new), which integrates exactly.  A cell without
 * history takes c_new.  N <- N_old + N_new.  Requires hist_mode != NONE.
 * After it, pps_query returns the blended value.  Errors: PPS_EINVAL, PPS_ESTATE.
 */
int pps_blend(pps_table *t, float alpha, void *stream);

/*
 * pps_query: one lookup per vertex (Sec. 3.3.1): the cell average sum / count
 * (FP32 round-to-nearest division), or the blended history value after
 * pps_blend.  slot_in (nullable) must come from pps_insert of the same vertices
 * this frame; without it the key is recomputed and the cell found by
 * read-only probing.  Errors: PPS_EINVAL.
 */
int pps_query(pps_table *t, const pps_vertices *v, size_t n, const uint32_t *slot_in,
              const pps_output *out, void *stream);

/*
 * pps_filter: the whole frame in one persistent cooperative launch: build,
 * insert, [blend if blend != 0], query and the per-frame clear, separated by
 * grid-wide barriers, with each vertex's cell index kept on chip (shared
 * memory) or, for large n, in a library-owned scratch buffer.  Results equal
 * pps_build + pps_insert + [pps_blend] + pps_query.  The table is left ready
 * for the next frame.  Errors: PPS_EINVAL, PPS_ENOMEM, PPS_ECUDA.
 */
int pps_filter(pps_table *t, const pps_camera *cam, uint32_t frame, const pps_vertices *v,
               size_t n, int blend, float alpha, const pps_output *out, void *stream);

/*
 * pps_filter_host: pps_filter on HOST arrays (pinned or pageable): copies the
 * nine input arrays to library-owned device buffers, filters, copies r, g, b
 * (and count / status when non-NULL) back, and synchronizes `stream`.
 * `v->id`, `v->dist` and `v->extra` must be NULL.  Errors: as pps_filter.
 */
int pps_filter_host(pps_table *t, const pps_camera *cam, uint32_t frame,
                    const pps_vertices *v_host, size_t n, int blend, float alpha,
                    const pps_output *out_host, void *stream);

/*
 * pps_filter_host_async: pps_filter_host without the final synchronization,
 * for frame loops.  Each call takes one of two library-owned staging slots
 * (alternating) and enqueues: the uploads of the nine input arrays on the
 * table's upload stream, once that slot's previous outputs are home; the
 * filter on `stream`, once the uploads are done; the downloads of the results
 * on the table's download stream, once the filter is done.  So the uploads of
 * one call overlap the filtering of the previous one and the downloads of the
 * one before.  The host arrays must stay untouched (inputs) and unread
 * (outputs) until pps_host_wait returns; pinned host memory is needed for
 * the copies to run asynchronously (pageable memory works, without overlap).
 * Calls on one table must come from one host thread, in frame order.
 * Errors: as pps_filter_host.
 */
int pps_filter_host_async(pps_table *t, const pps_camera *cam, uint32_t frame,
                          const pps_vertices *v_host, size_t n, int blend, float alpha,
                          const pps_output *out_host, void *stream);

/* pps_host_wait: block until the results of every earlier
 * pps_filter_host_async call on t are in host memory.  Errors: PPS_ECUDA. */
int pps_host_wait(pps_table *t);

/* pps_set_tuning / pps_get_tuning: set or read the launch shape (pps_tuning).
 * Results do not depend on it.  Errors: PPS_EINVAL. */
int pps_set_tuning(pps_table *t, const pps_tuning *tune);
int pps_get_tuning(pps_table *t, pps_tuning *tune);

/*
 * pps_keys: Algorithm 1 alone, for inspection: for each vertex write the full
 * 32-bit home hash h (the home cell is h & (T - 1)) and the fingerprint f
 * (never 0), using the camera and frame of the last pps_build / pps_filter.
 * The table is not touched.  h_out and f_out: n entries each (device).
 * Errors: PPS_EINVAL.
 */
int pps_keys(pps_table *t, const pps_vertices *v, size_t n, uint32_t *h_out, uint32_t *f_out,
             void *stream);

/*
 * pps_filter_noalloc: one frame of the plain filter (FP32 accumulation, no
 * history) that allocates no device memory.  The paper has no counterpart:
 * it serves callers that may not call cudaMalloc when they filter, such as a
 * plug-in whose host application owns the GPU memory budget, or a real-time
 * render thread that must not block on device allocation.  Results equal
 * pps_filter on a table created from `p` (FP32 atomics: equal up to
 * summation order).
 *  - Working memory is one static device array inside the library (about
 *    26 MB), held by every GPU that loads the library until the process exits.
 *    Limits: log2_slots <= 20 and n <= 524,288; larger requests, another
 *    accum_mode, or a history return PPS_EINVAL.
 *  - The first call in a CUDA context (the device's primary context, that
 *    device current) looks up the array's device address with
 *    cudaGetSymbolAddress; make that first call before any stream capture.  A
 *    context created later on the same device (after cudaDeviceReset) looks
 *    it up again on its first call.
 *  - All calls share the array and each starts by clearing what it uses; two
 *    calls that overlap on the GPU (streams not ordered) race and give wrong
 *    results.
 *  - The call's counters and device error word stay in the array until the
 *    next call clears them: read them with pps_noalloc_stats in between.
 * Arguments as for pps_params / pps_filter; every pointer is the caller's.
 * Errors: PPS_EINVAL (the checks of pps_create, and the limits above),
 * PPS_ECUDA.
 */
int pps_filter_noalloc(const pps_params *p, const pps_camera *cam, uint32_t frame,
                       const pps_vertices *v, size_t n, const pps_output *out, void *stream);

/*
 * pps_noalloc_stats: synchronize `stream` and read what the last
 * pps_filter_noalloc left in the library's static array: frame_cells,
 * overflow_vertices, vertices and device_error (the other fields are 0).  No
 * paper counterpart; like pps_filter_noalloc it allocates nothing.  Call it
 * after a pps_filter_noalloc and before the next one, on a stream ordered
 * after it.  Returns PPS_EDEVICE (message naming the bits) when a kernel
 * raised the device error word -- a grid-barrier timeout, say -- so that a
 * frame that went wrong on the GPU is not taken for a good one; the word is
 * then cleared.  Errors: PPS_EINVAL (out NULL), PPS_ECUDA, PPS_EDEVICE.
 */
int pps_noalloc_stats(pps_stats_t *out, void *stream);

/*
 * pps_stats: synchronize `stream` and read the table's counters.  Returns
 * PPS_EDEVICE if a kernel raised the device error word (the word is then
 * cleared).
 */
int pps_stats(pps_table *t, pps_stats_t *out, void *stream);

/*
 * pps_table_dump: synchronize `stream` and copy the table to host memory:
 * fp_host[T] fingerprints (0 = empty); acc_host (nullable) the accumulators as
 * 4 floats per cell {sum r, sum g, sum b, count} (FP32 mode) or 4 int64
 * {sum r, sum g, sum b, count} (fixed mode).  T = 2^log2_slots.  Used to audit
 * probe overflow and for inspection.  Errors: PPS_EINVAL, PPS_ECUDA.
 */
int pps_table_dump(pps_table *t, uint32_t *fp_host, void *acc_host, void *stream);

/* ---- batched views ------------------------------------------------------ */
/*
 * Several views (cameras) filtered in one persistent launch: every view keeps
 * its own table (own size, probe limit, history), camera and vertex batch
 * (Sec. 3 per view); the tiles of all views are handed out from one counter so
 * that views of uneven size share the GPU, and the launch is replayed from a
 * CUDA graph.
 *
 *  pps_view   table: the view's table; v, n: its vertices (device); out: its
 *             results (device; count and status optional).
 *
 * pps_batch_create records the launch for these arrays (pointers and sizes are
 * fixed from then on); blend != 0 blends the views whose table keeps a history
 * (alpha as in pps_blend).  While the batch exists, use its tables only
 * through pps_batch_run (and pps_stats / pps_table_dump between runs).
 * pps_batch_run filters one frame of every view: cams[i] is view i's camera,
 * `frame` the jitter key word; it may wait for the run two calls back.
 * Errors: PPS_EINVAL, PPS_ESTATE, PPS_ENOMEM, PPS_ECUDA.
 */
typedef struct pps_view {
  pps_table *table;
  pps_vertices v;
  size_t n;
  pps_output out;
} pps_view;

typedef struct pps_batch pps_batch;

int pps_batch_create(pps_batch **out, const pps_view *views, uint32_t nviews, int blend,
                     float alpha);
int pps_batch_run(pps_batch *b, const pps_camera *cams, uint32_t frame, void *stream);
int pps_batch_destroy(pps_batch *b);

/* ---- learned fallback --------------------------------------------------- */
/*
 * A small network that answers for vertices whose cell holds too few samples
 * (the low-density case of Sec. 3.3), trained online on the averages of
 * well-populated cells that the filter itself produces.  Input: per axis
 * sin/cos(pi 2^k p), k = 0..11, of the position normalized to the box (72),
 * the unit normal (3), 5 zeros; three hidden layers of 64 with ReLU; linear
 * RGB out.  BF16 weights and activations, FP32 accumulation (tensor cores).
 * Loss 1/(2 batch) sum (y - t)^2; Adam on FP32 master weights.
 *
 * Parameter vector (13,699 floats, this order): W1 [64][80], b1 [64],
 * W2 [64][64], b2 [64], W3 [64][64], b3 [64], W4 [3][64], b4 [3] (W as
 * [out][in]).
 *
 *  box_min, box_max   position normalization box (p clamped to [0, 1]^3).
 *  lr, beta1, beta2, eps  Adam.
 *  batch              samples per training step, a multiple of 128.
 *  steps              training steps per pps_mlp_train call.
 *  train_min_count    a vertex is a training sample if its count >= this.
 *  infer_max_count    pps_mlp_infer answers for counts below this.
 *  seed               He initialisation and training-sample selection.
 */
typedef struct pps_mlp_params {
  float box_min[3];
  float box_max[3];
  float lr, beta1, beta2, eps;
  uint32_t batch;
  uint32_t steps;
  uint32_t train_min_count;
  uint32_t infer_max_count;
  uint32_t seed;
  uint32_t reserved[3];
} pps_mlp_params;

typedef struct pps_mlp pps_mlp;

/* pps_mlp_create: allocate a network on the current device; init_host
 * (nullable, 13,699 floats) gives the initial weights, else He initialisation
 * with zero biases from `seed`.  Errors: PPS_EINVAL, PPS_ENOMEM, PPS_ECUDA. */
int pps_mlp_create(pps_mlp **out, const pps_mlp_params *p, const float *init_host);
int pps_mlp_destroy(pps_mlp *m);

/* Set / read the FP32 master weights (host arrays of 13,699 floats); setting
 * also resets the Adam moments and step count.  Both synchronize the device. */
int pps_mlp_set_weights(pps_mlp *m, const float *host, size_t count);
int pps_mlp_get_weights(pps_mlp *m, float *host, size_t count);

/*
 * pps_mlp_train: `steps` Adam steps.  Each step draws `batch` samples: for
 * sample i the first of 16 candidate vertices (Philox4x32-10, key (seed,
 * frame), counter (i, step, try, 0); index = high 32 bits of x0 * n) whose
 * filtered count is >= train_min_count (no candidate: the sample is left
 * out); the target is that vertex's filtered value.  `filtered` holds the
 * filter's per-vertex r, g, b and count (device).
 */
int pps_mlp_train(pps_mlp *m, const pps_vertices *v, size_t n, const pps_output *filtered,
                  uint32_t frame, void *stream);

/* pps_mlp_infer: for every vertex with count < infer_max_count whose status
 * is not OVERFLOW, replace out->r, g, b by the network's prediction and set
 * status PPS_STATUS_MLP.  out->count and out->status are required. */
int pps_mlp_infer(pps_mlp *m, const pps_vertices *v, size_t n, const pps_output *out,
                  void *stream);

/* pps_mlp_forward: the network's prediction for every vertex (device r, g, b). */
int pps_mlp_forward(pps_mlp *m, const pps_vertices *v, size_t n, float *r, float *g, float *b,
                    void *stream);

/* pps_mlp_gradient: the loss gradient (13,699 floats, device) over `batch`
 * samples: vertex idx[i] (-1: left out) with target (tr, tg, tb)[idx[i]],
 * normalised by `batch` (a multiple of 128).  No weights change.  grad_out
 * must be 16-byte aligned (PPS_EINVAL otherwise). */
int pps_mlp_gradient(pps_mlp *m, const pps_vertices *v, const float *tr, const float *tg,
                     const float *tb, const int32_t *idx, uint32_t batch, float *grad_out,
                     void *stream);

/*
 * pps_selftest_wait: exercise one of the library's bounded device waits on a
 * condition that never comes true, so that callers can check that a stuck
 * wait ends with an error status instead of a hang.
 *   kind 0  the persistent kernels' grid barrier, waiting for one CTA more
 *           than the launch has (the barrier of the fused filter);
 *   kind 1  the tensor-core kernels' mbarrier wait, on a phase that no
 *           operation completes (the learned fallback's kernels).
 * The wait gives up after limit_us microseconds (1 .. 2,000,000) and the
 * kernel returns.  *error_word (host) receives the device error word the
 * kernel left: for kind 0 the filter's barrier-timeout bit (1), for kind 1
 * the learned fallback's wait-timeout bit (1); 0 would mean the wait did not
 * give up.  Synchronous on the current device; uses its own device memory.
 * PPS_EINVAL for a bad kind, limit or NULL error_word (checked before any
 * CUDA call).
 */
int pps_selftest_wait(int kind, uint32_t limit_us, uint32_t *error_word);

#ifdef __cplusplus
}
#endif

#endif /* PPS_H */
