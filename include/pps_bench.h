/*
 * pps_bench.h -- measurement helper shipped with the filter library.
 *
 * The paper has no counterpart: this entry point measures the GPU's own rate
 * of random memory operations (the denominator for the filter's L2 atomic
 * traffic), not part of the method.
 */
#ifndef PPS_BENCH_H
#define PPS_BENCH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPS_RATE_RED_V4_F32 0 /* red.add.v4.f32 of 16 bytes                   */
#define PPS_RATE_CAS_B32 1    /* 32-bit compare-and-swap (returns old value)  */
#define PPS_RATE_RED_F32 2    /* scalar float reduction                        */
#define PPS_RATE_GATHER_V4 3  /* 16-byte load at L2 (ld.global.cg)             */

/*
 * pps_bench_rate: time about `ops` operations of `kind`, each on its own
 * randomly chosen 32-byte sector of the device buffer `scratch` (region_bytes
 * long, >= 4096, owned by the caller, contents overwritten), on `stream`; one
 * untimed warm-up launch precedes the timed one.  Writes operations per second
 * to *ops_per_second and synchronizes the stream.
 * Returns 0, 1 (bad argument) or 3 (a CUDA call failed).
 */
int pps_bench_rate(int kind, size_t region_bytes, size_t ops, void *scratch, void *stream,
                   double *ops_per_second);

#ifdef __cplusplus
}
#endif

#endif /* PPS_BENCH_H */
