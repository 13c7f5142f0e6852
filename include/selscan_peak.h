/*
 * selscan_peak — integer-pipe peak measurement of the GPU (a measurement
 * helper, built as libselscan_peak.so beside the scan library; the paper has
 * no counterpart).  The scan kernels are bound by integer instruction issue,
 * so their roofline is taken against the rates measured here: one operation
 * (LOP3, PRMT, IMNMX, the 16x2 SIMD minimum, POPC, funnel shift, add) in
 * eight independent chains per thread over 64 resident warps on every SM.
 *
 * selscan_peak_int runs the operation `which` for `iters` x 16 chain steps
 * per thread (two launches on the legacy default stream, the second timed
 * with CUDA events; it synchronises), with `scratch` a device buffer of at
 * least selscan_peak_scratch_bytes() bytes (16-byte aligned) that it
 * overwrites.  Returns SELSCAN_PEAK_OK and fills *res, or an error code
 * (bad arguments, or a CUDA call that failed).
 */
#ifndef SELSCAN_PEAK_H
#define SELSCAN_PEAK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SELSCAN_PEAK_OK        0
#define SELSCAN_PEAK_ERR_ARG  -1
#define SELSCAN_PEAK_ERR_CUDA -4

#define SELSCAN_PEAK_LOP3     0   /* lop3.b32 (three-input logic) */
#define SELSCAN_PEAK_PRMT     1   /* prmt.b32 (byte permute) */
#define SELSCAN_PEAK_IMNMX    2   /* min.u32 */
#define SELSCAN_PEAK_VIMNMX2  3   /* min.u16x2 (two 16-bit minima) */
#define SELSCAN_PEAK_POPC     4   /* popc.b32 (+ one add per step) */
#define SELSCAN_PEAK_SHF      5   /* shf.r.wrap.b32 (funnel shift) */
#define SELSCAN_PEAK_IADD3    6   /* add.u32 (+ one add per step) */
#define SELSCAN_PEAK_NUM      7

typedef struct {
    double ops;                  /* integer operations executed by the timed launch */
    double ms;                   /* its duration (CUDA events) */
    double ops_per_s;            /* ops / duration */
    double cycles;               /* SM cycles of the longest CTA (clock64) */
    double ops_per_sm_per_cycle; /* ops / SMs / cycles */
    double clock_mhz_attr;       /* the device's reported clock */
    double clock_mhz_implied;    /* cycles / duration */
    int32_t sms;
    int32_t reserved;
} selscan_peak_result;

size_t selscan_peak_scratch_bytes(void);
int selscan_peak_int(int32_t which, int32_t iters, void *scratch, size_t scratch_bytes,
                     selscan_peak_result *res);

#ifdef __cplusplus
}
#endif

#endif /* SELSCAN_PEAK_H */
