// Host/device structures shared by the kernels and the C ABI layer.
#pragma once
#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime.h>

#include "walk.cuh"

namespace selscan {

// Work queue state in the workspace (device).
struct Queue {
    unsigned long long head;      // next item of the current pass
    unsigned long long n2;        // items appended for the second pass
    unsigned long long pad[14];   // keep counters on separate 128-byte lines
};

// Where one scan's per-item results go.
struct ItemSink {
    int mode;                     // 0 iHS (4 items per core), 1 XPEHH (2 items per core)
    int8_t *core_status;          // [m] (MAF_FILTERED marks cores that are not walked)
    int8_t *item_status;          // [items]
    double *item_ihh;             // [items * 2] (XPEHH: A, B)
    int32_t *stop;                // out->stop  [items]
    unsigned long long *digest;   // out->digest: iHS [items], XPEHH [items * 3]
    uint32_t *list2;              // second-pass items
    uint32_t *key2;               // their sort keys
    uint32_t *sorted2;            // second-pass items sorted longest-first
    uint32_t *bucket;             // [NBUCKET + 1] histogram / offsets
    uint32_t *slotmap;            // plain launch: bitmap of busy global scratch slots
    Queue *q;
};

constexpr int NBUCKET = 256;

// Per-warp scratch layout in global memory.
struct Scratch {
    unsigned char *base;          // nwarps * per_warp bytes
    size_t per_warp;
    int cap;                      // entries per global buffer (>= n_total)
    int gcap;                     // groups per global array
    int cap_s, gcap_s;            // on-chip capacities
};

// bytes of one warp's on-chip slice: two entry buffers + three group arrays
__host__ __device__ inline size_t smem_per_warp(int cap_s, int gcap_s)
{
    size_t b = (size_t)cap_s * 2 * 8 + (size_t)cap_s * 2 * 4 + (size_t)gcap_s * 3 * 4;
    return (b + 15) & ~(size_t)15;
}

// bytes of one warp's global slice: entries never exceed the sample size,
// groups (two or more members each) never exceed half of it
__host__ __device__ constexpr size_t scratch_per_warp(int n_total)
{
    return ((size_t)n_total * 2 * 8 + (size_t)n_total * 2 * 4 + ((size_t)n_total / 2 + 1) * 3 * 4 +
            255) & ~(size_t)255;
}

// kernel launchers (kernels.cu)
cudaError_t launch_validate(const long long *pos, const double *gmap, long long m, int32_t *err,
                            cudaStream_t s);
cudaError_t launch_core_select(const ScanArgs &a, int mode, unsigned maf_num, unsigned maf_den,
                               int maf_filter, int32_t *n1, int8_t *core_status, cudaStream_t s);
cudaError_t launch_walk(const ScanArgs &a, const ItemSink &sink, const Scratch &sc,
                        int schedule, int warps_per_cta, int ctas, int probe_steps,
                        long long n_items, cudaStream_t s);
cudaError_t launch_finalize_ihs(const ItemSink &sink, long long m, double *ihh1, double *ihh0,
                                double *lnratio, int8_t *status, cudaStream_t s);
cudaError_t launch_finalize_xpehh(const ItemSink &sink, long long m, double *ihhA,
                                  double *ihhB, double *lnratio, int8_t *status, cudaStream_t s);
cudaError_t launch_ehh(const ScanArgs &a, long long locus, const Scratch &sc,
                       unsigned long long *S, long long cap, long long *len, int32_t *stop,
                       int8_t *status, double *ihh, unsigned long long *denom, cudaStream_t s);
cudaError_t launch_pack(const uint8_t *hap01, int n, long long m, int hap_major,
                        unsigned long long *rows, long long ld, cudaStream_t s);
int max_ctas_per_sm(int schedule, int warps_per_cta, size_t smem_bytes);

}  // namespace selscan
