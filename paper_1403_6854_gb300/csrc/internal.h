// Host/device structures shared by the kernels and the C ABI layer.
#pragma once
#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime.h>

#include "../../include/selscan.h"
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
    unsigned char *base;          // nslots * per_warp bytes
    size_t per_warp;
    int cap;                      // pool entries per walk
    int tcap;                     // table rows per walk
    int cap_s, tcap_s;            // on-chip tier sizes (multiples of 32)
    int R;                        // marker-window rows per buffer
    int rowcap, poscap;           // window buffer bytes (rows; positions or map values)
    int bigt;                     // whole-warp group threshold (entries)
    int *err;                     // device error word
};

// pool: live entries never exceed the sample size (disjoint, non-empty member
// masks) and one step at most doubles the pool before it is compacted
__host__ __device__ constexpr int list_cap(int n_total) { return ((2 * n_total + 64) + 31) & ~31; }
// table: live groups have two or more members, one step at most doubles the rows
__host__ __device__ constexpr int table_cap(int n_total) { return ((n_total + 64) + 31) & ~31; }

// marker window: rows per buffer so that one buffer holds about 1 KB of rows
__host__ __device__ constexpr int window_rows(long long ld)
{
    return 1024 / (ld * 8) < 2 ? 2 : (1024 / (ld * 8) > 64 ? 64 : (int)(1024 / (ld * 8)));
}
// one buffer's bytes: R rows (+ up to 8 bytes of alignment), 16-byte multiple
__host__ __device__ constexpr int win_rowcap(int R, long long ld) { return (int)((R * ld * 8 + 8 + 15) & ~15ll); }
// positions (or map values) of R + 2 markers (+ alignment)
__host__ __device__ constexpr int win_poscap(int R) { return ((R + 2) * 8 + 8 + 15) & ~15; }

// bytes of one warp's on-chip slice: pool entries, one table word per row,
// and the marker window (two row buffers, two position and two map buffers,
// two mbarriers)
__host__ __device__ constexpr size_t smem_per_warp(int cap_s, int tcap_s, int rowcap, int poscap)
{
    return (size_t)cap_s * 8 + (size_t)tcap_s * 8 + 2 * (size_t)rowcap + 4 * (size_t)poscap + 16;
}

// bytes of one warp's global slice: pool, one table word and one 16-bit
// row list per row
__host__ __device__ constexpr size_t scratch_per_warp(int n_total)
{
    return ((size_t)list_cap(n_total) * 8 + (size_t)table_cap(n_total) * 10 + 255) & ~(size_t)255;
}

// kernel launchers (kernels.cu)
cudaError_t launch_validate(const long long *pos, const double *gmap, long long m, int32_t *err,
                            cudaStream_t s, int check_map = 1);
cudaError_t launch_core_select(const ScanArgs &a, int mode, unsigned maf_num, unsigned maf_den,
                               int maf_filter, int32_t *n1, int8_t *core_status, cudaStream_t s);
cudaError_t launch_walk(const ScanArgs &a, const ItemSink &sink, const Scratch &sc,
                        int schedule, int warps_per_cta, int ctas, int probe_steps, int fetch,
                        int minb, long long n_items, cudaStream_t s);
// per-core results of cores [k0, k1) (iHH_c = down + up, status, ln ratio)
cudaError_t launch_finalize_ihs(const ItemSink &sink, long long k0, long long k1, double *ihh1,
                                double *ihh0, double *lnratio, int8_t *status, cudaStream_t s);
cudaError_t launch_finalize_xpehh(const ItemSink &sink, long long k0, long long k1, double *ihhA,
                                  double *ihhB, double *lnratio, int8_t *status, cudaStream_t s);
cudaError_t launch_ehh(const ScanArgs &a, long long locus, const Scratch &sc,
                       unsigned long long *S, long long cap, long long *len, int32_t *stop,
                       int8_t *status, double *ihh, unsigned long long *denom, cudaStream_t s);
cudaError_t launch_pack(const uint8_t *hap01, int n, long long m, int hap_major,
                        unsigned long long *rows, long long ld, cudaStream_t s);
int max_ctas_per_sm(int schedule, int warps_per_cta, size_t smem_bytes, int minb);

// Second pass of the per-step walk over the items queued in sink.list2.
cudaError_t launch_pass2(const ScanArgs &a, const ItemSink &sink, const Scratch &sc,
                         int warps_per_cta, int ctas, int minb, cudaStream_t s);

// ---- argument checks and the single-locus report (api.cu), shared by
// selscan_ehh and selscan_ehh_noalloc
bool params_ok(const selscan_params *p);
// Checks the arguments of a single-locus report (n at most max_n) and fills
// the walk arguments and the six walks' scratch layout; the scratch base is
// left null for the caller: scratch_off is where it starts inside a workspace
// of ws_need bytes.  SELSCAN_ERR_UNSUPPORTED when the walks' on-chip slices
// (whose marker window grows with the row stride) exceed one CTA's shared
// memory.
int ehh_prepare(const uint64_t *hap, int64_t ld, int32_t n, int64_t m, const int64_t *pos_bp,
                const double *gmap, int64_t locus, const selscan_params *p,
                const selscan_ehh_out *out, int64_t capacity, int32_t max_n, ScanArgs *a,
                Scratch *sc, size_t *scratch_off, size_t *ws_need);
// Clears the error word, validates positions / map and launches the report.
int ehh_run(const ScanArgs &a, int64_t locus, const selscan_params *p, const Scratch &sc,
            const selscan_ehh_out *out, int64_t capacity, void *stream);

// ---- sorted-sweep walks (sweep.cu)
constexpr int kSplitWarps = 8;       // warps of one split-walk CTA
constexpr int kSweepMaxN = 16383;    // haplotypes the sweep keeps on chip (14-bit counts)

struct SweepArgs {
    ScanArgs a;
    ItemSink sk;
    int n;                   // haplotypes sorted (iHS: n; XPEHH: n_A + n_B)
    int threads;             // threads of one sweep CTA (256 or 512)
    int nch;                 // chunks of cores per direction
    long long B;             // cores per chunk
    int L;                   // markers swept before a chunk's first core
    int R;                   // cores per chunk and stage
    int stage, nstages;
    unsigned short *st;      // per chunk and direction: sorted order, run lengths
    unsigned char *slots;    // [2][nch][R] slots of slot_bytes
    size_t slot_bytes;
    int split_bytes;         // shared memory of one split-walk tile
    int split_tile;          // lanes per split walk: 32 (a warp) or 16 (two walks per warp)
    unsigned char *wscratch; // per split-walk tile: window staging and step lists
    size_t wscratch_bytes;
    int walk_ctas;           // persistent split-walk grid
    unsigned long long *walk_head;   // slot counter of the current walk launch
    int32_t *err;                    // device error word of the call
    void *sweep_done_event;          // optional event after the first stage's sort
};

size_t sweep_smem_bytes(int n, int W, int T, int R);
size_t sweep_slot_bytes(int n, int xpehh);
size_t sweep_state_bytes(int n, int T);
size_t sweep_elements(int n, int T);     // sorted elements of one CTA (n and its padding)
size_t split_smem_per_warp(int n, int xpehh);
size_t split_scratch_per_warp(int n);
int split_walk_ctas(int n, int xpehh, int tile);
cudaError_t launch_sweep_path(const SweepArgs &w, cudaStream_t s);

}  // namespace selscan
