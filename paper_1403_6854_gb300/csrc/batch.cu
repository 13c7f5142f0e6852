// Batched scans: several admitted scans (iHS and XPEHH, any sizes) share one
// persistent walk launch ("tick").  The host hands each tick up to
// SELSCAN_BATCH_MAX_UNITS core ranges from up to SELSCAN_BATCH_MAX_SCANS scans;
// the tick walks the concatenation of those ranges, one core per queue fetch
// (neighbouring cores near a sweep all have long walks, so finer fetches
// balance the warps), so walks of different scans run side by side on the
// GPU.  Used by the serving loop for continuous batching; the statistics are
// exactly those of selscan_ihs / selscan_xpehh (same walk code, same
// finalize).  A tick issues no host-to-device copy: the scan descriptors and
// the ranges travel as the kernel's parameter block.
#include <string.h>

#include "../../include/selscan.h"
#include "device_common.cuh"
#include "internal.h"

namespace selscan {
int device_sms();
int max_ctas_per_sm(int schedule, int warps_per_cta, size_t smem_bytes, int minb);
}

using namespace selscan;

namespace {

constexpr int kBatchWarps = 4;
constexpr int kBatchSmemEntries = 512;

struct BatchDesc {
    ScanArgs a;
    ItemSink sk;
    int R;          // window rows per buffer for this scan's row stride
    int *err;
};

// The whole tick, passed by value as the kernel's parameter block (at most
// 32,764 bytes on this architecture).
struct TickParams {
    BatchDesc d[SELSCAN_BATCH_MAX_SCANS];
    int scan[SELSCAN_BATCH_MAX_UNITS];            // scan of unit u
    long long c0[SELSCAN_BATCH_MAX_UNITS];        // first core of unit u
    long long off[SELSCAN_BATCH_MAX_UNITS + 1];   // tick index of unit u's first core
    int nunits;
    Scratch sc;
    unsigned long long *head;
};
static_assert(sizeof(TickParams) <= 32000, "tick parameter block too large");

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct BatchPlan {
    int ctas, wpc, nslots, carveout;
    Scratch sc;     // base filled at run time
    size_t smem;
};

BatchPlan batch_plan(int max_n_total, long long max_ld)
{
    BatchPlan p;
    p.wpc = kBatchWarps;
    p.sc.cap = list_cap(max_n_total);
    p.sc.tcap = table_cap(max_n_total);
    p.sc.cap_s = kBatchSmemEntries;
    p.sc.tcap_s = kBatchSmemEntries / 4;
    p.sc.R = window_rows(max_ld);
    p.sc.rowcap = win_rowcap(p.sc.R, max_ld);   // >= 2 rows of the widest scan
    p.sc.poscap = win_poscap(64);               // narrower scans use up to 64 rows
    p.sc.per_warp = scratch_per_warp(max_n_total);
    p.sc.bigt = 32;
    p.sc.err = nullptr;
    p.sc.base = nullptr;
    p.smem = smem_per_warp(p.sc.cap_s, p.sc.tcap_s, p.sc.rowcap, p.sc.poscap) * (size_t)p.wpc;
    int per_sm = max_ctas_per_sm(SELSCAN_SCHED_IN_ORDER, p.wpc, p.smem, 2);
    if (per_sm < 1) per_sm = 64 / p.wpc;
    p.ctas = device_sms() * per_sm;
    p.nslots = p.ctas * p.wpc;
    // shared memory for the resident CTAs, the rest of the array stays L1
    // (the global tier of the pools goes through it)
    const size_t need = (p.smem + 1024) * (size_t)per_sm;
    const int pct = (int)((need * 100 + 228 * 1024 - 1) / (228 * 1024));
    p.carveout = pct > 100 ? 100 : (pct < 10 ? 10 : pct);
    return p;
}

struct BatchLayout {
    size_t head, scratch, total;
};

BatchLayout batch_layout(int nslots, size_t per_warp)
{
    BatchLayout l;
    size_t o = 0;
    l.head = o;    o += 256;
    l.scratch = o; o += (size_t)nslots * per_warp;
    l.total = o;
    return l;
}

size_t item_bytes_layout(long long m, int mode, size_t *off_ihh)
{
    const long long items = m * (mode == SELSCAN_MODE_XPEHH ? 2 : 4);
    const size_t a = up256((size_t)items);
    if (off_ihh) *off_ihh = a;
    return a + up256((size_t)items * 8 * (mode == SELSCAN_MODE_XPEHH ? 2 : 1));
}

bool scan_ok(const selscan_scan *s)
{
    if (!s || !s->hap || !s->pos_bp || !s->gmap || !s->status || !s->n1 || !s->ihh_a || !s->ihh_b ||
        !s->lnratio || !s->stop || !s->digest || !s->error || !s->items)
        return false;
    if (s->mode != SELSCAN_MODE_IHS && s->mode != SELSCAN_MODE_XPEHH) return false;
    const int nB = s->mode == SELSCAN_MODE_XPEHH ? s->nB : 0;
    if (s->nA < 2 || (s->mode == SELSCAN_MODE_XPEHH && s->nB < 2) || (long long)s->nA + nB > 65000)
        return false;
    if (s->m < 1 || s->m >= (1ll << 30) || s->ld < (s->nA + 63) / 64 + (nB + 63) / 64) return false;
    const selscan_params *p = &s->params;
    if (p->ehh_cut_den == 0 || p->maf_den == 0 || p->gap_scale_bp <= 0 || p->max_gap_bp < 0 ||
        (p->include_crossing_term != 0 && p->include_crossing_term != 1) ||
        (p->use_physical_map != 0 && p->use_physical_map != 1))
        return false;
    return ((uintptr_t)s->items & 255) == 0;
}

BatchDesc make_desc(const selscan_scan *s)
{
    BatchDesc d;
    const int nB = s->mode == SELSCAN_MODE_XPEHH ? s->nB : 0;
    ScanArgs &a = d.a;
    a.hap = (const unsigned long long *)s->hap;
    a.ld = s->ld;
    a.m = s->m;
    a.k0 = 0;                 // ticks name their own core ranges; outputs span the scan
    a.k1 = s->m;
    a.pos = (const long long *)s->pos_bp;
    a.gmap = s->gmap;
    a.WA = (s->nA + 63) / 64;
    a.W = a.WA + (nB + 63) / 64;
    a.nA = s->nA;
    a.nB = nB;
    a.lastA = (s->nA % 64) ? ((1ull << (s->nA % 64)) - 1ull) : ~0ull;
    a.lastB = nB > 0 ? ((nB % 64) ? ((1ull << (nB % 64)) - 1ull) : ~0ull) : ~0ull;
    a.cut_num = s->params.ehh_cut_num;
    a.cut_den = s->params.ehh_cut_den;
    a.gap_scale = s->params.gap_scale_bp;
    a.max_gap = s->params.max_gap_bp;
    a.crossing = s->params.include_crossing_term;
    a.physical = s->params.use_physical_map;
    size_t off_ihh = 0;
    item_bytes_layout(s->m, s->mode, &off_ihh);
    ItemSink &k = d.sk;
    memset(&k, 0, sizeof(k));
    k.mode = s->mode == SELSCAN_MODE_XPEHH ? 1 : 0;
    k.core_status = s->status;
    k.item_status = (int8_t *)s->items;
    k.item_ihh = (double *)((unsigned char *)s->items + off_ihh);
    k.stop = s->stop;
    k.digest = (unsigned long long *)s->digest;
    d.R = 2;
    d.err = s->error;
    return d;
}

}  // namespace

namespace selscan {

__global__ void __launch_bounds__(256, 2) walk_batch_kernel(const __grid_constant__ TickParams t)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const long long gw = (long long)blockIdx.x * wpc + warp;
    WarpBufs b = make_bufs(smem + (size_t)warp * slice_bytes(t.sc),
                           t.sc.base + (size_t)gw * t.sc.per_warp, t.sc);
    init_window(b);
    unsigned wpar[2] = {0u, 0u};
    const unsigned long long total = (unsigned long long)t.off[t.nunits];
    int u = 0;
    for (;;) {
        unsigned long long idx = 0;
        if (lane == 0) idx = atomicAdd(t.head, 1ull);
        idx = __shfl_sync(FULLMASK, idx, 0);
        if (idx >= total) break;
        // a warp's fetches increase, so its unit only moves forward
        while (idx >= (unsigned long long)t.off[u + 1]) ++u;
        const BatchDesc &d = t.d[t.scan[u]];
        const long long c = t.c0[u] + (long long)(idx - (unsigned long long)t.off[u]);
        if (d.sk.core_status[c] == (int8_t)SELSCAN_LOCUS_MAF_FILTERED) continue;
        b.R = d.R;
        b.err = d.err;
        // a timed-out window wait stops this warp (the tick's results are void)
        if (d.sk.mode == 1) {
            for (int q = 0; q < 2; ++q)
                if (!run_item<2>(d.a, d.sk, b, (uint32_t)(c * 2 + q), 0, wpar)) return;
        } else {
            for (int q = 0; q < 4; ++q)
                if (!run_item<1>(d.a, d.sk, b, (uint32_t)(c * 4 + q), 0, wpar)) return;
        }
    }
}

}  // namespace selscan

extern "C" {

size_t selscan_batch_item_bytes(int64_t m, int32_t mode)
{
    if (m < 1 || (mode != SELSCAN_MODE_IHS && mode != SELSCAN_MODE_XPEHH)) return 0;
    return item_bytes_layout(m, mode, nullptr);
}

size_t selscan_batch_workspace_bytes(int32_t max_n_total, int64_t max_ld, int32_t max_scans,
                                     int32_t max_units)
{
    if (max_n_total < 2 || max_ld < 1 || max_scans < 1 || max_units < 1 ||
        max_scans > SELSCAN_BATCH_MAX_SCANS || max_units > SELSCAN_BATCH_MAX_UNITS)
        return 0;
    // slots for the most warps an SM can hold, independent of the launch shape
    return batch_layout(device_sms() * 64, scratch_per_warp(max_n_total)).total;
}

int selscan_batch_prepare(const selscan_scan *s, void *stream)
{
    if (!scan_ok(s)) return SELSCAN_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const BatchDesc d = make_desc(s);
    size_t off_ihh = 0;
    const size_t ib = item_bytes_layout(s->m, s->mode, &off_ihh);
    if (cudaMemsetAsync(s->items, 0, ib, st) != cudaSuccess) return SELSCAN_ERR_CUDA;
    if (cudaMemsetAsync(s->error, 0, sizeof(int32_t), st) != cudaSuccess) return SELSCAN_ERR_CUDA;
    if (launch_validate((const long long *)s->pos_bp, s->gmap, s->m, s->error, st,
                        !s->params.use_physical_map) != cudaSuccess)
        return SELSCAN_ERR_CUDA;
    if (launch_core_select(d.a, d.sk.mode, s->params.maf_num, s->params.maf_den,
                           s->params.xpehh_maf_filter, s->n1, s->status, st) != cudaSuccess)
        return SELSCAN_ERR_CUDA;
    return SELSCAN_OK;
}

int selscan_batch_run(const selscan_scan *scans, int32_t nscans, const int32_t *unit_scan,
                      const int64_t *unit_c0, const int64_t *unit_c1, int32_t nunits,
                      int32_t max_n_total, int64_t max_ld, void *workspace, size_t ws_bytes,
                      void *stream)
{
    if (!scans || nscans < 1 || nscans > SELSCAN_BATCH_MAX_SCANS || !unit_scan || !unit_c0 ||
        !unit_c1 || nunits < 0 || nunits > SELSCAN_BATCH_MAX_UNITS || !workspace)
        return SELSCAN_ERR_INVALID_ARG;
    if (nunits == 0) return SELSCAN_OK;
    BatchPlan plan = batch_plan(max_n_total, max_ld);
    const BatchLayout l = batch_layout(plan.nslots, plan.sc.per_warp);
    if (ws_bytes < l.total || ((uintptr_t)workspace & 255)) return SELSCAN_ERR_WORKSPACE;
    // static: the block is large, and it is consumed by the launch below
    // before this function returns
    static thread_local TickParams t;
    for (int i = 0; i < nscans; ++i) {
        const selscan_scan *s = scans + i;
        const int nB = s->mode == SELSCAN_MODE_XPEHH ? s->nB : 0;
        if (!scan_ok(s) || s->nA + nB > max_n_total || s->ld > max_ld) return SELSCAN_ERR_INVALID_ARG;
        t.d[i] = make_desc(s);
        int R = (plan.sc.rowcap - 16) / (int)(s->ld * 8);
        t.d[i].R = R < 2 ? 2 : (R > 64 ? 64 : R);
    }
    long long off = 0;
    for (int u = 0; u < nunits; ++u) {
        const int si = unit_scan[u];
        if (si < 0 || si >= nscans || unit_c0[u] < 0 || unit_c1[u] < unit_c0[u] || unit_c1[u] > scans[si].m)
            return SELSCAN_ERR_INVALID_ARG;
        t.scan[u] = si;
        t.c0[u] = unit_c0[u];
        t.off[u] = off;
        off += unit_c1[u] - unit_c0[u];
    }
    t.off[nunits] = off;
    t.nunits = nunits;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *ws = (unsigned char *)workspace;
    plan.sc.base = ws + l.scratch;
    t.sc = plan.sc;
    t.head = (unsigned long long *)(ws + l.head);
    if (cudaMemsetAsync(ws + l.head, 0, 256, st) != cudaSuccess) return SELSCAN_ERR_CUDA;
    if (cudaFuncSetAttribute(walk_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)plan.smem) != cudaSuccess ||
        cudaFuncSetAttribute(walk_batch_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             plan.carveout) != cudaSuccess)
        return SELSCAN_ERR_CUDA;
    walk_batch_kernel<<<plan.ctas, plan.wpc * 32, plan.smem, st>>>(t);
    return cudaGetLastError() == cudaSuccess ? SELSCAN_OK : SELSCAN_ERR_CUDA;
}

int selscan_batch_finalize(const selscan_scan *s, void *stream)
{
    if (!scan_ok(s)) return SELSCAN_ERR_INVALID_ARG;
    const BatchDesc d = make_desc(s);
    cudaError_t e;
    if (s->mode == SELSCAN_MODE_XPEHH)
        e = launch_finalize_xpehh(d.sk, 0, s->m, s->ihh_a, s->ihh_b, s->lnratio, s->status,
                                  (cudaStream_t)stream);
    else
        e = launch_finalize_ihs(d.sk, 0, s->m, s->ihh_a, s->ihh_b, s->lnratio, s->status,
                                (cudaStream_t)stream);
    return e == cudaSuccess ? SELSCAN_OK : SELSCAN_ERR_CUDA;
}

}  // extern "C"
