// C ABI of the scan library (see include/selscan.h for the contract).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/selscan.h"
#include "internal.h"

namespace selscan {
int device_sms();
}

using namespace selscan;

namespace selscan {

bool params_ok(const selscan_params *p)
{
    return p && p->ehh_cut_den > 0 && p->maf_den > 0 && p->gap_scale_bp > 0 && p->max_gap_bp >= 0 &&
           (p->include_crossing_term == 0 || p->include_crossing_term == 1) &&
           (p->use_physical_map == 0 || p->use_physical_map == 1);
}

}  // namespace selscan

namespace {

constexpr int kDefaultWarpsPerCta = 8;
constexpr int kDefaultSmemEntries = 512;
constexpr int kDefaultProbeSteps = 48;
constexpr int kDefaultBigGroup = 32;
constexpr int kMaxHaplotypes = 65000;
constexpr int kDefaultSweepWarmup = 1536;
constexpr int kDefaultSplitTile = 32;
constexpr size_t kSweepSlotBudget = (size_t)24 << 30;  // bytes of sweep slots per scan
constexpr long long kSweepMinMarkers = 32768;          // default sweep: m >= this +
constexpr long long kSweepMinPerHaplotype = 4;         // this x n
constexpr size_t kMaxSmemPerCta = 227 * 1024;

struct SweepPlan {
    int nch, L, R, nstages, threads;
    long long B;
    size_t state_bytes, slot_bytes;
    int split_bytes;
    int split_tile;           // lanes per split walk (32 or 16)
    int walk_ctas;
    size_t wscratch_bytes;    // per split-walk tile
};

struct Plan {
    int schedule;
    SweepPlan sw;
    int wpc;            // warps per CTA of the walk kernel
    int ctas;           // persistent grid size
    int nslots;         // global scratch slices (warps)
    int cap_s, tcap_s;
    int probe;
    int R, rowcap, poscap;
    int fetch;
    int minb;
    int bigt;
};

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }


SweepPlan make_sweep_plan(int n_total, long long m, int mode, const selscan_launch *L)
{
    SweepPlan w;
    w.L = (L && L->sweep_warmup > 0) ? L->sweep_warmup : kDefaultSweepWarmup;
    if (w.L < 16) w.L = 16;
    if (w.L > 16384) w.L = 16384;
    w.R = (L && L->sweep_stage_cores > 0) ? L->sweep_stage_cores : 0;
    if (w.R > 8192) w.R = 8192;
    // chunks are at least as long as their warm-up
    const long long per = w.L > 256 ? w.L : 256;
    long long nch = (m + per - 1) / per;
    const int sms = device_sms();
    // sorting CTA width, for a small sample the narrowest of 32 / 64 / 128 /
    // 256 threads that keeps it at about g elements per thread: g = 8 while
    // every chunk runs at once anyway (a marker's latency is what counts: one
    // warp sorting 8 elements a lane beats eight warps sorting mostly padding,
    // and loses with 16), g = 16 when the chromosome has more chunks than three
    // 256-thread CTAs per SM hold (narrow CTAs then run more, shorter chunks at
    // once).  Larger samples: 256 threads up to 6,144 haplotypes, else 512
    const int want = L ? L->sweep_threads : 0;
    const long long g = nch > (3ll * sms) / 2 ? 16 : 8;
    if (want == 32 || want == 64 || want == 128 || want == 256 || want == 512) w.threads = want;
    else if (n_total <= 128 * g)
        w.threads = n_total <= 32 * g ? 32 : n_total <= 64 * g ? 64 : 128;
    else w.threads = n_total <= 256 * 24 ? 256 : 512;
    // a thread's allele bits live in one 32-bit word: at most 32 elements per thread
    while (w.threads < 512 && n_total > w.threads * 32) w.threads *= 2;
    // the resident sweep CTAs split over both directions: three 256-thread
    // CTAs per SM, two of 512, sixteen warps of the narrow widths
    int per_sm = w.threads == 512 ? 2 : (w.threads == 256 ? 3 : 512 / w.threads);
    const int want_sm = L ? L->sweep_ctas_per_sm : 0;
    if (want_sm > 0 && w.threads >= 256) per_sm = want_sm < 2048 / w.threads ? want_sm : 2048 / w.threads;
    const int nmax = (per_sm * sms) / 2;
    if (nch > nmax) nch = nmax;
    if (nch < 1) nch = 1;
    // run lengths are 16-bit: a chunk plus its warm-up stays below 65,000 markers
    const long long maxB = 65000 - w.L;
    if ((m + nch - 1) / nch > maxB) nch = (m + maxB - 1) / maxB;
    w.nch = (int)nch;
    w.B = (m + nch - 1) / nch;
    const int xp = mode == SELSCAN_MODE_XPEHH;
    w.state_bytes = sweep_state_bytes(n_total, w.threads);
    w.slot_bytes = sweep_slot_bytes(n_total, xp);
    if (w.R <= 0) {
        // default stage: the whole chunk if its slots fit the slot budget,
        // else as many cores as fit (fewer, longer stages launch less)
        const long long fit = (long long)(kSweepSlotBudget / ((size_t)2 * w.nch * w.slot_bytes));
        long long r = w.B < fit ? w.B : fit;
        if (r > 8192) r = 8192;
        if (r < 16) r = 16;
        w.R = (int)r;
    }
    w.nstages = (int)((w.B + w.R - 1) / w.R);
    w.split_bytes = (int)split_smem_per_warp(n_total, xp);
    w.split_tile = (L && (L->sweep_split_tile == 16 || L->sweep_split_tile == 32))
                       ? L->sweep_split_tile : kDefaultSplitTile;
    w.walk_ctas = split_walk_ctas(n_total, xp, w.split_tile);
    w.wscratch_bytes = split_scratch_per_warp(n_total);
    return w;
}

// The schedule of a default launch: the sorted sweep once the chromosome is
// long enough for its chunks' sequential sorts (each about B + warm-up
// markers, n elements per marker) to cost less than walking every step, the
// in-order per-step schedule otherwise.  The crossover depends on the walk
// lengths: on mosaics of n / 25 founders (long walks) about 7k markers at
// n = 100, 12k at 1,000, 23k at 2,000 and 30k at 5,000; on a 22k-marker
// chromosome with short walks the per-step walk is still 2-4x faster.  The
// rule sits above both.
int default_schedule(int mode, long long n_total, long long m)
{
    if (mode == SELSCAN_MODE_EHH || n_total < 2 || n_total > kSweepMaxN) return SELSCAN_SCHED_IN_ORDER;
    return m >= kSweepMinMarkers + kSweepMinPerHaplotype * n_total ? SELSCAN_SCHED_SWEEP
                                                                   : SELSCAN_SCHED_IN_ORDER;
}

Plan make_plan(int mode, long long ld, const selscan_launch *L, int n_total = 0, long long m = 0)
{
    Plan p;
    p.schedule = (L && L->schedule != SELSCAN_SCHED_DEFAULT) ? L->schedule
                                                              : default_schedule(mode, n_total, m);
    if (p.schedule < 0 || p.schedule > SELSCAN_SCHED_SWEEP) p.schedule = -1;
    memset(&p.sw, 0, sizeof(p.sw));
    if (p.schedule == SELSCAN_SCHED_SWEEP) {
        if (mode == SELSCAN_MODE_EHH || n_total > kSweepMaxN || n_total < 2 || m < 1)
            p.schedule = SELSCAN_SCHED_IN_ORDER;
        else
            p.sw = make_sweep_plan(n_total, m, mode, L);
    }
    p.cap_s = (L && L->smem_entries > 0) ? L->smem_entries : kDefaultSmemEntries;
    if (p.cap_s > 8192) p.cap_s = 8192;
    p.cap_s = (p.cap_s + 31) & ~31;
    p.tcap_s = ((p.cap_s / 4) + 31) & ~31;
    p.probe = (L && L->probe_steps > 0) ? L->probe_steps : kDefaultProbeSteps;
    p.R = (L && L->window_rows > 0) ? (L->window_rows < 2 ? 2 : (L->window_rows > 64 ? 64 : L->window_rows))
                                     : window_rows(ld);
    p.fetch = (L && L->cores_per_fetch > 0) ? (L->cores_per_fetch > 1024 ? 1024 : L->cores_per_fetch) : 1;
    p.minb = (L && L->min_ctas_per_sm == 3) ? 3 : 2;
    p.bigt = (L && L->big_group_entries > 0) ? L->big_group_entries : kDefaultBigGroup;
    p.rowcap = win_rowcap(p.R, ld);
    p.poscap = win_poscap(p.R);
    const int sms = device_sms();
    if (mode == SELSCAN_MODE_EHH) {
        p.schedule = SELSCAN_SCHED_IN_ORDER;
        p.wpc = 6;
        p.ctas = 1;
        p.nslots = 6;
        return p;
    }
    const int ipc = mode == SELSCAN_MODE_XPEHH ? 2 : 4;
    if (p.schedule == SELSCAN_SCHED_PLAIN) {
        // one scratch slot per warp an SM can ever hold (64): a resident warp
        // always finds a free slot, whatever the kernel's occupancy
        p.wpc = ipc;
        p.ctas = 0;
        p.nslots = sms * 64;
        return p;
    }
    p.wpc = (L && L->warps_per_cta > 0) ? L->warps_per_cta : kDefaultWarpsPerCta;
    if (p.wpc > 8) p.wpc = 8;
    const size_t smem = smem_per_warp(p.cap_s, p.tcap_s, p.rowcap, p.poscap) * (size_t)p.wpc;
    // the sweep schedule's second pass is an in-order persistent launch
    const int psched = p.schedule == SELSCAN_SCHED_SWEEP ? SELSCAN_SCHED_IN_ORDER : p.schedule;
    int per_sm = max_ctas_per_sm(psched, p.wpc, smem, p.minb);
    if (per_sm < 1) per_sm = 64 / p.wpc > 0 ? 64 / p.wpc : 1;
    int want = (L && L->ctas_per_sm > 0) ? L->ctas_per_sm : per_sm;
    if (want > per_sm) want = per_sm;
    p.ctas = sms * want;
    p.nslots = p.ctas * p.wpc;
    return p;
}

struct Layout {
    size_t queue, slotmap, item_status, item_ihh, list2, key2, sorted2, bucket, scratch, total;
    size_t per_warp;
    size_t sweep_state, sweep_slots, sweep_head, sweep_wscratch;
};

Layout make_layout(int n_total, long long m, int mode, int nslots, const SweepPlan *sw = nullptr)
{
    Layout l;
    const long long items = mode == SELSCAN_MODE_EHH ? 0 : m * (mode == SELSCAN_MODE_XPEHH ? 2 : 4);
    size_t o = 0;
    l.queue = o;        o += up256(sizeof(Queue));
    l.slotmap = o;      o += up256(((size_t)nslots + 31) / 32 * 4);
    l.item_status = o;  o += up256((size_t)items);
    l.item_ihh = o;     o += up256((size_t)items * 8 * (mode == SELSCAN_MODE_XPEHH ? 2 : 1));
    l.list2 = o;        o += up256((size_t)items * 4);
    l.key2 = o;         o += up256((size_t)items * 4);
    l.sorted2 = o;      o += up256((size_t)items * 4);
    l.bucket = o;       o += up256((NBUCKET + 1) * 4);
    l.per_warp = scratch_per_warp(n_total);
    l.scratch = o;      o += (size_t)nslots * l.per_warp;
    l.sweep_state = l.sweep_slots = l.sweep_head = l.sweep_wscratch = 0;
    if (sw && sw->nch > 0) {
        l.sweep_head = o;     o += 256;
        l.sweep_state = o;    o += up256((size_t)2 * sw->nch * sw->state_bytes);
        l.sweep_slots = o;    o += up256((size_t)2 * sw->nch * sw->R * sw->slot_bytes);
        l.sweep_wscratch = o;
        o += (size_t)sw->walk_ctas * (kSplitWarps * 32 / sw->split_tile) * sw->wscratch_bytes;
    }
    l.total = o;
    return l;
}

inline unsigned long long last_mask(int n)
{
    return (n % 64) ? ((1ull << (n % 64)) - 1ull) : ~0ull;
}

ScanArgs make_args(const uint64_t *hap, int64_t ld, int nA, int nB, int64_t m, const int64_t *pos,
                   const double *gmap, const selscan_params *p)
{
    ScanArgs a;
    a.hap = (const unsigned long long *)hap;
    a.ld = ld;
    a.m = m;
    a.pos = (const long long *)pos;
    a.gmap = gmap;
    a.WA = (nA + 63) / 64;
    a.W = a.WA + (nB + 63) / 64;
    a.nA = nA;
    a.nB = nB;
    a.lastA = last_mask(nA);
    a.lastB = nB > 0 ? last_mask(nB) : ~0ull;
    a.cut_num = p->ehh_cut_num;
    a.cut_den = p->ehh_cut_den;
    a.gap_scale = p->gap_scale_bp;
    a.max_gap = p->max_gap_bp;
    a.crossing = p->include_crossing_term;
    a.physical = p->use_physical_map;
    return a;
}

Scratch make_scratch(unsigned char *ws, const Layout &l, int n_total, const Plan &p)
{
    Scratch sc;
    sc.base = ws ? ws + l.scratch : nullptr;
    sc.per_warp = l.per_warp;
    sc.cap = list_cap(n_total);
    sc.tcap = table_cap(n_total);
    sc.cap_s = p.cap_s;
    sc.tcap_s = p.tcap_s;
    sc.R = p.R;
    sc.rowcap = p.rowcap;
    sc.poscap = p.poscap;
    sc.bigt = p.bigt;
    return sc;
}

// Device pointer to element -k of p: the kernels index per-core outputs by
// the global core k in [k0, k1), and an output array of k1 - k0 entries starts
// at core k0.  Only addresses of the caller's array are ever formed from it.
template <typename T>
inline T *at_core(T *p, long long k, long long per_core = 1)
{
    return (T *)((uintptr_t)p - (uintptr_t)(k * per_core) * sizeof(T));
}

// One scan of the cores [k0, k1) of an m-marker chromosome (a whole scan: k0
// = 0, k1 = m).  Outputs hold k1 - k0 cores; the plan and the workspace are
// those of a scan of k1 - k0 cores; walks still reach every marker.
int run_scan(int mode, const uint64_t *hap, int64_t ld, int32_t nA, int32_t nB, int64_t m,
             int64_t k0, int64_t k1, const int64_t *pos, const double *gmap,
             const selscan_params *p, int8_t *status, int32_t *n1, int32_t *stop,
             uint64_t *digest, int32_t *err, double *o1, double *o2, double *lnratio,
             void *workspace, size_t ws_bytes, const selscan_launch *launch, void *stream)
{
    const int n_total = nA + nB;
    const long long ncores = k1 - k0;
    const Plan plan = make_plan(mode, ld, launch, n_total, ncores);
    if (plan.schedule < 0 || (launch && launch->warps_per_cta < 0)) return SELSCAN_ERR_INVALID_ARG;
    if (smem_per_warp(plan.cap_s, plan.tcap_s, plan.rowcap, plan.poscap) * (size_t)plan.wpc > kMaxSmemPerCta)
        return SELSCAN_ERR_UNSUPPORTED;
    const bool sweep = plan.schedule == SELSCAN_SCHED_SWEEP;
    if (sweep && (sweep_smem_bytes(n_total, (nA + 63) / 64 + (nB + 63) / 64, plan.sw.threads, plan.sw.R) > kMaxSmemPerCta ||
                  (size_t)plan.sw.split_bytes * (kSplitWarps * 32 / plan.sw.split_tile) > kMaxSmemPerCta))
        return SELSCAN_ERR_UNSUPPORTED;
    if (sweep && (plan.sw.slot_bytes & 15)) return SELSCAN_ERR_UNSUPPORTED;   // slots are read in 16-byte units
    const Layout l = make_layout(n_total, ncores, mode, plan.nslots, sweep ? &plan.sw : nullptr);
    if (!workspace || ws_bytes < l.total || ((uintptr_t)workspace & 255)) return SELSCAN_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *ws = (unsigned char *)workspace;

    ScanArgs a = make_args(hap, ld, nA, nB, m, pos, gmap, p);
    a.k0 = k0;
    a.k1 = k1;
    const int ipc = mode == SELSCAN_MODE_XPEHH ? 2 : 4;
    status = at_core(status, k0);
    n1 = at_core(n1, k0);
    stop = at_core(stop, k0, ipc);
    digest = at_core(digest, k0, mode == SELSCAN_MODE_XPEHH ? 6 : 4);
    o1 = at_core(o1, k0);
    o2 = at_core(o2, k0);
    lnratio = at_core(lnratio, k0);
    ItemSink sk;
    sk.mode = mode == SELSCAN_MODE_XPEHH ? 1 : 0;
    sk.core_status = status;
    sk.item_status = at_core((int8_t *)(ws + l.item_status), k0, ipc);
    sk.item_ihh = at_core((double *)(ws + l.item_ihh), k0, 4);   // four sums per core either mode
    sk.stop = stop;
    sk.digest = (unsigned long long *)digest;
    sk.list2 = (uint32_t *)(ws + l.list2);
    sk.key2 = (uint32_t *)(ws + l.key2);
    sk.sorted2 = (uint32_t *)(ws + l.sorted2);
    sk.bucket = (uint32_t *)(ws + l.bucket);
    sk.slotmap = (uint32_t *)(ws + l.slotmap);
    sk.q = (Queue *)(ws + l.queue);
    Scratch sc = make_scratch(ws, l, n_total, plan);
    sc.err = err;

    cudaError_t e;
    if ((e = cudaMemsetAsync(ws, 0, l.item_status, s)) != cudaSuccess) return SELSCAN_ERR_CUDA;
    if ((e = cudaMemsetAsync(ws + l.bucket, 0, (NBUCKET + 1) * 4, s)) != cudaSuccess) return SELSCAN_ERR_CUDA;
    if ((e = cudaMemsetAsync(err, 0, sizeof(int32_t), s)) != cudaSuccess) return SELSCAN_ERR_CUDA;
    if (launch_validate((const long long *)pos, gmap, m, err, s, !p->use_physical_map) != cudaSuccess)
        return SELSCAN_ERR_CUDA;
    if (launch_core_select(a, sk.mode, p->maf_num, p->maf_den, p->xpehh_maf_filter, n1, status, s) !=
        cudaSuccess)
        return SELSCAN_ERR_CUDA;
    const int ctas_or_slots = plan.schedule == SELSCAN_SCHED_PLAIN ? plan.nslots : plan.ctas;
    if (launch && launch->walk_begin_event &&
        cudaEventRecord((cudaEvent_t)launch->walk_begin_event, s) != cudaSuccess)
        return SELSCAN_ERR_CUDA;
    if (sweep) {
        SweepArgs w;
        w.a = a;
        w.sk = sk;
        w.n = n_total;
        w.threads = plan.sw.threads;
        w.nch = plan.sw.nch;
        w.B = plan.sw.B;
        w.L = plan.sw.L;
        w.R = plan.sw.R;
        w.stage = 0;
        w.nstages = plan.sw.nstages;
        w.st = (unsigned short *)(ws + l.sweep_state);
        w.slots = ws + l.sweep_slots;
        w.slot_bytes = plan.sw.slot_bytes;
        w.split_bytes = plan.sw.split_bytes;
        w.split_tile = plan.sw.split_tile;
        w.wscratch = ws + l.sweep_wscratch;
        w.wscratch_bytes = plan.sw.wscratch_bytes;
        w.walk_ctas = plan.sw.walk_ctas;
        w.walk_head = (unsigned long long *)(ws + l.sweep_head);
        w.err = err;
        w.sweep_done_event = launch ? launch->sweep_done_event : nullptr;
        if (launch_sweep_path(w, s) != cudaSuccess) return SELSCAN_ERR_CUDA;
        if (launch_pass2(a, sk, sc, plan.wpc, plan.ctas, plan.minb, s) != cudaSuccess)
            return SELSCAN_ERR_CUDA;
    } else if (launch_walk(a, sk, sc, plan.schedule, plan.wpc, ctas_or_slots, plan.probe, plan.fetch,
                           plan.minb, ncores, s) != cudaSuccess) {
        return SELSCAN_ERR_CUDA;
    }
    if (launch && launch->walk_end_event &&
        cudaEventRecord((cudaEvent_t)launch->walk_end_event, s) != cudaSuccess)
        return SELSCAN_ERR_CUDA;
    if (sk.mode == 1)
        e = launch_finalize_xpehh(sk, k0, k1, o1, o2, lnratio, status, s);
    else
        e = launch_finalize_ihs(sk, k0, k1, o1, o2, lnratio, status, s);
    return e == cudaSuccess ? SELSCAN_OK : SELSCAN_ERR_CUDA;
}

}  // namespace

namespace selscan {

int ehh_prepare(const uint64_t *hap, int64_t ld, int32_t n, int64_t m, const int64_t *pos_bp,
                const double *gmap, int64_t locus, const selscan_params *p,
                const selscan_ehh_out *out, int64_t capacity, int32_t max_n, ScanArgs *a,
                Scratch *sc, size_t *scratch_off, size_t *ws_need)
{
    if (!hap || !pos_bp || !gmap || !out || !params_ok(p)) return SELSCAN_ERR_INVALID_ARG;
    if (n < 2 || n > max_n || n > kMaxHaplotypes || m < 1 || m >= (1ll << 30) ||
        ld < (n + 63) / 64 || locus < 0 || locus >= m || capacity < 0)
        return SELSCAN_ERR_INVALID_ARG;
    if ((capacity > 0 && !out->S) || !out->len || !out->stop || !out->status || !out->ihh ||
        !out->denom || !out->error)
        return SELSCAN_ERR_INVALID_ARG;
    const Plan plan = make_plan(SELSCAN_MODE_EHH, ld, nullptr);
    // six walks, each with its on-chip slice (pool, table, marker window): a
    // wide row stride can push the window past the per-CTA limit
    if (smem_per_warp(plan.cap_s, plan.tcap_s, plan.rowcap, plan.poscap) * (size_t)plan.wpc >
        kMaxSmemPerCta)
        return SELSCAN_ERR_UNSUPPORTED;
    const Layout l = make_layout(n, m, SELSCAN_MODE_EHH, plan.nslots);
    *a = make_args(hap, ld, n, 0, m, pos_bp, gmap, p);
    *sc = make_scratch(nullptr, l, n, plan);
    sc->base = nullptr;
    sc->err = out->error;
    *scratch_off = l.scratch;
    *ws_need = l.total;
    return SELSCAN_OK;
}

int ehh_run(const ScanArgs &a, int64_t locus, const selscan_params *p, const Scratch &sc,
            const selscan_ehh_out *out, int64_t capacity, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(out->error, 0, sizeof(int32_t), s) != cudaSuccess) return SELSCAN_ERR_CUDA;
    if (launch_validate(a.pos, a.gmap, a.m, out->error, s, !p->use_physical_map) != cudaSuccess)
        return SELSCAN_ERR_CUDA;
    if (launch_ehh(a, locus, sc, (unsigned long long *)out->S, capacity, (long long *)out->len,
                   out->stop, out->status, out->ihh, (unsigned long long *)out->denom, s) !=
        cudaSuccess)
        return SELSCAN_ERR_CUDA;
    return SELSCAN_OK;
}

}  // namespace selscan

extern "C" {

void selscan_default_params(selscan_params *p)
{
    if (!p) return;
    p->ehh_cut_num = 1;
    p->ehh_cut_den = 20;
    p->maf_num = 1;
    p->maf_den = 20;
    p->gap_scale_bp = 20000;
    p->max_gap_bp = 200000;
    p->include_crossing_term = 0;
    p->xpehh_maf_filter = 0;
    p->use_physical_map = 0;
    p->reserved = 0;
}

size_t selscan_workspace_bytes(int32_t n_total, int64_t m, int32_t mode, const selscan_launch *launch)
{
    if (n_total < 2 || m < 1 || mode < 0 || mode > 2) return 0;
    // scratch slots for the most warps an SM can hold (64), so the size does
    // not depend on the row stride, registers or shared memory of the call
    const Plan p = make_plan(mode, (n_total + 63) / 64, launch, n_total, m);
    const int nslots = mode == SELSCAN_MODE_EHH ? p.nslots : device_sms() * 64;
    return make_layout(n_total, m, mode, nslots,
                       p.schedule == SELSCAN_SCHED_SWEEP ? &p.sw : nullptr).total;
}

int32_t selscan_default_schedule(int32_t n_total, int64_t m, int32_t mode)
{
    if (n_total < 2 || m < 1 || (mode != SELSCAN_MODE_IHS && mode != SELSCAN_MODE_XPEHH)) return -1;
    return default_schedule(mode, n_total, m);
}

int selscan_sweep_work(int32_t n_total, int64_t m, int32_t mode, const selscan_launch *launch,
                       int64_t *marker_passes, int64_t *elements)
{
    if (n_total < 2 || m < 1 || (mode != SELSCAN_MODE_IHS && mode != SELSCAN_MODE_XPEHH) ||
        !marker_passes || !elements)
        return SELSCAN_ERR_INVALID_ARG;
    const Plan p = make_plan(mode, (n_total + 63) / 64, launch, n_total, m);
    if (p.schedule != SELSCAN_SCHED_SWEEP) return SELSCAN_ERR_INVALID_ARG;
    long long passes = 0;
    for (int c = 0; c < p.sw.nch; ++c) {
        const long long c0 = (long long)c * p.sw.B;
        if (c0 >= m) break;
        const long long c1 = c0 + p.sw.B < m ? c0 + p.sw.B : m;
        const long long s0 = c0 - p.sw.L > 0 ? c0 - p.sw.L : 0;
        const long long e0 = c1 - 1 + p.sw.L < m - 1 ? c1 - 1 + p.sw.L : m - 1;
        passes += (c1 - s0) + (e0 - c0 + 1);       // toward lower / higher indices
    }
    *marker_passes = passes;
    *elements = (int64_t)sweep_elements(n_total, p.sw.threads);
    return SELSCAN_OK;
}

int32_t selscan_launch_count(int32_t n_total, int64_t m, int32_t mode, const selscan_launch *launch)
{
    if (n_total < 2 || m < 1 || (mode != SELSCAN_MODE_IHS && mode != SELSCAN_MODE_XPEHH)) return -1;
    const Plan p = make_plan(mode, (n_total + 63) / 64, launch, n_total, m);
    switch (p.schedule) {
    case SELSCAN_SCHED_LONGEST_FIRST: return 8;   // validate, select, probe pass, 3 bucket kernels, pass 2, finalize
    case SELSCAN_SCHED_IN_ORDER:
    case SELSCAN_SCHED_PLAIN: return 4;           // validate, select, walk, finalize
    case SELSCAN_SCHED_SWEEP: return 7 + 2 * p.sw.nstages;   // + sweep and split walk per stage
    default: return -1;
    }
}

int selscan_ihs_range(const uint64_t *hap, int64_t ld, int32_t n, int64_t m, int64_t k0,
                      int64_t k1, const int64_t *pos_bp, const double *gmap,
                      const selscan_params *p, const selscan_ihs_out *out, void *workspace,
                      size_t ws_bytes, const selscan_launch *launch, void *stream)
{
    if (!hap || !pos_bp || !gmap || !out || !params_ok(p)) return SELSCAN_ERR_INVALID_ARG;
    if (n < 2 || n > kMaxHaplotypes || m < 1 || m >= (1ll << 30) || ld < (n + 63) / 64)
        return SELSCAN_ERR_INVALID_ARG;
    if (k0 < 0 || k1 <= k0 || k1 > m) return SELSCAN_ERR_INVALID_ARG;
    if (!out->status || !out->n1 || !out->ihh1 || !out->ihh0 || !out->lnratio || !out->stop ||
        !out->digest || !out->error)
        return SELSCAN_ERR_INVALID_ARG;
    return run_scan(SELSCAN_MODE_IHS, hap, ld, n, 0, m, k0, k1, pos_bp, gmap, p, out->status,
                    out->n1, out->stop, out->digest, out->error, out->ihh1, out->ihh0, out->lnratio,
                    workspace, ws_bytes, launch, stream);
}

int selscan_ihs(const uint64_t *hap, int64_t ld, int32_t n, int64_t m, const int64_t *pos_bp,
                const double *gmap, const selscan_params *p, const selscan_ihs_out *out,
                void *workspace, size_t ws_bytes, const selscan_launch *launch, void *stream)
{
    return selscan_ihs_range(hap, ld, n, m, 0, m, pos_bp, gmap, p, out, workspace, ws_bytes, launch,
                             stream);
}

int selscan_xpehh_range(const uint64_t *hap, int64_t ld, int32_t nA, int32_t nB, int64_t m,
                        int64_t k0, int64_t k1, const int64_t *pos_bp, const double *gmap,
                        const selscan_params *p, const selscan_xpehh_out *out, void *workspace,
                        size_t ws_bytes, const selscan_launch *launch, void *stream)
{
    if (!hap || !pos_bp || !gmap || !out || !params_ok(p)) return SELSCAN_ERR_INVALID_ARG;
    if (nA < 2 || nB < 2 || (long long)nA + nB > kMaxHaplotypes || m < 1 || m >= (1ll << 30) ||
        ld < (nA + 63) / 64 + (nB + 63) / 64)
        return SELSCAN_ERR_INVALID_ARG;
    if (k0 < 0 || k1 <= k0 || k1 > m) return SELSCAN_ERR_INVALID_ARG;
    if (!out->status || !out->n1 || !out->ihhA || !out->ihhB || !out->lnratio || !out->stop ||
        !out->digest || !out->error)
        return SELSCAN_ERR_INVALID_ARG;
    return run_scan(SELSCAN_MODE_XPEHH, hap, ld, nA, nB, m, k0, k1, pos_bp, gmap, p, out->status,
                    out->n1, out->stop, out->digest, out->error, out->ihhA, out->ihhB,
                    out->lnratio, workspace, ws_bytes, launch, stream);
}

int selscan_xpehh(const uint64_t *hap, int64_t ld, int32_t nA, int32_t nB, int64_t m,
                  const int64_t *pos_bp, const double *gmap, const selscan_params *p,
                  const selscan_xpehh_out *out, void *workspace, size_t ws_bytes,
                  const selscan_launch *launch, void *stream)
{
    return selscan_xpehh_range(hap, ld, nA, nB, m, 0, m, pos_bp, gmap, p, out, workspace, ws_bytes,
                               launch, stream);
}

int selscan_ehh(const uint64_t *hap, int64_t ld, int32_t n, int64_t m, const int64_t *pos_bp,
                const double *gmap, int64_t locus, const selscan_params *p,
                const selscan_ehh_out *out, int64_t capacity, void *workspace, size_t ws_bytes,
                void *stream)
{
    ScanArgs a;
    Scratch sc;
    size_t scratch_off = 0, need = 0;
    const int rc = ehh_prepare(hap, ld, n, m, pos_bp, gmap, locus, p, out, capacity, kMaxHaplotypes,
                               &a, &sc, &scratch_off, &need);
    if (rc != SELSCAN_OK) return rc;
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255)) return SELSCAN_ERR_WORKSPACE;
    sc.base = (unsigned char *)workspace + scratch_off;
    return ehh_run(a, locus, p, sc, out, capacity, stream);
}

int selscan_pack(const uint8_t *hap01, int32_t n, int64_t m, int32_t hap_major, uint64_t *rows,
                 int64_t ld, void *stream)
{
    if (!hap01 || !rows || n < 1 || m < 1 || ld < (n + 63) / 64 || (hap_major != 0 && hap_major != 1))
        return SELSCAN_ERR_INVALID_ARG;
    if (launch_pack(hap01, n, m, hap_major, (unsigned long long *)rows, ld, (cudaStream_t)stream) !=
        cudaSuccess)
        return SELSCAN_ERR_CUDA;
    return SELSCAN_OK;
}

const char *selscan_strerror(int code)
{
    switch (code) {
    case SELSCAN_OK: return "ok";
    case SELSCAN_ERR_INVALID_ARG: return "invalid argument";
    case SELSCAN_ERR_UNSORTED: return "positions or genetic map decrease";
    case SELSCAN_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
    case SELSCAN_ERR_CUDA: return "CUDA launch or runtime error";
    case SELSCAN_ERR_TIMEOUT: return "bounded device wait gave up";
    case SELSCAN_ERR_UNSUPPORTED: return "unsupported device or launch shape";
    case SELSCAN_ERR_INTERNAL: return "internal consistency check failed on the device";
    default: return "unknown error code";
    }
}

}  // extern "C"
