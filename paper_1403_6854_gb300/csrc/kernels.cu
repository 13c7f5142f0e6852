// Kernels of the EHH / iHS / XPEHH scan (sm_103a).
//
//   validate      positions and map non-decreasing (device error word)
//   core_select   derived count n_1 per marker and the MAF filter (Section 1.2)
//   walk_*        the EHH walks (walk.cuh): persistent with a global queue, or
//                 one CTA per core (plain launch)
//   bucket_*      longest-first ordering of the walks that outlive the probe pass
//   finalize_*    iHH_c = downstream + upstream, status, ln ratio (Eq. 4, Eq. 5)
//   ehh_trace     the single-locus report (Eq. 1, Eq. 3 per step)
//   pack          0/1 bytes -> bit rows
#include <math.h>

#include "../../include/selscan.h"
#include "internal.h"
#include "device_common.cuh"

namespace selscan {

// ------------------------------------------------------------ validate
__global__ void validate_kernel(const long long *pos, const double *gmap, long long m, int32_t *err,
                                int check_map)
{
    for (long long k = 1 + blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m;
         k += (long long)gridDim.x * blockDim.x) {
        if (pos[k] < pos[k - 1] || (check_map && !(gmap[k] >= gmap[k - 1])))
            atomicExch(err, SELSCAN_ERR_UNSORTED);
    }
    if (check_map && blockIdx.x == 0 && threadIdx.x == 0 && m >= 1 && !(gmap[0] == gmap[0]))
        atomicExch(err, SELSCAN_ERR_UNSORTED);
}

cudaError_t launch_validate(const long long *pos, const double *gmap, long long m, int32_t *err,
                            cudaStream_t s, int check_map)
{
    long long blocks = (m + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    validate_kernel<<<(unsigned)blocks, 256, 0, s>>>(pos, gmap, m, err, check_map);
    return cudaGetLastError();
}

// ------------------------------------------------------------ core select
// A warp counts the derived alleles of kCoreRows rows at once: lane l reads the
// 64-bit words l, l + 32, ... of each of them, all of a round's loads issued
// before the popcounts, then one warp sum per row.
constexpr int kCoreRows = 4;
__global__ void core_select_kernel(ScanArgs a, int mode, unsigned maf_num, unsigned maf_den,
                                   int maf_filter, int32_t *n1, int8_t *core_status)
{
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned n_total = (unsigned)(a.nA + a.nB);
    const unsigned long long *hap = (const unsigned long long *)a.hap;
    for (long long k0 = a.k0 + warp * kCoreRows; k0 < a.k1; k0 += nw * kCoreRows) {
        unsigned c[kCoreRows];
#pragma unroll
        for (int r = 0; r < kCoreRows; ++r) c[r] = 0u;
        for (int w = lane; w < a.W; w += 32) {
            const unsigned long long vm = (unsigned long long)valid32(a, 2 * w) |
                                          ((unsigned long long)valid32(a, 2 * w + 1) << 32);
            unsigned long long v[kCoreRows];
#pragma unroll
            for (int r = 0; r < kCoreRows; ++r)
                v[r] = k0 + r < a.k1 ? __ldg(hap + (k0 + r) * a.ld + w) : 0ull;
#pragma unroll
            for (int r = 0; r < kCoreRows; ++r) c[r] += (unsigned)__popcll(v[r] & vm);
        }
#pragma unroll
        for (int r = 0; r < kCoreRows; ++r) {
            const unsigned cr = __reduce_add_sync(FULLMASK, c[r]);
            const long long k = k0 + r;
            if (lane == 0 && k < a.k1) {
                n1[k] = (int32_t)cr;
                const unsigned minor = cr < n_total - cr ? cr : n_total - cr;
                const bool filt = (mode == 0 || maf_filter) &&
                                  (unsigned long long)maf_den * minor < (unsigned long long)maf_num * n_total;
                core_status[k] = filt ? (int8_t)SELSCAN_LOCUS_MAF_FILTERED : (int8_t)0;
            }
        }
    }
}

cudaError_t launch_core_select(const ScanArgs &a, int mode, unsigned maf_num, unsigned maf_den,
                               int maf_filter, int32_t *n1, int8_t *core_status, cudaStream_t s)
{
    const long long warps = (a.k1 - a.k0 + kCoreRows - 1) / kCoreRows;
    long long blocks = (warps * 32 + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    core_select_kernel<<<(unsigned)blocks, 256, 0, s>>>(a, mode, maf_num, maf_den, maf_filter,
                                                         n1, core_status);
    return cudaGetLastError();
}

// ------------------------------------------------------------ walks
// Persistent walk kernel.  pass 1: items in core order (a warp takes one
// core's items per queue fetch), optionally capped at max_steps; pass 2:
// the sorted list of walks the first pass left unfinished, one per fetch.
// MINB: resident 8-warp CTAs per SM the build is compiled for (register cap
// 65536 / (256 * MINB)): 2 (128 registers) or 3 (85 registers)
template <int NPOP, int MINB>
__global__ void __launch_bounds__(256, MINB) walk_persistent_kernel(ScanArgs a, ItemSink sk, Scratch sc,
                                                              long long n_cores, int pass,
                                                              int max_steps, int fetch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const long long gw = (long long)blockIdx.x * wpc + warp;
    WarpBufs b = make_bufs(smem + (size_t)warp * slice_bytes(sc),
                           sc.base + (size_t)gw * sc.per_warp, sc);
    init_window(b);
    unsigned wpar[2] = {0u, 0u};
    const int ipc = NPOP == 2 ? 2 : 4;
    const unsigned long long total = pass == 2 ? sk.q->n2 : (unsigned long long)n_cores;
    const unsigned long long step = pass == 2 ? 1ull : (unsigned long long)fetch;
    for (;;) {
        unsigned long long idx = 0;
        if (lane == 0) idx = atomicAdd(&sk.q->head, step);
        idx = __shfl_sync(FULLMASK, idx, 0);
        if (idx >= total) break;
        if (pass == 2) {
            if (!run_item<NPOP>(a, sk, b, sk.sorted2[idx], 0, wpar)) return;
            continue;
        }
        const unsigned long long end = idx + step < total ? idx + step : total;
        for (unsigned long long c = (unsigned long long)a.k0 + idx; c < (unsigned long long)a.k0 + end;
             ++c) {
            if (sk.core_status[c] == (int8_t)SELSCAN_LOCUS_MAF_FILTERED) continue;
            for (int q = 0; q < ipc; ++q)
                if (!run_item<NPOP>(a, sk, b, (uint32_t)(c * ipc + q), max_steps, wpar)) return;
        }
    }
}

// Plain launch: one CTA per core, one warp per walk; global scratch slots
// are taken from a bitmap (at most nslots warps are resident at once).
template <int NPOP>
__global__ void __launch_bounds__(128) walk_plain_kernel(ScanArgs a, ItemSink sk, Scratch sc,
                                                         unsigned int *slotmap, int nslots)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long core = a.k0 + blockIdx.x;
    if (sk.core_status[core] == (int8_t)SELSCAN_LOCUS_MAF_FILTERED) return;
    int slot = -1;
    if (lane == 0) {
        const int start = (int)(((long long)blockIdx.x * (blockDim.x >> 5) + warp) % nslots);
        for (int t = 0; t < nslots; ++t) {
            const int s = (start + t) % nslots;
            const unsigned bit = 1u << (s & 31);
            if (!(atomicOr(slotmap + (s >> 5), bit) & bit)) { slot = s; break; }
        }
        __threadfence();
    }
    slot = __shfl_sync(FULLMASK, slot, 0);
    if (slot < 0) {                       // cannot happen: nslots >= resident warps
        if (lane == 0) {
            sk.item_status[core * (NPOP == 2 ? 2 : 4) + warp] = (int8_t)WALK_UNFINISHED;
            atomicExch(sc.err, SELSCAN_ERR_INTERNAL);
        }
        return;
    }
    WarpBufs b = make_bufs(smem + (size_t)warp * slice_bytes(sc),
                           sc.base + (size_t)slot * sc.per_warp, sc);
    init_window(b);
    unsigned wpar[2] = {0u, 0u};
    // a warp whose copies may still be in flight keeps its slot (nothing else reuses it)
    if (!run_item<NPOP>(a, sk, b, (uint32_t)(core * (NPOP == 2 ? 2 : 4) + warp), 0, wpar)) return;
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        atomicAnd(slotmap + (slot >> 5), ~(1u << (slot & 31)));
    }
}

__global__ void bucket_hist_kernel(ItemSink sk)
{
    const unsigned long long n2 = sk.q->n2;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n2;
         i += (unsigned long long)gridDim.x * blockDim.x)
        atomicAdd(sk.bucket + sk.key2[i], 1u);
}

__global__ void bucket_scan_kernel(ItemSink sk)
{
    // one block of NBUCKET threads: exclusive scan in place, head reset
    __shared__ uint32_t t[NBUCKET];
    const int i = threadIdx.x;
    t[i] = sk.bucket[i];
    __syncthreads();
    for (int o = 1; o < NBUCKET; o <<= 1) {
        uint32_t v = i >= o ? t[i - o] : 0u;
        __syncthreads();
        t[i] += v;
        __syncthreads();
    }
    sk.bucket[i] = t[i] - sk.bucket[i];
    if (i == 0) sk.q->head = 0ull;
}

__global__ void bucket_scatter_kernel(ItemSink sk)
{
    const unsigned long long n2 = sk.q->n2;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n2;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t p = atomicAdd(sk.bucket + sk.key2[i], 1u);
        sk.sorted2[p] = sk.list2[i];
    }
}

static int g_sms = 0;
static int sm_count()
{
    if (g_sms == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            g_sms = v;
        else
            return 152;
    }
    return g_sms;
}

template <typename K>
static int occupancy_of(K kernel, int warps_per_cta, size_t smem_bytes, bool carve)
{
    int nb = 0;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (carve) cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, warps_per_cta * 32, smem_bytes) !=
        cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return nb;
}

int max_ctas_per_sm(int schedule, int warps_per_cta, size_t smem_bytes, int minb)
{
    int a, b;
    if (schedule == SELSCAN_SCHED_PLAIN) {
        a = occupancy_of(walk_plain_kernel<1>, warps_per_cta, smem_bytes, false);
        b = occupancy_of(walk_plain_kernel<2>, warps_per_cta, smem_bytes, false);
    } else if (minb == 3) {
        a = occupancy_of(walk_persistent_kernel<1, 3>, warps_per_cta, smem_bytes, true);
        b = occupancy_of(walk_persistent_kernel<2, 3>, warps_per_cta, smem_bytes, true);
    } else {
        a = occupancy_of(walk_persistent_kernel<1, 2>, warps_per_cta, smem_bytes, true);
        b = occupancy_of(walk_persistent_kernel<2, 2>, warps_per_cta, smem_bytes, true);
    }
    // the smaller of the two builds: a plan must fit either population count
    if (a < 1) return b;
    if (b < 1) return a;
    return a < b ? a : b;
}

int device_sms() { return sm_count(); }

// percentage of the unified L1/shared array to reserve for shared memory so
// that the CTAs one SM holds at once fit (228 KB per SM on this part)
static int carveout_pct(size_t smem_per_cta, int ctas)
{
    const int per_sm = (ctas + sm_count() - 1) / sm_count();
    const size_t need = (smem_per_cta + 1024) * (size_t)per_sm;
    int pct = (int)((need * 100 + 228 * 1024 - 1) / (228 * 1024));
    return pct > 100 ? 100 : (pct < 10 ? 10 : pct);
}

template <int NPOP, int MINB>
static cudaError_t persistent_impl(const ScanArgs &a, const ItemSink &sk, const Scratch &sc,
                                   int schedule, int wpc, int ctas, int probe, int fetch,
                                   long long n_cores, cudaStream_t s)
{
    const size_t smem = slice_bytes(sc) * (size_t)wpc;
    cudaError_t e = cudaFuncSetAttribute(walk_persistent_kernel<NPOP, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // shared memory as large as the resident CTAs need; the rest stays L1
    e = cudaFuncSetAttribute(walk_persistent_kernel<NPOP, MINB>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, carveout_pct(smem, ctas));
    if (e != cudaSuccess) return e;
    const int cap = schedule == SELSCAN_SCHED_LONGEST_FIRST ? probe : 0;
    walk_persistent_kernel<NPOP, MINB><<<ctas, wpc * 32, smem, s>>>(a, sk, sc, n_cores, 1, cap,
                                                                     cap > 0 ? 1 : fetch);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (schedule == SELSCAN_SCHED_LONGEST_FIRST && probe > 0) {
        bucket_hist_kernel<<<2 * sm_count(), 256, 0, s>>>(sk);
        bucket_scan_kernel<<<1, NBUCKET, 0, s>>>(sk);
        bucket_scatter_kernel<<<2 * sm_count(), 256, 0, s>>>(sk);
        walk_persistent_kernel<NPOP, MINB><<<ctas, wpc * 32, smem, s>>>(a, sk, sc, n_cores, 2, 0, 1);
    }
    return cudaGetLastError();
}

template <int NPOP>
static cudaError_t walk_impl(const ScanArgs &a, const ItemSink &sk, const Scratch &sc,
                             int schedule, int wpc, int ctas, int probe, int fetch, int minb,
                             long long n_cores, cudaStream_t s)
{
    if (schedule == SELSCAN_SCHED_PLAIN) {
        const int ipc = NPOP == 2 ? 2 : 4;
        const size_t smem_p = slice_bytes(sc) * (size_t)ipc;
        cudaError_t e = cudaFuncSetAttribute(walk_plain_kernel<NPOP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p);
        if (e != cudaSuccess) return e;
        // `ctas` carries the number of scratch slots; the bitmap was reset by the caller
        walk_plain_kernel<NPOP><<<(unsigned)n_cores, ipc * 32, smem_p, s>>>(a, sk, sc, sk.slotmap,
                                                                            ctas);
        return cudaGetLastError();
    }
    if (minb == 3)
        return persistent_impl<NPOP, 3>(a, sk, sc, schedule, wpc, ctas, probe, fetch, n_cores, s);
    return persistent_impl<NPOP, 2>(a, sk, sc, schedule, wpc, ctas, probe, fetch, n_cores, s);
}

template <int NPOP, int MINB>
static cudaError_t pass2_impl(const ScanArgs &a, const ItemSink &sk, const Scratch &sc, int wpc,
                              int ctas, cudaStream_t s)
{
    const size_t smem = slice_bytes(sc) * (size_t)wpc;
    cudaError_t e = cudaFuncSetAttribute(walk_persistent_kernel<NPOP, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(walk_persistent_kernel<NPOP, MINB>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, carveout_pct(smem, ctas));
    if (e != cudaSuccess) return e;
    bucket_hist_kernel<<<2 * sm_count(), 256, 0, s>>>(sk);
    bucket_scan_kernel<<<1, NBUCKET, 0, s>>>(sk);
    bucket_scatter_kernel<<<2 * sm_count(), 256, 0, s>>>(sk);
    walk_persistent_kernel<NPOP, MINB><<<ctas, wpc * 32, smem, s>>>(a, sk, sc, 0, 2, 0, 1);
    return cudaGetLastError();
}

cudaError_t launch_pass2(const ScanArgs &a, const ItemSink &sink, const Scratch &sc,
                         int warps_per_cta, int ctas, int minb, cudaStream_t s)
{
    if (sink.mode == 1)
        return minb == 3 ? pass2_impl<2, 3>(a, sink, sc, warps_per_cta, ctas, s)
                         : pass2_impl<2, 2>(a, sink, sc, warps_per_cta, ctas, s);
    return minb == 3 ? pass2_impl<1, 3>(a, sink, sc, warps_per_cta, ctas, s)
                     : pass2_impl<1, 2>(a, sink, sc, warps_per_cta, ctas, s);
}

cudaError_t launch_walk(const ScanArgs &a, const ItemSink &sink, const Scratch &sc,
                        int schedule, int warps_per_cta, int ctas, int probe_steps, int fetch,
                        int minb, long long n_cores, cudaStream_t s)
{
    if (sink.mode == 1)
        return walk_impl<2>(a, sink, sc, schedule, warps_per_cta, ctas, probe_steps, fetch, minb,
                            n_cores, s);
    return walk_impl<1>(a, sink, sc, schedule, warps_per_cta, ctas, probe_steps, fetch, minb,
                        n_cores, s);
}

// ------------------------------------------------------------ finalize
__global__ void finalize_ihs_kernel(ItemSink sk, long long k0, long long k1, double *ihh1, double *ihh0,
                                    double *lnratio, int8_t *status)
{
    for (long long c = k0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; c < k1;
         c += (long long)gridDim.x * blockDim.x) {
        if (sk.core_status[c] == (int8_t)SELSCAN_LOCUS_MAF_FILTERED) {
            ihh1[c] = 0.0;
            ihh0[c] = 0.0;
            lnratio[c] = __longlong_as_double(0x7ff8000000000000ll);
            for (int q = 0; q < 4; ++q) { sk.stop[4 * c + q] = 0; sk.digest[4 * c + q] = 0ull; }
            continue;
        }
        int worst = 0;
        for (int q = 0; q < 4; ++q) {
            const int st = sk.item_status[4 * c + q];
            worst = st > worst ? st : worst;
        }
        const double a1 = sk.item_ihh[4 * c] + sk.item_ihh[4 * c + 1];   // down + up
        const double a0 = sk.item_ihh[4 * c + 2] + sk.item_ihh[4 * c + 3];
        if (worst == 0 && (a1 == 0.0 || a0 == 0.0)) worst = SELSCAN_LOCUS_UNDEFINED;
        ihh1[c] = a1;
        ihh0[c] = a0;
        status[c] = (int8_t)worst;
        lnratio[c] = worst == 0 ? log(a1 / a0) : __longlong_as_double(0x7ff8000000000000ll);
    }
}

__global__ void finalize_xpehh_kernel(ItemSink sk, long long k0, long long k1, double *ihhA, double *ihhB,
                                      double *lnratio, int8_t *status)
{
    for (long long c = k0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; c < k1;
         c += (long long)gridDim.x * blockDim.x) {
        if (sk.core_status[c] == (int8_t)SELSCAN_LOCUS_MAF_FILTERED) {
            ihhA[c] = 0.0;
            ihhB[c] = 0.0;
            lnratio[c] = __longlong_as_double(0x7ff8000000000000ll);
            for (int q = 0; q < 2; ++q) sk.stop[2 * c + q] = 0;
            for (int q = 0; q < 6; ++q) sk.digest[6 * c + q] = 0ull;
            continue;
        }
        int worst = 0;
        for (int q = 0; q < 2; ++q) {
            const int st = sk.item_status[2 * c + q];
            worst = st > worst ? st : worst;
        }
        const double a = sk.item_ihh[4 * c] + sk.item_ihh[4 * c + 2];      // down + up, pop A
        const double bb = sk.item_ihh[4 * c + 1] + sk.item_ihh[4 * c + 3]; // pop B
        if (worst == 0 && (a == 0.0 || bb == 0.0)) worst = SELSCAN_LOCUS_UNDEFINED;
        ihhA[c] = a;
        ihhB[c] = bb;
        status[c] = (int8_t)worst;
        lnratio[c] = worst == 0 ? log(a / bb) : __longlong_as_double(0x7ff8000000000000ll);
    }
}

cudaError_t launch_finalize_ihs(const ItemSink &sink, long long k0, long long k1, double *ihh1,
                                double *ihh0, double *lnratio, int8_t *status, cudaStream_t s)
{
    long long blocks = (k1 - k0 + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    finalize_ihs_kernel<<<(unsigned)blocks, 256, 0, s>>>(sink, k0, k1, ihh1, ihh0, lnratio, status);
    return cudaGetLastError();
}

cudaError_t launch_finalize_xpehh(const ItemSink &sink, long long k0, long long k1, double *ihhA,
                                  double *ihhB, double *lnratio, int8_t *status, cudaStream_t s)
{
    long long blocks = (k1 - k0 + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    finalize_xpehh_kernel<<<(unsigned)blocks, 256, 0, s>>>(sink, k0, k1, ihhA, ihhB, lnratio, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------ EHH trace
__global__ void __launch_bounds__(192) ehh_trace_kernel(ScanArgs a, long long locus, Scratch sc,
                                                        unsigned long long *S, long long cap,
                                                        long long *len, int32_t *stop,
                                                        int8_t *status, double *ihh,
                                                        unsigned long long *denom)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int q = threadIdx.x >> 5;           // walk w = q / 2, direction q % 2
    WarpBufs b = make_bufs(smem + (size_t)q * slice_bytes(sc),
                           sc.base + (size_t)q * sc.per_warp, sc);
    init_window(b);
    unsigned wpar[2] = {0u, 0u};
    const int w = q >> 1, dir = q & 1;
    WalkOut o = walk<1>(a, locus, dir, w, b, S + (size_t)q * cap, cap, 0, wpar);
    if (lane == 0) {
        long long steps = 0;
        if (o.status == WALK_OK) steps = o.stop + 1;
        else if (o.status == WALK_EDGE || o.status == WALK_GAP) steps = o.stop;
        len[q] = steps;
        stop[q] = o.stop;
        status[q] = (int8_t)o.status;
        ihh[q] = o.ihh[0];
    }
    if (q == 0 && lane == 0) {
        // denominators from the core row
        const unsigned int *row = (const unsigned int *)(a.hap + locus * a.ld);
        unsigned long long c1 = 0;
        for (int k = 0; k < 2 * a.W; ++k) c1 += (unsigned long long)__popc(row[k] & valid32(a, k));
        const unsigned long long n = (unsigned long long)a.nA;
        denom[0] = choose2(c1);
        denom[1] = choose2(n - c1);
        denom[2] = choose2(n);
    }
}

cudaError_t launch_ehh(const ScanArgs &a, long long locus, const Scratch &sc,
                       unsigned long long *S, long long cap, long long *len, int32_t *stop,
                       int8_t *status, double *ihh, unsigned long long *denom, cudaStream_t s)
{
    const size_t smem = slice_bytes(sc) * 6;
    cudaError_t e = cudaFuncSetAttribute(ehh_trace_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ehh_trace_kernel<<<1, 192, smem, s>>>(a, locus, sc, S, cap, len, stop, status, ihh, denom);
    return cudaGetLastError();
}

// ------------------------------------------------------------ pack
// marker-major input [m, n] bytes: a warp packs whole marker rows.  For word w
// lane l reads the bytes of haplotypes 64 w + l and 64 w + 32 + l (two
// coalesced 32-byte reads) and two ballots make the word; lane w % 32 keeps it
// and the warp stores 32 consecutive words at once.
__global__ void __launch_bounds__(256) pack_mm_kernel(const uint8_t *hap01, int n, long long m,
                                                      int W, unsigned long long *rows, long long ld)
{
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = warp; k < m; k += nw) {
        const uint8_t *src = hap01 + k * n;
        unsigned long long *dst = rows + k * ld;
        for (long long w0 = 0; w0 < ld; w0 += 32) {
            unsigned long long mine = 0;
            for (int j = 0; j < 32 && w0 + j < ld; ++j) {      // warp-uniform bounds
                const long long w = w0 + j;
                unsigned lo = 0, hi = 0;
                if (w < W) {
                    const long long h0 = 64 * w + lane, h1 = h0 + 32;
                    lo = __ballot_sync(FULLMASK, h0 < n && (src[h0] & 1));
                    hi = __ballot_sync(FULLMASK, h1 < n && (src[h1] & 1));
                }
                if (lane == j) mine = (unsigned long long)lo | ((unsigned long long)hi << 32);
            }
            if (w0 + lane < ld) dst[w0 + lane] = mine;
        }
    }
}

// bit 0 of each of the four bytes of x, as bits 0..3: with one bit per byte
// kept, the multiply moves byte i's bit to bit 24 + i and nothing else reaches
// bits 24..31
__device__ __forceinline__ unsigned byte_lsbs(unsigned x) { return ((x & 0x01010101u) * 0x01020408u) >> 24; }

// Bit j of (a, b) = bit 0 of p[j] (a: j < 32, b: j >= 32) for j < nk <= 64;
// VEC: p is 16-byte aligned and nk = 64 (four 16-byte loads).
template <bool VEC>
__device__ __forceinline__ void lsb_mask64(const uint4 *v, const uint8_t *p, int nk, unsigned &a,
                                           unsigned &b)
{
    a = 0u;
    b = 0u;
    if (VEC && nk == 64) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const unsigned s = byte_lsbs(v[i].x) | (byte_lsbs(v[i].y) << 4) |
                               (byte_lsbs(v[i].z) << 8) | (byte_lsbs(v[i].w) << 12);
            if (i < 2) a |= s << (16 * i);
            else b |= s << (16 * (i - 2));
        }
    } else {
        for (int j = 0; j < nk; ++j) {
            const unsigned bit = __ldg(p + j) & 1u;
            if (j < 32) a |= bit << j;
            else b |= bit << (j - 32);
        }
    }
}

// 32 x 32 bit transpose across a warp: lane l holds row l (bit c = entry (l, c));
// afterwards lane j holds column j (bit i = entry (i, j)).  Five butterfly stages
// exchange the off-diagonal blocks of halving size with the partner lane.
__device__ __forceinline__ unsigned warp_transpose32(unsigned x, int lane)
{
    unsigned msk = 0x0000FFFFu;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1, msk ^= msk << s) {
        const unsigned y = __shfl_xor_sync(FULLMASK, x, s);
        x = (lane & s) ? ((x & ~msk) | ((y >> s) & msk)) : ((x & msk) | ((y << s) & ~msk));
    }
    return x;
}

// haplotype-major input [n, m] bytes, markers [kbeg, m) (the ragged tail of
// the staged kernel below, or everything when rows do not start on 16-byte
// boundaries): a warp packs word w of 64 consecutive markers.  Lane l reads markers [k0, k0 + 64) of haplotypes 64 w + l and
// 64 w + 32 + l (contiguous bytes of their rows, both rows' loads issued
// together), keeps bit 0 of each byte in a 64-bit mask per haplotype, and four
// 32 x 32 bit transposes across the warp turn the masks into the markers'
// words; lane j stores the words of markers k0 + j and k0 + 32 + j.
// Consecutive warps take consecutive words of the same markers, so the stores
// of a row segment meet in L2.
template <bool VEC>
__global__ void __launch_bounds__(256) pack_hm_kernel(const uint8_t *hap01, int n, long long m,
                                                      int W, unsigned long long *rows, long long ld,
                                                      long long kbeg)
{
    const int lane = threadIdx.x & 31;
    const long long tasks = (m - kbeg + 63) / 64 * ld;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; t < tasks; t += nw) {
        const long long kb = t / ld;
        const long long w = t - kb * ld;
        const long long k0 = kbeg + kb * 64;
        const int nk = m - k0 < 64 ? (int)(m - k0) : 64;
        unsigned a0 = 0u, a1 = 0u, b0 = 0u, b1 = 0u;     // haplotype 64 w + l: a; + 32: b
        if (w < W) {
            const long long h0 = 64 * w + lane, h1 = h0 + 32;
            const bool v0 = h0 < n, v1 = h1 < n;
            // rows past n read row 0 (it exists) and are dropped
            const uint8_t *p0 = hap01 + (v0 ? h0 : 0) * m + k0;
            const uint8_t *p1 = hap01 + (v1 ? h1 : 0) * m + k0;
            uint4 q0[4], q1[4];
            if (VEC && nk == 64) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    q0[i] = __ldg((const uint4 *)p0 + i);
                    q1[i] = __ldg((const uint4 *)p1 + i);
                }
            }
            lsb_mask64<VEC>(q0, p0, nk, a0, a1);
            lsb_mask64<VEC>(q1, p1, nk, b0, b1);
            if (!v0) { a0 = 0u; a1 = 0u; }
            if (!v1) { b0 = 0u; b1 = 0u; }
        }
        const unsigned lo0 = warp_transpose32(a0, lane), hi0 = warp_transpose32(b0, lane);
        const unsigned lo1 = warp_transpose32(a1, lane), hi1 = warp_transpose32(b1, lane);
        if (lane < nk) rows[(k0 + lane) * ld + w] = (unsigned long long)lo0 | ((unsigned long long)hi0 << 32);
        if (lane + 32 < nk)
            rows[(k0 + 32 + lane) * ld + w] = (unsigned long long)lo1 | ((unsigned long long)hi1 << 32);
    }
}

// haplotype-major input [n, m] bytes, m a multiple of 16 and the input 16-byte
// aligned, whole tiles of kPackTile markers: a CTA packs word w of one tile.
// Warp v reads rows 64 w + 8 v .. + 7 as whole kPackTile-byte pieces (one
// coalesced 16-byte load per lane and row), folds each lane's 16 bytes into a
// 16-bit mask and pairs the masks of neighbouring lanes into the row's 32-bit
// mask words in shared memory (stride 17 words: the transpose's reads of one
// word of 32 rows hit distinct banks); then warp v transposes markers
// [64 v, 64 v + 64) of the tile as the warp kernel does.
constexpr int kPackTile = 512;
__global__ void __launch_bounds__(256) pack_hm_staged_kernel(const uint8_t *hap01, int n,
                                                             long long m, int W,
                                                             unsigned long long *rows, long long ld)
{
    __shared__ unsigned msk[64][kPackTile / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long tasks = m / kPackTile * ld;
    for (long long t = blockIdx.x; t < tasks; t += gridDim.x) {
        const long long kb = t / ld;
        const long long w = t - kb * ld;
        const long long k0 = kb * kPackTile;
        if (w < W) {
            uint4 q[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {              // all eight loads in flight at once
                const long long h = 64 * w + 8 * warp + r;
                q[r] = __ldg((const uint4 *)(hap01 + (h < n ? h : 0) * m + k0) + lane);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const long long h = 64 * w + 8 * warp + r;
                unsigned v = byte_lsbs(q[r].x) | (byte_lsbs(q[r].y) << 4) |
                             (byte_lsbs(q[r].z) << 8) | (byte_lsbs(q[r].w) << 12);
                if (h >= n) v = 0u;
                const unsigned hi = __shfl_down_sync(FULLMASK, v, 1);
                if ((lane & 1) == 0) msk[8 * warp + r][lane >> 1] = v | (hi << 16);
            }
        }
        __syncthreads();
        unsigned a0 = 0u, a1 = 0u, b0 = 0u, b1 = 0u;
        if (w < W) {
            a0 = msk[lane][2 * warp];
            a1 = msk[lane][2 * warp + 1];
            b0 = msk[lane + 32][2 * warp];
            b1 = msk[lane + 32][2 * warp + 1];
        }
        __syncthreads();                               // the next tile may refill msk
        const unsigned lo0 = warp_transpose32(a0, lane), hi0 = warp_transpose32(b0, lane);
        const unsigned lo1 = warp_transpose32(a1, lane), hi1 = warp_transpose32(b1, lane);
        const long long k = k0 + 64 * warp + lane;
        rows[k * ld + w] = (unsigned long long)lo0 | ((unsigned long long)hi0 << 32);
        rows[(k + 32) * ld + w] = (unsigned long long)lo1 | ((unsigned long long)hi1 << 32);
    }
}

cudaError_t launch_pack(const uint8_t *hap01, int n, long long m, int hap_major,
                        unsigned long long *rows, long long ld, cudaStream_t s)
{
    const int W = (n + 63) / 64;
    // grid-stride warps: 16 CTAs of 8 warps per SM at most
    const long long cap = 16ll * device_sms();
    if (hap_major) {
        const bool vec = m % 16 == 0 && ((uintptr_t)hap01 & 15) == 0;
        long long kbeg = 0;
        if (vec && m >= kPackTile) {
            const long long tiles = m / kPackTile * ld;
            const long long blocks = tiles < cap ? tiles : cap;
            pack_hm_staged_kernel<<<(unsigned)blocks, 256, 0, s>>>(hap01, n, m, W, rows, ld);
            kbeg = m / kPackTile * kPackTile;
        }
        if (kbeg < m) {
            const long long tasks = (m - kbeg + 63) / 64 * ld;
            long long blocks = (tasks + 7) / 8;
            if (blocks > cap) blocks = cap;
            if (vec)
                pack_hm_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(hap01, n, m, W, rows, ld, kbeg);
            else
                pack_hm_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(hap01, n, m, W, rows, ld, kbeg);
        }
    } else {
        long long blocks = (m + 7) / 8;
        if (blocks > cap) blocks = cap;
        pack_mm_kernel<<<(unsigned)blocks, 256, 0, s>>>(hap01, n, m, W, rows, ld);
    }
    return cudaGetLastError();
}

}  // namespace selscan
