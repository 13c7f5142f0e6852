// Allocation-free single-locus EHH report (selscan_ehh_noalloc).
//
// Same result as selscan_ehh, but the walks' scratch comes from a fixed
// array in the library's own device memory instead of a caller workspace.
// It serves callers that must not allocate device memory while they run:
// for example a host process whose device memory is owned by another
// framework's pool, a service that reserves all of its memory at start-up
// and forbids later allocation, or a caller on a path where the implicit
// synchronisation or failure modes of cudaMalloc are unacceptable.  The
// paper has no counterpart: this is an interface convenience only.
//
// The array (about 1.2 MiB) is a module-scope __device__ variable, so every
// GPU that loads the library holds it until the process exits.  Host code
// cannot use its name as a device address: the set-up below asks the
// runtime for the address once per device (with that device current) and
// passes it to the kernel.  The first call on each device performs that
// set-up, so it should happen before any stream capture.  All calls share
// the one array and it keeps the previous call's contents: every walk
// initialises each word before it reads it, so nothing there has to start
// at zero; calls that overlap on the same GPU (for example on two streams) race on it, so the caller must
// order them (each device has its own copy of the array).
#include <mutex>

#include "../../include/selscan.h"
#include "internal.h"

using namespace selscan;

namespace {

constexpr int kWalks = 6;   // (allele 1, allele 0, whole sample) x (down, up)
constexpr size_t kSliceBytes = scratch_per_warp(SELSCAN_EHH_NOALLOC_MAX_N);
constexpr int kSmemEntries = 128;

static __device__ __align__(256) unsigned char g_ehh_scratch[kWalks * kSliceBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// device address of g_ehh_scratch on the current device (looked up once per device)
int scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SELSCAN_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SELSCAN_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_ehh_scratch) != cudaSuccess || !p) return SELSCAN_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return SELSCAN_OK;
}

}  // namespace

extern "C" int selscan_ehh_noalloc(const uint64_t *hap, int64_t ld, int32_t n, int64_t m,
                                   const int64_t *pos_bp, const double *gmap, int64_t locus,
                                   const selscan_params *p, const selscan_ehh_out *out,
                                   int64_t capacity, void *stream)
{
    if (!hap || !pos_bp || !gmap || !out || !p) return SELSCAN_ERR_INVALID_ARG;
    if (p->ehh_cut_den == 0 || p->maf_den == 0 || p->gap_scale_bp <= 0 || p->max_gap_bp < 0 ||
        (p->include_crossing_term != 0 && p->include_crossing_term != 1) ||
        (p->use_physical_map != 0 && p->use_physical_map != 1))
        return SELSCAN_ERR_INVALID_ARG;
    // the fixed array holds six slices of the size a sample of
    // SELSCAN_EHH_NOALLOC_MAX_N haplotypes needs: larger samples are refused
    if (n < 2 || n > SELSCAN_EHH_NOALLOC_MAX_N || m < 1 || m >= (1ll << 30) ||
        ld < (n + 63) / 64 || locus < 0 || locus >= m || capacity < 0)
        return SELSCAN_ERR_INVALID_ARG;
    if ((capacity > 0 && !out->S) || !out->len || !out->stop || !out->status || !out->ihh ||
        !out->denom || !out->error)
        return SELSCAN_ERR_INVALID_ARG;
    void *base = nullptr;
    const int rc = scratch_address(&base);
    if (rc != SELSCAN_OK) return rc;

    ScanArgs a;
    a.hap = (const unsigned long long *)hap;
    a.ld = ld;
    a.m = m;
    a.pos = (const long long *)pos_bp;
    a.gmap = gmap;
    a.WA = (n + 63) / 64;
    a.W = a.WA;
    a.nA = n;
    a.nB = 0;
    a.lastA = (n % 64) ? ((1ull << (n % 64)) - 1ull) : ~0ull;
    a.lastB = ~0ull;
    a.cut_num = p->ehh_cut_num;
    a.cut_den = p->ehh_cut_den;
    a.gap_scale = p->gap_scale_bp;
    a.max_gap = p->max_gap_bp;
    a.crossing = p->include_crossing_term;
    a.physical = p->use_physical_map;

    Scratch sc;
    sc.base = (unsigned char *)base;
    sc.per_warp = scratch_per_warp(n);   // six slices of this size fit in the array
    sc.cap = list_cap(n);
    sc.tcap = table_cap(n);
    sc.cap_s = kSmemEntries;
    sc.tcap_s = kSmemEntries / 4;
    sc.R = window_rows(ld);
    sc.rowcap = win_rowcap(sc.R, ld);
    sc.poscap = win_poscap(sc.R);
    sc.bigt = 32;
    sc.err = out->error;

    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(out->error, 0, sizeof(int32_t), s) != cudaSuccess) return SELSCAN_ERR_CUDA;
    if (launch_validate((const long long *)pos_bp, gmap, m, out->error, s, !p->use_physical_map) !=
        cudaSuccess)
        return SELSCAN_ERR_CUDA;
    if (launch_ehh(a, locus, sc, (unsigned long long *)out->S, capacity, (long long *)out->len,
                   out->stop, out->status, out->ihh, (unsigned long long *)out->denom, s) !=
        cudaSuccess)
        return SELSCAN_ERR_CUDA;
    return SELSCAN_OK;
}
