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
// runtime for the address (with the device current) and passes it to the
// kernel.  The set-up runs on the first call on each device, and again on
// the first call after that device's context was destroyed and re-created
// (cudaDeviceReset), since the array may then sit at another address; the
// first call on a device should therefore come before any stream capture.
// All calls share the one array and it keeps the previous call's contents:
// every walk initialises each word before it reads it, so nothing there has
// to start at zero; calls that overlap on the same GPU (for example on two
// streams) race on it, so the caller must order them (each device has its
// own copy of the array).
//
// Walk arguments, the plan (on-chip tier sizes, marker window) and the
// argument checks are those of selscan_ehh (ehh_prepare in api.cu); only
// the scratch base differs.
#include <mutex>

#include "../../include/selscan.h"
#include "internal.h"

using namespace selscan;

namespace {

constexpr int kWalks = 6;   // (allele 1, allele 0, whole sample) x (down, up)
constexpr size_t kSliceBytes = scratch_per_warp(SELSCAN_EHH_NOALLOC_MAX_N);

static __device__ __align__(256) unsigned char g_ehh_scratch[kWalks * kSliceBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct DeviceScratch {
    unsigned long long ctx;   // context the address was looked up in (0: unknown)
    void *addr;
};
DeviceScratch g_dev[kMaxDevices] = {};

// cuCtxGetId, reached through the runtime (no link against the driver
// library): a process-unique identifier of the current context, so that a
// context re-created after a device reset is told apart from the old one.
using CtxGetId = int (*)(void *ctx, unsigned long long *id);
CtxGetId g_ctx_get_id = nullptr;
std::once_flag g_ctx_once;

unsigned long long current_context_id()
{
    std::call_once(g_ctx_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = (CtxGetId)fn;
    });
    unsigned long long id = 0;
    if (!g_ctx_get_id || g_ctx_get_id(nullptr, &id) != 0) return 0;
    return id;
}

// Device address of g_ehh_scratch on the current device: looked up once per
// device context (every call, if the context cannot be identified).
int scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SELSCAN_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SELSCAN_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceScratch &d = g_dev[dev];
    const unsigned long long id = current_context_id();
    if (id == 0 || d.addr == nullptr || d.ctx != id) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_ehh_scratch) != cudaSuccess || !p) return SELSCAN_ERR_CUDA;
        d.addr = p;
        d.ctx = id != 0 ? id : current_context_id();   // the look-up made the context current
    }
    *out = d.addr;
    return SELSCAN_OK;
}

}  // namespace

extern "C" int selscan_ehh_noalloc(const uint64_t *hap, int64_t ld, int32_t n, int64_t m,
                                   const int64_t *pos_bp, const double *gmap, int64_t locus,
                                   const selscan_params *p, const selscan_ehh_out *out,
                                   int64_t capacity, void *stream)
{
    // the fixed array holds six slices of the size a sample of
    // SELSCAN_EHH_NOALLOC_MAX_N haplotypes needs: larger samples are refused
    ScanArgs a;
    Scratch sc;
    size_t scratch_off = 0, ws_need = 0;
    int rc = ehh_prepare(hap, ld, n, m, pos_bp, gmap, locus, p, out, capacity,
                         SELSCAN_EHH_NOALLOC_MAX_N, &a, &sc, &scratch_off, &ws_need);
    if (rc != SELSCAN_OK) return rc;
    if ((size_t)kWalks * sc.per_warp > sizeof(g_ehh_scratch)) return SELSCAN_ERR_INTERNAL;
    void *base = nullptr;
    if ((rc = scratch_address(&base)) != SELSCAN_OK) return rc;
    sc.base = (unsigned char *)base;
    return ehh_run(a, locus, p, sc, out, capacity, stream);
}
