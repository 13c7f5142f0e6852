// Standardised scores (Eq. 7 for iHS, Eq. 11 for XPEHH): each unstandardised
// score is centred and scaled by the mean and standard deviation of its
// frequency bin, over all markers passed in (the caller's genome).
//
// Deterministic reduction, two forms.  Up to kNormPrivMaxBins bins: CTA s reads
// segment s of the markers once; each of its threads adds its markers (thread
// stride) into its own per-bin accumulators in shared memory, then one thread
// per bin adds the threads' values in thread order.  More bins: CTA (b, s)
// sums bin b over segment s (thread stride, then a fixed tree).  Either way
// the segments are combined in segment order.  Two passes: the mean, then the
// sum of squared deviations about it (no cancellation of E[x^2] - E[x]^2).
#include <limits.h>
#include <math.h>

#include "../../include/selscan.h"
#include "internal.h"

namespace selscan {

namespace {

constexpr int kNormThreads = 256;
constexpr int kNormSegments = 16;           // per-bin form: segments per bin
constexpr int kNormPrivThreads = 64;        // private-accumulator form
constexpr int kNormPrivMaxBins = 128;       // its accumulators: 128 x 64 x 12 B = 96 KB
constexpr int kNormPrivSegments = 304;
constexpr int kNormMaxSegments = kNormPrivSegments > kNormSegments ? kNormPrivSegments : kNormSegments;

__device__ __forceinline__ int bin_of(int32_t n1, int n, int nbins)
{
    // derived-allele frequency n1 / n in nbins equal bins, decided in integers
    if (nbins == 1) return 0;
    long long b = ((long long)n1 * nbins) / n;
    return b >= nbins ? nbins - 1 : (b < 0 ? 0 : (int)b);
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kNormThreads / 32; ++w) t += red[w];
    __syncthreads();
    return t;                       // valid in thread 0
}

// The markers of bin b are those with n1 in [lo, hi): bin_of(n1) = b exactly
// when b n <= n1 nbins < (b + 1) n, i.e. ceil(b n / nbins) <= n1 <
// ceil((b + 1) n / nbins), the first bin open below and the last open above
// (bin_of clamps).  One interval per CTA, two compares per marker.
__device__ __forceinline__ void bin_interval(int b, int n, int nbins, long long &lo, long long &hi)
{
    lo = b == 0 ? LLONG_MIN : ((long long)b * n + nbins - 1) / nbins;
    hi = b == nbins - 1 ? LLONG_MAX : ((long long)(b + 1) * n + nbins - 1) / nbins;
}

// pass 0: count and sum per (bin, segment); pass 1: squared deviations about mean[bin]
__global__ void __launch_bounds__(kNormThreads) norm_partial_kernel(
    const double *score, const int8_t *status, const int32_t *n1, long long m, int n, int nbins,
    int pass, const double *mean, double *part_sum, long long *part_cnt)
{
    __shared__ double red_d[kNormThreads / 32];
    __shared__ long long red_c[kNormThreads / 32];
    const int b = blockIdx.x / kNormSegments, seg = blockIdx.x % kNormSegments;
    const long long per = (m + kNormSegments - 1) / kNormSegments;
    const long long lo = (long long)seg * per, hi = lo + per < m ? lo + per : m;
    long long n1lo, n1hi;
    bin_interval(b, n, nbins, n1lo, n1hi);
    double acc = 0.0;
    long long cnt = 0;
    const double mu = pass == 1 ? mean[b] : 0.0;
    for (long long k = lo + threadIdx.x; k < hi; k += kNormThreads) {
        if (status[k] != (int8_t)SELSCAN_LOCUS_OK) continue;
        const long long c = n1[k];
        if (c < n1lo || c >= n1hi) continue;
        const double x = score[k];
        if (pass == 0) { acc += x; ++cnt; }
        else { const double d = x - mu; acc += d * d; }
    }
    const double s = block_sum(acc, red_d);
    const long long c = block_sum(cnt, red_c);
    if (threadIdx.x == 0) {
        part_sum[blockIdx.x] = s;
        if (pass == 0) part_cnt[blockIdx.x] = c;
    }
}

// pass 0: count and sum per (segment, bin); pass 1: squared deviations about
// mean[bin].  Shared memory: sums [nbins][64] (double), counts [nbins][64].
__global__ void __launch_bounds__(kNormPrivThreads) norm_partial_private_kernel(
    const double *score, const int8_t *status, const int32_t *n1, long long m, int n, int nbins,
    int pass, const double *mean, double *part_sum, long long *part_cnt)
{
    extern __shared__ double psum[];
    int *pcnt = (int *)(psum + (size_t)nbins * kNormPrivThreads);
    const int t = threadIdx.x;
    for (int b = 0; b < nbins; ++b) {
        psum[b * kNormPrivThreads + t] = 0.0;
        pcnt[b * kNormPrivThreads + t] = 0;
    }
    const long long per = (m + kNormPrivSegments - 1) / kNormPrivSegments;
    const long long lo = (long long)blockIdx.x * per, hi = lo + per < m ? lo + per : m;
    const bool small = (unsigned long long)n * (unsigned long long)nbins < (1ull << 32);
    constexpr int U = 4;                         // markers whose loads are in flight together
    for (long long k0 = lo + t; k0 < hi; k0 += U * kNormPrivThreads) {
        int8_t st[U];
        int32_t c1[U];
        double x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long k = k0 + (long long)u * kNormPrivThreads;
            st[u] = k < hi ? status[k] : (int8_t)-1;
            c1[u] = k < hi ? n1[k] : 0;
            x[u] = k < hi ? score[k] : 0.0;
        }
        // in marker order, as one marker at a time would add them
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (st[u] != (int8_t)SELSCAN_LOCUS_OK) continue;
            // bin_of in 32 bits where n nbins fits them (0 <= n1 < n): n1 >= n is
            // the last bin, n1 <= 0 the first
            int b;
            if (!small) b = bin_of(c1[u], n, nbins);
            else if (c1[u] <= 0) b = 0;
            else if (c1[u] >= n) b = nbins - 1;
            else b = (int)((unsigned)c1[u] * (unsigned)nbins / (unsigned)n);
            double v = x[u];
            if (pass == 1) { const double d = x[u] - mean[b]; v = d * d; }
            psum[b * kNormPrivThreads + t] += v;   // this thread's slot: no other writer
            pcnt[b * kNormPrivThreads + t] += 1;
        }
    }
    __syncthreads();
    for (int b = t; b < nbins; b += kNormPrivThreads) {
        double sum = 0.0;
        long long c = 0;
        for (int j = 0; j < kNormPrivThreads; ++j) {
            sum += psum[b * kNormPrivThreads + j];
            c += pcnt[b * kNormPrivThreads + j];
        }
        part_sum[(size_t)b * kNormPrivSegments + blockIdx.x] = sum;
        if (pass == 0) part_cnt[(size_t)b * kNormPrivSegments + blockIdx.x] = c;
    }
}

// Per-bin totals of the nseg segment partials, segments in order: pass 0 the
// count and the sum, pass 1 the sum of squared deviations.
__global__ void norm_sums_kernel(int nbins, int pass, int nseg, const double *part_sum,
                                 const long long *part_cnt, long long *bin_count, double *bin_sum)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        double s = 0.0;
        long long c = 0;
#pragma unroll 8
        for (int seg = 0; seg < nseg; ++seg) {
            s += part_sum[(size_t)b * nseg + seg];
            c += part_cnt[(size_t)b * nseg + seg];
        }
        bin_sum[b] = s;
        if (pass == 0) bin_count[b] = c;
    }
}

// Mean (pass 0) or sample SD (pass 1) of each bin from its totals.
__global__ void norm_finish_kernel(int nbins, int pass, const long long *bin_count,
                                   const double *bin_sum, double *bin_mean, double *bin_sd)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        const long long c = bin_count[b];
        const double s = bin_sum[b];
        if (pass == 0)
            bin_mean[b] = c > 0 ? s / (double)c : __longlong_as_double(0x7ff8000000000000ll);
        else
            bin_sd[b] = c > 1 ? sqrt(s / (double)(c - 1)) : __longlong_as_double(0x7ff8000000000000ll);
    }
}

__global__ void norm_apply_kernel(const double *score, const int8_t *status, const int32_t *n1,
                                  long long m, int n, int nbins, const double *bin_mean,
                                  const double *bin_sd, const long long *bin_count, double *out)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m;
         k += (long long)gridDim.x * blockDim.x) {
        double r = __longlong_as_double(0x7ff8000000000000ll);
        if (status[k] == (int8_t)SELSCAN_LOCUS_OK) {
            const int b = bin_of(n1[k], n, nbins);
            const double sd = bin_sd[b];
            if (bin_count[b] >= 2 && sd > 0.0) r = (score[k] - bin_mean[b]) / sd;
        }
        out[k] = r;
    }
}

}  // namespace

}  // namespace selscan

using namespace selscan;

namespace {

size_t parts_bytes(int nbins)
{
    return ((size_t)nbins * kNormMaxSegments * 8 + 255) & ~(size_t)255;
}

bool norm_args_ok(const double *score, const int8_t *status, const int32_t *n1, int64_t m,
                  int32_t n, int32_t nbins)
{
    return score && status && n1 && m >= 1 && n >= 1 && nbins >= 1 && nbins <= SELSCAN_NORM_MAX_BINS;
}

// pass 0: bin_count and bin_sum (sum of the scores); pass 1: bin_sum = sum of
// squared deviations about bin_mean.  part_sum / part_cnt: workspace.
void launch_bin_sums(const double *score, const int8_t *status, const int32_t *n1, int64_t m,
                     int32_t n, int32_t nbins, int pass, const double *bin_mean,
                     long long *bin_count, double *bin_sum, double *part_sum, long long *part_cnt,
                     cudaStream_t s)
{
    int nseg = kNormSegments;
    if (nbins <= kNormPrivMaxBins) {
        const size_t smem = (size_t)nbins * kNormPrivThreads * (sizeof(double) + sizeof(int));
        cudaFuncSetAttribute(norm_partial_private_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)kNormPrivMaxBins * kNormPrivThreads * 12));
        norm_partial_private_kernel<<<kNormPrivSegments, kNormPrivThreads, smem, s>>>(
            score, status, n1, m, n, nbins, pass, bin_mean, part_sum, part_cnt);
        nseg = kNormPrivSegments;
    } else {
        const unsigned grid = (unsigned)(nbins * kNormSegments);
        norm_partial_kernel<<<grid, kNormThreads, 0, s>>>(score, status, n1, m, n, nbins, pass,
                                                          bin_mean, part_sum, part_cnt);
    }
    norm_sums_kernel<<<(nbins + 127) / 128, 128, 0, s>>>(nbins, pass, nseg, part_sum, part_cnt,
                                                         bin_count, bin_sum);
}

void launch_apply(const double *score, const int8_t *status, const int32_t *n1, int64_t m,
                  int32_t n, int32_t nbins, const double *bin_mean, const double *bin_sd,
                  const long long *bin_count, double *out, cudaStream_t s)
{
    long long blocks = (m + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    norm_apply_kernel<<<(unsigned)blocks, 256, 0, s>>>(score, status, n1, m, n, nbins, bin_mean,
                                                       bin_sd, bin_count, out);
}

}  // namespace

extern "C" {

size_t selscan_normalize_workspace_bytes(int32_t nbins)
{
    if (nbins < 1 || nbins > SELSCAN_NORM_MAX_BINS) return 0;
    return parts_bytes(nbins) * 2 + (((size_t)nbins * 8 + 255) & ~(size_t)255);
}

int selscan_normalize(const double *score, const int8_t *status, const int32_t *n1, int64_t m,
                      int32_t n, int32_t nbins, double *out, int64_t *bin_count, double *bin_mean,
                      double *bin_sd, void *workspace, size_t ws_bytes, void *stream)
{
    if (!norm_args_ok(score, status, n1, m, n, nbins) || !out || !bin_count || !bin_mean || !bin_sd)
        return SELSCAN_ERR_INVALID_ARG;
    const size_t need = selscan_normalize_workspace_bytes(nbins);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255)) return SELSCAN_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    double *part_sum = (double *)workspace;
    long long *part_cnt = (long long *)((unsigned char *)workspace + parts_bytes(nbins));
    double *bin_sum = (double *)((unsigned char *)workspace + 2 * parts_bytes(nbins));
    long long *cnt = (long long *)bin_count;
    for (int pass = 0; pass < 2; ++pass) {
        launch_bin_sums(score, status, n1, m, n, nbins, pass, bin_mean, cnt, bin_sum, part_sum,
                        part_cnt, s);
        norm_finish_kernel<<<(nbins + 127) / 128, 128, 0, s>>>(nbins, pass, cnt, bin_sum, bin_mean,
                                                               bin_sd);
    }
    launch_apply(score, status, n1, m, n, nbins, bin_mean, bin_sd, cnt, out, s);
    return cudaGetLastError() == cudaSuccess ? SELSCAN_OK : SELSCAN_ERR_CUDA;
}

int selscan_normalize_bin_sums(const double *score, const int8_t *status, const int32_t *n1,
                               int64_t m, int32_t n, int32_t nbins, int32_t pass,
                               const double *bin_mean, int64_t *bin_count, double *bin_sum,
                               void *workspace, size_t ws_bytes, void *stream)
{
    if (!norm_args_ok(score, status, n1, m, n, nbins) || !bin_sum || (pass != 0 && pass != 1) ||
        (pass == 0 && !bin_count) || (pass == 1 && !bin_mean))
        return SELSCAN_ERR_INVALID_ARG;
    const size_t need = selscan_normalize_workspace_bytes(nbins);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255)) return SELSCAN_ERR_WORKSPACE;
    double *part_sum = (double *)workspace;
    long long *part_cnt = (long long *)((unsigned char *)workspace + parts_bytes(nbins));
    launch_bin_sums(score, status, n1, m, n, nbins, pass, bin_mean, (long long *)bin_count, bin_sum,
                    part_sum, part_cnt, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? SELSCAN_OK : SELSCAN_ERR_CUDA;
}

int selscan_normalize_finish(int32_t nbins, int32_t pass, const int64_t *bin_count,
                             const double *bin_sum, double *bin_mean, double *bin_sd, void *stream)
{
    if (nbins < 1 || nbins > SELSCAN_NORM_MAX_BINS || (pass != 0 && pass != 1) || !bin_count ||
        !bin_sum || (pass == 0 && !bin_mean) || (pass == 1 && !bin_sd))
        return SELSCAN_ERR_INVALID_ARG;
    norm_finish_kernel<<<(nbins + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        nbins, pass, (const long long *)bin_count, bin_sum, bin_mean, bin_sd);
    return cudaGetLastError() == cudaSuccess ? SELSCAN_OK : SELSCAN_ERR_CUDA;
}

int selscan_normalize_apply(const double *score, const int8_t *status, const int32_t *n1,
                            int64_t m, int32_t n, int32_t nbins, const int64_t *bin_count,
                            const double *bin_mean, const double *bin_sd, double *out, void *stream)
{
    if (!norm_args_ok(score, status, n1, m, n, nbins) || !bin_count || !bin_mean || !bin_sd || !out)
        return SELSCAN_ERR_INVALID_ARG;
    launch_apply(score, status, n1, m, n, nbins, bin_mean, bin_sd, (const long long *)bin_count, out,
                 (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? SELSCAN_OK : SELSCAN_ERR_CUDA;
}

}  // extern "C"
