/*
 * selscan_gb300 — C ABI of the GB300 (sm_103a) EHH / iHS / XPEHH scan library.
 *
 * The statistics are those of selscan (Szpiech & Hernandez, arXiv:1403.6854):
 *   EHH    Eq. 1   whole-sample extended haplotype homozygosity
 *   EHH_c  Eq. 3   EHH of the carriers of core allele c
 *   iHH_c  Eq. 4   trapezoid integral of EHH_c over the genetic map, both ways
 *   iHS    Sec 1.2 ln(iHH_1 / iHH_0) (unstandardised; opposite sign to Voight)
 *   XPEHH  Eq. 5 / Sec 1.3  ln(iHH_A / iHH_B), both sums truncated where the
 *          EHH of the pooled A+B sample falls below the cutoff
 * with the Section 1.2 rules: sums truncated once EHH < cutoff, the genetic
 * step scaled by gap_scale/b when the physical gap b exceeds gap_scale, the
 * locus aborted at a gap b > max_gap or at the end of the marker array, and
 * no iHS at cores whose minor allele frequency is below the MAF cutoff.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Haplotype matrix ("rows"): marker-major, row k starts at rows + k * ld
 * (ld >= W words, W = ceil(n / 64)); haplotype h is bit (h % 64) of word
 * h / 64, bit value 1 = derived allele, 0 = ancestral.  Pad bits above n in
 * the last word are ignored (masked by the library).  For XPEHH a row holds
 * the W_A words of population A followed by the W_B words of population B
 * (each population starts on a word boundary; ld >= W_A + W_B).
 * Positions: int64 bp, non-decreasing.  Genetic map: double, non-decreasing,
 * in the caller's units (cM by convention); g(x_{i-1}, x_i) = |map difference|.
 * Walk directions: 0 = toward lower marker indices, 1 = toward higher.
 * Walk step i = 0 is the core itself; `stop` is the step at which a walk
 * ended: the first i >= 1 with EHH < cutoff (status OK), the step whose gap
 * exceeded max_gap (ABORT_GAP), or the first step past the array end
 * (ABORT_EDGE).  The term of the step that crosses the cutoff is not summed
 * unless include_crossing_term is set.  digest = sum over the computed steps
 * of (i + 1) * S(i) mod 2^64, where S(i) = sum over distinct extended
 * haplotypes of C(n_h, 2) — an exact integer fingerprint of the EHH numerators.
 *
 * Memory: every pointer passed to a scan entry point is DEVICE memory owned by
 * the caller (inputs, outputs and the workspace).  The library allocates and
 * frees nothing.  All scan calls are asynchronous on the given stream
 * (a cudaStream_t passed as void*; NULL = the legacy default stream); results
 * and the device error word are valid after the stream is synchronised.
 * Calls that share a workspace must be ordered on one stream.
 *
 * Errors: entry points return SELSCAN_OK (0) or a negative SELSCAN_ERR_*
 * code for problems visible on the host (bad sizes, null pointers, a bad
 * rational, a short workspace, a failed launch).  Problems found on the
 * device (decreasing positions or map, a watchdog timeout) are written to the
 * output's `error` word (0 = none) instead.  Per-locus outcomes are status
 * codes, not errors.  No C++ exception crosses this boundary.
 * SELSCAN_ERR_TIMEOUT in an error word voids every result of that launch:
 * a warp whose bounded wait for its marker-window copies gave up stops taking
 * walks (a late copy could still land in its buffers), so walks go unwritten;
 * for selscan_batch_run that is every scan of the tick, whichever scan's word
 * carries the code.
 *
 * Limits: n (iHS) and n_A + n_B (XPEHH) at most 65,000 haplotypes; m < 2^30
 * markers.
 */
#ifndef SELSCAN_GB300_H
#define SELSCAN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define SELSCAN_OK                 0
#define SELSCAN_ERR_INVALID_ARG   -1  /* null pointer, n < 2, m < 1, bad rational, ld < W, limits */
#define SELSCAN_ERR_UNSORTED      -2  /* (device error word) positions or map decrease */
#define SELSCAN_ERR_WORKSPACE     -3  /* ws_bytes < selscan_workspace_bytes(...) */
#define SELSCAN_ERR_CUDA          -4  /* a kernel launch or CUDA runtime call failed */
#define SELSCAN_ERR_TIMEOUT       -5  /* (device error word) a bounded device wait gave up */
#define SELSCAN_ERR_UNSUPPORTED   -6  /* no sm_103a device, or a launch shape it cannot run */
#define SELSCAN_ERR_INTERNAL      -7  /* (device error word) an internal consistency check failed */

/* ---- per-locus status (Section 1.2 rules) ---- */
#define SELSCAN_LOCUS_OK            0
#define SELSCAN_LOCUS_MAF_FILTERED  1  /* core MAF below the cutoff: not walked, no score */
#define SELSCAN_LOCUS_UNDEFINED     2  /* n_c < 2 or an iHH of 0: ratio undefined */
#define SELSCAN_LOCUS_ABORT_EDGE    3  /* a walk reached the array end with EHH >= cutoff */
#define SELSCAN_LOCUS_ABORT_GAP     4  /* a walk met a gap b > max_gap while running */

/* Statistic parameters (Section 1.2, "flexible parameters").  Cutoffs are
 * rationals so that "EHH < cutoff" and "MAF < cutoff" are decided exactly in
 * integers (den * S < num * C(N,2); den * minor < num * n). */
typedef struct {
    uint32_t ehh_cut_num, ehh_cut_den;   /* EHH truncation, default 1/20 */
    uint32_t maf_num, maf_den;           /* core MAF cutoff, default 1/20 */
    int64_t gap_scale_bp;                /* default 20000: b > 20 kbp => g * 20/b */
    int64_t max_gap_bp;                  /* default 200000: b > 200 kbp => abort */
    int32_t include_crossing_term;       /* 0 (default) or 1 */
    int32_t xpehh_maf_filter;            /* 0 (default): XPEHH at every marker */
    int32_t use_physical_map;            /* 0 (default): g = genetic-map distance (Section 1.2);
                                            1: g = physical distance in position units (the
                                            rehh convention of Section 2), same gap rules; the
                                            map's values are then neither read for g nor
                                            checked, but gmap must still point to m doubles */
    int32_t reserved;                    /* 0 */
} selscan_params;

/* Scheduling of the walk kernels.  Changes how the work runs, never the
 * results.  A NULL selscan_launch* selects the library defaults: the sorted
 * sweep for iHS / XPEHH scans of at least 131,072 markers and up to 16383
 * haplotypes, else the in-order persistent schedule; 8 warps per CTA and 512
 * on-chip group words per warp for the per-step kernels. */
#define SELSCAN_SCHED_DEFAULT      -1  /* the library's choice (as for a NULL selscan_launch*) */
#define SELSCAN_SCHED_LONGEST_FIRST 0  /* persistent kernel, probe pass + longest-first queue */
#define SELSCAN_SCHED_IN_ORDER      1  /* persistent kernel, one queue in core order */
#define SELSCAN_SCHED_PLAIN         2  /* one CTA per core, no persistence, no ordering */
#define SELSCAN_SCHED_SWEEP         3  /* sorted sweep: per chunk of cores the haplotypes are kept
                                          sorted by their sequence read outward from the core, and
                                          a walk applies only the neighbour pairs that part at each
                                          step; walks longer than the chunk's history finish in a
                                          second in-order pass.  Needs n_total <= 16383 (else the
                                          in-order schedule runs). */
typedef struct {
    int32_t schedule;       /* SELSCAN_SCHED_* */
    int32_t warps_per_cta;  /* 1..8 (0 = default) */
    int32_t ctas_per_sm;    /* persistent grid = SMs x this (0 = max resident) */
    int32_t smem_entries;   /* per-warp on-chip group-word capacity (0 = default) */
    int32_t probe_steps;    /* first-pass step cap of the longest-first schedule (0 = default) */
    int32_t window_rows;    /* rows per TMA window buffer, 2..64 (0 = about 1 KB of rows) */
    int32_t cores_per_fetch;/* cores a warp takes per queue fetch, in-order schedule (0 = 1) */
    int32_t min_ctas_per_sm;/* persistent build: 2 (default, 128 registers) or 3 (85 registers) */
    void *walk_begin_event; /* optional cudaEvent_t, recorded on the stream before the first walk kernel */
    void *walk_end_event;   /* optional cudaEvent_t, recorded after the last walk kernel */
    int32_t big_group_entries; /* groups with at least this many 32-bit words are split by the
                                  whole warp, smaller ones one lane each (0 = 32) */
    int32_t sweep_warmup;      /* sweep schedule: markers sorted before a chunk's first core,
                                  16..16384 (0 = 1536); walks longer than this may take the
                                  second pass */
    int32_t sweep_stage_cores; /* sweep schedule: cores per chunk between walk launches,
                                  1..8192 (0 = the whole chunk, capped so that the slot
                                  buffer stays near 24 GiB); sizes the slot buffer */
    int32_t sweep_threads;     /* sweep schedule: threads per sorting CTA, 32, 64, 128, 256
                                  or 512 (0 = the narrowest of 32 / 64 / 128 holding at most
                                  8 haplotypes per thread, 16 on chromosomes with more
                                  chunks than three 256-thread CTAs per SM hold; else 256
                                  up to 6144 haplotypes, else 512); a width is doubled until
                                  it holds at most 32 haplotypes per thread */
    int32_t sweep_split_tile;  /* sweep schedule: lanes per split walk, 32 or 16 (two walks
                                  per warp) (0 = default, 32).  16 sums each trapezoid in 16
                                  per-lane partial sums instead of 32: iHH may differ from the
                                  default in the last bits; integer results are identical */
    int32_t sweep_ctas_per_sm; /* sweep schedule, 256- and 512-thread sorts: sorting CTAs per SM
                                  over both directions, which sets the chunk count (0 = 3 of
                                  256 threads, 2 of 512; at most 2,048 threads per SM; a count
                                  the SM cannot hold at once runs in waves).  More CTAs hide
                                  more latency, but every chunk sorts its warm-up again */
    void *sweep_done_event;    /* optional cudaEvent_t, recorded after the sorting kernel of the
                                  first stage (sweep schedule): with walk_begin_event it times
                                  the sort of a one-stage scan on its own */
} selscan_launch;

/* iHS outputs: device arrays of length m (one record per marker). */
typedef struct {
    int8_t *status;     /* SELSCAN_LOCUS_* */
    int32_t *n1;        /* derived-allele count at the marker */
    double *ihh1;       /* iHH of the derived allele (down + up) */
    double *ihh0;       /* iHH of the ancestral allele */
    double *lnratio;    /* ln(ihh1 / ihh0) if status == OK, else NaN */
    int32_t *stop;      /* [m * 4]: (allele 1, down), (1, up), (0, down), (0, up) */
    uint64_t *digest;   /* [m * 4], same order */
    int32_t *error;     /* [1] device error word (0 or SELSCAN_ERR_*) */
} selscan_ihs_out;

/* XPEHH outputs: device arrays of length m. */
typedef struct {
    int8_t *status;
    int32_t *n1;        /* pooled derived-allele count */
    double *ihhA;
    double *ihhB;
    double *lnratio;    /* ln(ihhA / ihhB) if status == OK, else NaN */
    int32_t *stop;      /* [m * 2]: down, up (pooled truncation) */
    uint64_t *digest;   /* [m * 6]: down (A, B, pooled), up (A, B, pooled) */
    int32_t *error;
} selscan_xpehh_out;

/* Single-locus EHH report: walks w = 0 (carriers of allele 1, Eq. 3),
 * w = 1 (carriers of allele 0, Eq. 3), w = 2 (whole sample, Eq. 1), each in
 * both directions, index q = w * 2 + dir. */
typedef struct {
    uint64_t *S;        /* [6 * capacity]: S[q * capacity + i] = S(i), i < capacity */
    int64_t *len;       /* [6] S values computed (> capacity means truncated) */
    int32_t *stop;      /* [6] */
    int8_t *status;     /* [6] SELSCAN_LOCUS_OK / UNDEFINED / ABORT_EDGE / ABORT_GAP */
    double *ihh;        /* [6] the walk's trapezoid sum (Eq. 4 / Eq. 5, one direction) */
    uint64_t *denom;    /* [3] C(n_c,2) for allele 1, allele 0, C(n,2) */
    int32_t *error;
} selscan_ehh_out;

#define SELSCAN_MODE_IHS   0
#define SELSCAN_MODE_XPEHH 1
#define SELSCAN_MODE_EHH   2

/* Fill p with the Section 1.2 defaults (cutoffs 1/20, 20 kbp, 200 kbp). */
void selscan_default_params(selscan_params *p);

/* Workspace bytes needed by one call of the given mode on a problem of
 * n_total haplotypes (n, or n_A + n_B) and m markers, for the given launch
 * (NULL = defaults); for a core-range call, m = its number of cores k1 - k0.
 * The workspace must be 256-byte aligned. */
size_t selscan_workspace_bytes(int32_t n_total, int64_t m, int32_t mode,
                               const selscan_launch *launch);

/* iHS at every marker (Eq. 3, Eq. 4, Section 1.2).  hap/pos/gmap: device
 * inputs as described above; out: device outputs of length m. */
int selscan_ihs(const uint64_t *hap, int64_t ld, int32_t n, int64_t m,
                const int64_t *pos_bp, const double *gmap, const selscan_params *p,
                const selscan_ihs_out *out, void *workspace, size_t ws_bytes,
                const selscan_launch *launch, void *stream);

/* XPEHH at every marker (Eq. 1, Eq. 5, Section 1.3). */
int selscan_xpehh(const uint64_t *hap, int64_t ld, int32_t nA, int32_t nB, int64_t m,
                  const int64_t *pos_bp, const double *gmap, const selscan_params *p,
                  const selscan_xpehh_out *out, void *workspace, size_t ws_bytes,
                  const selscan_launch *launch, void *stream);

/* The scans of one chromosome restricted to the cores [k0, k1) (0 <= k0 <
 * k1 <= m), for splitting one scan over several GPUs or calls (Section 3:
 * the sites are independent and every walk may read the whole data set).
 * Each call needs the whole matrix, positions and map of all m markers --
 * walks run to wherever their EHH or the rules stop them, outside the range
 * too -- but walks only from its own cores: outputs are arrays of k1 - k0
 * cores (entry j is core k0 + j; stop and digest as for the whole scan, 4 or
 * 2 / 6 per core).  The results of core k equal those of the whole scan bit
 * for bit, whatever the split.  Workspace: selscan_workspace_bytes(n_total,
 * k1 - k0, mode, launch); the default schedule is chosen for k1 - k0 cores.
 * SELSCAN_ERR_INVALID_ARG for an empty or out-of-bounds range. */
int selscan_ihs_range(const uint64_t *hap, int64_t ld, int32_t n, int64_t m, int64_t k0,
                      int64_t k1, const int64_t *pos_bp, const double *gmap,
                      const selscan_params *p, const selscan_ihs_out *out, void *workspace,
                      size_t ws_bytes, const selscan_launch *launch, void *stream);
int selscan_xpehh_range(const uint64_t *hap, int64_t ld, int32_t nA, int32_t nB, int64_t m,
                        int64_t k0, int64_t k1, const int64_t *pos_bp, const double *gmap,
                        const selscan_params *p, const selscan_xpehh_out *out, void *workspace,
                        size_t ws_bytes, const selscan_launch *launch, void *stream);

/* EHH decay around one locus (Eq. 1 and Eq. 3 at every step, Section 1.1),
 * S(i) recorded for i < capacity.  SELSCAN_ERR_UNSUPPORTED when the six
 * walks' shared-memory slices (their marker window holds rows of ld words)
 * exceed one CTA's shared memory, e.g. ld above about 1,000 words. */
int selscan_ehh(const uint64_t *hap, int64_t ld, int32_t n, int64_t m,
                const int64_t *pos_bp, const double *gmap, int64_t locus,
                const selscan_params *p, const selscan_ehh_out *out, int64_t capacity,
                void *workspace, size_t ws_bytes, void *stream);

/* Allocation-free variant of selscan_ehh, for callers that must not allocate
 * device memory while they run (a process whose device memory belongs to
 * another framework's pool, a service that reserves everything at start-up,
 * or a path that cannot afford cudaMalloc's implicit synchronisation).  The
 * paper has no counterpart; the results are those of selscan_ehh.  The walks'
 * scratch is a fixed array inside the library's device image (about 1.2 MiB,
 * held by every GPU that loads the library until the process exits), so there
 * is no workspace argument and nothing is allocated or freed.
 * - n above SELSCAN_EHH_NOALLOC_MAX_N is refused with SELSCAN_ERR_INVALID_ARG.
 * - The first call on each device looks up the array's device address (with
 *   that device current), and so does the first call after the device's
 *   context was destroyed and re-created (cudaDeviceReset); make the first
 *   call on a device before any stream capture.
 * - Every call on a device shares the one array, which keeps the last call's
 *   contents (each call initialises what it reads, so no clearing is needed);
 *   calls that overlap on the same GPU race, so order them on one stream. */
#define SELSCAN_EHH_NOALLOC_MAX_N 8192
int selscan_ehh_noalloc(const uint64_t *hap, int64_t ld, int32_t n, int64_t m,
                        const int64_t *pos_bp, const double *gmap, int64_t locus,
                        const selscan_params *p, const selscan_ehh_out *out, int64_t capacity,
                        void *stream);

/* ---- batched scans (continuous batching) -------------------------------
 * Several scans (iHS and XPEHH, any sizes) share one persistent walk launch
 * ("tick"): the caller hands each tick core ranges from any admitted scans,
 * and walks of different scans run side by side on the GPU.  Results are
 * exactly those of selscan_ihs / selscan_xpehh on each scan alone.
 * Life of a scan: selscan_batch_prepare (validate + core selection), one or
 * more ticks covering every core [0, m) exactly once, selscan_batch_finalize.
 * All buffers in selscan_scan are caller-owned device memory; ticks and the
 * prepare/finalize calls of one scan must be ordered on one stream (or by
 * events between streams). */
#define SELSCAN_BATCH_MAX_SCANS 64    /* scans in one tick */
#define SELSCAN_BATCH_MAX_UNITS 256   /* core ranges in one tick */
typedef struct {
    int32_t mode;                 /* SELSCAN_MODE_IHS or SELSCAN_MODE_XPEHH */
    int32_t nA, nB;               /* iHS: n, (ignored); XPEHH: n_A, n_B */
    int64_t m, ld;
    const uint64_t *hap;          /* rows as for selscan_ihs / selscan_xpehh */
    const int64_t *pos_bp;
    const double *gmap;
    selscan_params params;
    int8_t *status;               /* outputs: as selscan_ihs_out / selscan_xpehh_out */
    int32_t *n1;
    double *ihh_a;                /* iHH_1 (iHS) or iHH_A (XPEHH) */
    double *ihh_b;                /* iHH_0 (iHS) or iHH_B (XPEHH) */
    double *lnratio;
    int32_t *stop;
    uint64_t *digest;
    int32_t *error;
    void *items;                  /* per-walk results, selscan_batch_item_bytes(m, mode) bytes, 256-aligned */
} selscan_scan;

size_t selscan_batch_item_bytes(int64_t m, int32_t mode);
/* Workspace of one tick for scans of at most max_n_total haplotypes and row
 * stride max_ld (max_scans <= SELSCAN_BATCH_MAX_SCANS and max_units <=
 * SELSCAN_BATCH_MAX_UNITS, else 0; neither changes the size).  Two ticks in
 * flight at once need two workspaces. */
size_t selscan_batch_workspace_bytes(int32_t max_n_total, int64_t max_ld, int32_t max_scans,
                                     int32_t max_units);
int selscan_batch_prepare(const selscan_scan *scan, void *stream);
/* One tick: core ranges [unit_c0[u], unit_c1[u]) of scans[unit_scan[u]],
 * u < nunits <= SELSCAN_BATCH_MAX_UNITS, nscans <= SELSCAN_BATCH_MAX_SCANS
 * (host arrays, read before the call returns: the tick copies nothing to the
 * device, its descriptors travel in the launch's parameter block).  Cores
 * are walked in unit order, one core per fetch of a warp.  max_n_total /
 * max_ld bound the scans of this tick.  SELSCAN_ERR_INVALID_ARG for counts
 * above the limits, ranges outside [0, m) or a scan that fails the checks of
 * selscan_batch_prepare; nothing is launched then. */
int selscan_batch_run(const selscan_scan *scans, int32_t nscans, const int32_t *unit_scan,
                      const int64_t *unit_c0, const int64_t *unit_c1, int32_t nunits,
                      int32_t max_n_total, int64_t max_ld, void *workspace, size_t ws_bytes,
                      void *stream);
int selscan_batch_finalize(const selscan_scan *scan, void *stream);

/* Standardised scores (Eq. 7 for iHS, Eq. 11 for XPEHH).  Markers with
 * status[k] == SELSCAN_LOCUS_OK are grouped by the derived-allele frequency of
 * the core, n1[k] / n, into nbins equal bins, bin = min(nbins - 1,
 * floor(nbins * n1 / n)) decided in integers (nbins = 1: one genome-wide bin,
 * as XPEHH's normalisation uses; n = n_A + n_B there).  Each bin's mean and
 * standard deviation (sample SD, count - 1 in the denominator) are taken over
 * the markers passed in -- concatenate the chromosomes of a genome into one
 * call -- and out[k] = (score[k] - mean) / SD; NaN for markers that are not OK
 * and for bins with fewer than two scores or SD 0.  All arrays are device
 * memory: score, status, n1, out [m] (the outputs of selscan_ihs /
 * selscan_xpehh: lnratio, status, n1), bin_count / bin_mean / bin_sd [nbins].
 * The reduction is deterministic (fixed summation order).  Workspace:
 * selscan_normalize_workspace_bytes(nbins), 256-byte aligned. */
#define SELSCAN_NORM_MAX_BINS 1024
size_t selscan_normalize_workspace_bytes(int32_t nbins);
int selscan_normalize(const double *score, const int8_t *status, const int32_t *n1, int64_t m,
                      int32_t n, int32_t nbins, double *out, int64_t *bin_count, double *bin_mean,
                      double *bin_sd, void *workspace, size_t ws_bytes, void *stream);

/* The steps of selscan_normalize, for scores spread over several calls or
 * GPUs (the shards of one genome): per-bin sums over one shard, then totals
 * summed across shards by the caller (e.g. an all-reduce), then the bin
 * statistics, then the scores.  Bins, statuses and the NaN rules are those
 * of selscan_normalize; the sums are deterministic within a shard, so a
 * split into shards changes only the order of the additions (the results
 * agree with one call to rounding).  Sequence, with totals summed across
 * shards after each bin_sums call:
 *   selscan_normalize_bin_sums(pass 0) -> bin_count [nbins], bin_sum = the
 *     shard's sum of its OK scores per bin
 *   selscan_normalize_finish(pass 0, totals) -> bin_mean
 *   selscan_normalize_bin_sums(pass 1, bin_mean) -> bin_sum = the shard's sum
 *     of squared deviations about the mean (bin_count is not written)
 *   selscan_normalize_finish(pass 1, totals) -> bin_sd (sample SD)
 *   selscan_normalize_apply(shard scores, bin statistics) -> out [m]
 * All arrays are device memory; bin_sums takes a workspace of
 * selscan_normalize_workspace_bytes(nbins) bytes (256-byte aligned). */
int selscan_normalize_bin_sums(const double *score, const int8_t *status, const int32_t *n1,
                               int64_t m, int32_t n, int32_t nbins, int32_t pass,
                               const double *bin_mean, int64_t *bin_count, double *bin_sum,
                               void *workspace, size_t ws_bytes, void *stream);
int selscan_normalize_finish(int32_t nbins, int32_t pass, const int64_t *bin_count,
                             const double *bin_sum, double *bin_mean, double *bin_sd, void *stream);
int selscan_normalize_apply(const double *score, const int8_t *status, const int32_t *n1,
                            int64_t m, int32_t n, int32_t nbins, const int64_t *bin_count,
                            const double *bin_mean, const double *bin_sd, double *out, void *stream);

/* Pack a 0/1 uint8 matrix into rows (Section 1.1 coding, 0 ancestral / 1
 * derived).  hap_major = 0: hap01 is [m][n] (marker-major); 1: [n][m].
 * Values other than 0/1 are read as (v & 1).  rows: [m][ld], pad bits and
 * words beyond W written as 0. */
int selscan_pack(const uint8_t *hap01, int32_t n, int64_t m, int32_t hap_major,
                 uint64_t *rows, int64_t ld, void *stream);

/* The schedule a default launch (NULL, or schedule SELSCAN_SCHED_DEFAULT)
 * takes for a scan of n_total haplotypes (n_A + n_B for XPEHH) and m
 * markers: SELSCAN_SCHED_SWEEP for m >= 32768 + 4 n_total and at most 16383
 * haplotypes, else SELSCAN_SCHED_IN_ORDER; -1 for bad arguments (mode
 * SELSCAN_MODE_IHS or SELSCAN_MODE_XPEHH).  Host only: no device work. */
int32_t selscan_default_schedule(int32_t n_total, int64_t m, int32_t mode);

/* Work of the sorting kernels of a sweep-schedule call: *marker_passes = the
 * markers all sorting CTAs step through over every stage (each chunk's cores
 * plus its warm-up, both directions), *elements = the sorted elements per
 * marker pass (n_total rounded up to the CTA's element grid).  Host only: no
 * device work.  Returns SELSCAN_OK, or SELSCAN_ERR_INVALID_ARG for bad
 * arguments or a launch that does not take the sweep schedule. */
int selscan_sweep_work(int32_t n_total, int64_t m, int32_t mode, const selscan_launch *launch,
                       int64_t *marker_passes, int64_t *elements);

/* Kernel launches one selscan_ihs / selscan_xpehh call makes with this
 * launch shape (mode SELSCAN_MODE_IHS or SELSCAN_MODE_XPEHH), or -1 for bad
 * arguments.  Host only: no device work. */
int32_t selscan_launch_count(int32_t n_total, int64_t m, int32_t mode, const selscan_launch *launch);

/* Read a TPED haplotype file (host code; no device work): one line per
 * marker with the chromosome, marker id, genetic position (map units),
 * physical position and then the n phased alleles coded 0 / 1 (Section 1.1),
 * separated by white space; blank lines are skipped.  Two calls: with
 * rows == NULL it only sets *n and *m; then with host buffers rows [m][ld]
 * (ld >= ceil(n / 64), filled bit-packed with pad bits 0 -- the layout of
 * selscan_ihs), pos_bp [m] and gmap [m], and *n, *m as returned.
 * SELSCAN_ERR_INVALID_ARG for an unreadable file, a malformed line or a
 * line of another width (*err_line = its 1-based marker-line index). */
int selscan_read_tped(const char *path, int32_t *n, int64_t *m, uint64_t *rows, int64_t ld,
                      int64_t *pos_bp, double *gmap, int64_t *err_line);

/* Static description of a return or error code. */
const char *selscan_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* SELSCAN_GB300_H */
