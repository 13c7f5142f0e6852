/*
 * CPU oracle for the EHH / iHS / XPEHH scans of selscan (Szpiech & Hernandez,
 * arXiv:1403.6854).  TEST INFRASTRUCTURE ONLY: it exists to check the CUDA
 * library and to be timed as a CPU baseline; nothing in the product path may
 * call it.  It shares no code with the CUDA path.
 *
 * It applies the paper's definitions literally, for every core x_0 and each
 * direction:
 *   - Section 1.1: the extended haplotype of haplotype h at step i is the
 *     string of its alleles at x_0, x_1, ..., x_i.  At every step the strings
 *     are rebuilt (one allele appended), sorted, and equal strings counted;
 *     S(i) = sum over distinct strings of C(n_h, 2).
 *   - Eq. 1: EHH(x_i)   = S(i) / C(n, 2)    over a whole sample.
 *   - Eq. 3: EHH_c(x_i) = S_c(i) / C(n_c, 2) over the carriers of core allele c.
 *   - Eq. 4: iHH_c = sum over the downstream and upstream walks of
 *     1/2 (EHH_c(x_{i-1}) + EHH_c(x_i)) g(x_{i-1}, x_i); iHS = ln(iHH_1/iHH_0).
 *   - Eq. 5: iHH_A, iHH_B from whole-sample EHH of each population, both
 *     truncated where the EHH of the pooled sample drops below the cutoff
 *     (Section 1.3); XPEHH = ln(iHH_A/iHH_B).
 *   - Section 1.2 rules: truncation once EHH < cutoff, g scaled by 20/b when
 *     the physical gap b (kbp) exceeds 20, abort at a gap b > 200 or at the
 *     end of the chromosome, no iHS at cores with MAF < 0.05; the three
 *     thresholds are parameters.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   c1  the term of the first step with EHH < cutoff is not summed (flag
 *       include_crossing_term adds it);
 *   c2  the comparison is strict: EHH exactly equal to the cutoff continues;
 *   c3  the cutoff is the rational num/den and EHH < cutoff is decided
 *       exactly as den * S < num * C(N,2) in integers;
 *   c4  scale iff gap_bp > gap_scale_bp, factor (gap_scale_bp/1000)/(gap_bp/1000);
 *   c5  abort iff gap_bp > max_gap_bp on a step taken while the walk is
 *       still running; the gap test precedes that step's EHH;
 *   c6  each (allele, direction) walk truncates on its own EHH_c; any abort
 *       aborts the locus;
 *   c7  "chromosome arm" = the ends of the marker array: a walk still
 *       running after the last marker aborts;
 *   c8  whole-sample EHH(x_0) counts the two core-allele classes;
 *   c9  XPEHH is reported at every marker unless xpehh_maf_filter is set
 *       (then the pooled MAF is tested);
 *   c11 n_c < 2 or a zero iHH leaves the score undefined;
 *   c12 g = |gmap(x_i) - gmap(x_{i-1})|;
 *   c13 allele 1 = derived; iHS = ln(iHH_1 / iHH_0).
 * Direction 0 walks toward lower marker indices, direction 1 toward higher.
 * The walk index i starts at 0 (the core) and stop = the step at which the
 * walk ended (first i with EHH < cutoff, the step of the gap, or the first
 * step past the array end).  digest = sum over the computed steps of
 * (i + 1) * S(i) mod 2^64.
 */
#define _GNU_SOURCE
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    uint32_t ehh_cut_num, ehh_cut_den;
    uint32_t maf_num, maf_den;
    int64_t gap_scale_bp;
    int64_t max_gap_bp;
    int32_t include_crossing_term;
    int32_t xpehh_maf_filter;
    int32_t use_physical_map;   /* g = physical distance b instead of the map (Section 2) */
    int32_t reserved;
} oracle_params;

enum { ST_OK = 0, ST_MAF_FILTERED = 1, ST_UNDEFINED = 2, ST_ABORT_EDGE = 3, ST_ABORT_GAP = 4 };

static inline int allele(const uint64_t *rows, int64_t ld, int64_t x, int64_t word_off, int32_t h)
{
    return (int)((rows[x * ld + word_off + (h >> 6)] >> (h & 63)) & 1ULL);
}

static inline uint64_t choose2(uint64_t k) { return k * (k - 1) / 2; }

/* EHH < num/den, i.e. den * S < num * D, exactly */
static inline int below_cutoff(uint64_t S, uint64_t D, const oracle_params *p)
{
    return (unsigned __int128)p->ehh_cut_den * S < (unsigned __int128)p->ehh_cut_num * D;
}

/* ---------------- extended haplotype strings ---------------- */
typedef struct {
    int32_t nmem;       /* haplotypes in the walk */
    int32_t *hap;       /* their indices */
    int8_t *popid;      /* population of each member (0 = A, 1 = B) */
    int64_t *word_off;  /* word offset of its population */
    int32_t *idx;       /* sort permutation over members */
    char *str;          /* nmem strings of capacity cap */
    int64_t cap, len;
} strings;

typedef struct { const char *str; int64_t cap, len; } cmp_ctx;

static int cmp_members(const void *a, const void *b, void *vctx)
{
    const cmp_ctx *c = (const cmp_ctx *)vctx;
    int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
    int r = memcmp(c->str + (int64_t)i * c->cap, c->str + (int64_t)j * c->cap, (size_t)c->len);
    if (r) return r;
    return (i > j) - (i < j);
}

static void strings_append(strings *s, const uint64_t *rows, int64_t ld, int64_t x)
{
    if (s->len == s->cap) {
        int64_t ncap = s->cap ? 2 * s->cap : 64;
        char *nstr = (char *)malloc((size_t)(ncap * (s->nmem ? s->nmem : 1)));
        for (int32_t k = 0; k < s->nmem; ++k)
            memcpy(nstr + k * ncap, s->str + k * s->cap, (size_t)s->len);
        free(s->str);
        s->str = nstr;
        s->cap = ncap;
    }
    for (int32_t k = 0; k < s->nmem; ++k)
        s->str[k * s->cap + s->len] = (char)('0' + allele(rows, ld, x, s->word_off[k], s->hap[k]));
    s->len += 1;
}

/* Sort the strings and count each class of equal strings: returns
 * S_pop[0..1] = sum of C(count within pop, 2), S_all = sum of C(count, 2). */
static void strings_count(strings *s, uint64_t *S_pop, uint64_t *S_all)
{
    for (int32_t k = 0; k < s->nmem; ++k) s->idx[k] = k;
    cmp_ctx c = { s->str, s->cap, s->len };
    qsort_r(s->idx, (size_t)s->nmem, sizeof(int32_t), cmp_members, &c);
    S_pop[0] = S_pop[1] = 0;
    *S_all = 0;
    int32_t k = 0;
    while (k < s->nmem) {
        int32_t e = k + 1;
        while (e < s->nmem && memcmp(s->str + (int64_t)s->idx[k] * s->cap,
                                     s->str + (int64_t)s->idx[e] * s->cap, (size_t)s->len) == 0)
            ++e;
        uint64_t cnt[2] = {0, 0};
        for (int32_t t = k; t < e; ++t) cnt[s->popid[s->idx[t]]] += 1;
        S_pop[0] += choose2(cnt[0]);
        S_pop[1] += choose2(cnt[1]);
        *S_all += choose2(cnt[0] + cnt[1]);
        k = e;
    }
}

static void strings_free(strings *s)
{
    free(s->hap); free(s->popid); free(s->word_off); free(s->idx); free(s->str);
    memset(s, 0, sizeof(*s));
}

/* ---------------- one walk ---------------- */
typedef struct {
    int status;          /* ST_OK, ST_ABORT_EDGE, ST_ABORT_GAP, ST_UNDEFINED */
    int32_t stop;
    double ihh[2];       /* per population (iHS uses [0]) */
    uint64_t digest[3];  /* pop A (or carriers), pop B, pooled */
    int64_t steps;       /* number of S values computed (i = 0 .. steps-1) */
} walk_out;

/*
 * Walk from core j in direction dir (0: lower indices, 1: higher) over the
 * members in s (their strings are empty on entry).  npop = 1: the members are
 * one sample (the carriers of a core allele, or a whole population) whose
 * EHH is S_all / C(n,2); npop = 2: two populations A and B, EHH per
 * population plus the pooled EHH that decides truncation (Section 1.3).
 * trace (optional, capacity cap per quantity) receives S(i) for i < cap.
 */
static walk_out walk(const uint64_t *rows, int64_t ld, int64_t m, const int64_t *pos,
                     const double *gmap, const oracle_params *p, strings *s,
                     int npop, int32_t nA, int32_t nB, int64_t j, int dir,
                     uint64_t *trace, int64_t cap)
{
    walk_out o;
    memset(&o, 0, sizeof(o));
    const int64_t step = dir ? 1 : -1;
    const uint64_t D_all = choose2((uint64_t)s->nmem);
    const uint64_t D_pop[2] = { choose2((uint64_t)nA), choose2((uint64_t)nB) };
    uint64_t S_pop[2], S_all;
    double ehh_prev[2], ehh_cur[2];

    if (D_all == 0) { o.status = ST_UNDEFINED; return o; }

    /* i = 0: the core marker alone */
    strings_append(s, rows, ld, j);
    strings_count(s, S_pop, &S_all);
    if (trace && cap > 0) trace[0] = S_all;
    if (npop == 1) {
        ehh_prev[0] = (double)S_all / (double)D_all;
        o.digest[0] += 1ULL * S_all;
    } else {
        ehh_prev[0] = (double)S_pop[0] / (double)D_pop[0];
        ehh_prev[1] = (double)S_pop[1] / (double)D_pop[1];
        o.digest[0] += S_pop[0];
        o.digest[1] += S_pop[1];
        o.digest[2] += S_all;
    }
    o.steps = 1;

    for (int64_t i = 1;; ++i) {
        int64_t x = j + step * i, xp = x - step;
        if (x < 0 || x >= m) { o.status = ST_ABORT_EDGE; o.stop = (int32_t)i; break; }
        int64_t b = pos[x] > pos[xp] ? pos[x] - pos[xp] : pos[xp] - pos[x];
        if (b > p->max_gap_bp) { o.status = ST_ABORT_GAP; o.stop = (int32_t)i; break; }
        double g = p->use_physical_map ? (double)b : fabs(gmap[x] - gmap[xp]);
        if (b > p->gap_scale_bp)
            g = g * (((double)p->gap_scale_bp / 1000.0) / ((double)b / 1000.0));

        strings_append(s, rows, ld, x);
        strings_count(s, S_pop, &S_all);
        if (trace && i < cap) trace[i] = S_all;
        o.steps = i + 1;

        int stop;
        if (npop == 1) {
            ehh_cur[0] = (double)S_all / (double)D_all;
            o.digest[0] += (uint64_t)(i + 1) * S_all;
            stop = below_cutoff(S_all, D_all, p);
        } else {
            ehh_cur[0] = (double)S_pop[0] / (double)D_pop[0];
            ehh_cur[1] = (double)S_pop[1] / (double)D_pop[1];
            o.digest[0] += (uint64_t)(i + 1) * S_pop[0];
            o.digest[1] += (uint64_t)(i + 1) * S_pop[1];
            o.digest[2] += (uint64_t)(i + 1) * S_all;
            stop = below_cutoff(S_all, D_all, p);
        }
        if (stop && !p->include_crossing_term) {
            o.status = ST_OK; o.stop = (int32_t)i; break;
        }
        for (int q = 0; q < npop; ++q) {
            o.ihh[q] += 0.5 * (ehh_prev[q] + ehh_cur[q]) * g;
            ehh_prev[q] = ehh_cur[q];
        }
        if (stop) { o.status = ST_OK; o.stop = (int32_t)i; break; }
    }
    return o;
}

static int params_ok(const oracle_params *p)
{
    return p && p->ehh_cut_den > 0 && p->maf_den > 0 && p->ehh_cut_num <= p->ehh_cut_den &&
           p->maf_num <= p->maf_den && p->gap_scale_bp > 0 && p->max_gap_bp >= 0 &&
           (p->use_physical_map == 0 || p->use_physical_map == 1);
}

static void set_members(strings *s, int32_t n, const int32_t *list, const int8_t *popid,
                        const int64_t *woff)
{
    s->nmem = n;
    s->hap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    s->popid = (int8_t *)malloc((size_t)(n ? n : 1));
    s->word_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    s->idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    for (int32_t k = 0; k < n; ++k) {
        s->hap[k] = list[k];
        s->popid[k] = popid ? popid[k] : 0;
        s->word_off[k] = woff ? woff[k] : 0;
    }
    s->str = NULL; s->cap = 0; s->len = 0;
}

/* ---------------- iHS ---------------- */
int oracle_ihs(const uint64_t *rows, int64_t ld, int32_t n, int64_t m, const int64_t *pos,
               const double *gmap, const oracle_params *p, const int64_t *cores, int64_t ncores,
               int nthreads, int8_t *status, int32_t *n1_out, double *ihh1, double *ihh0,
               double *lnratio, int32_t *stop, uint64_t *digest)
{
    if (!rows || !pos || !gmap || n < 2 || m < 1 || ld < (n + 63) / 64 || !params_ok(p))
        return -1;
    if (!cores) ncores = m;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < ncores; ++k) {
        int64_t j = cores ? cores[k] : k;
        int32_t *carriers[2];
        int32_t nc[2] = {0, 0};
        carriers[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        carriers[1] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        for (int32_t h = 0; h < n; ++h) {
            int a = allele(rows, ld, j, 0, h);
            carriers[a][nc[a]++] = h;
        }
        n1_out[k] = nc[1];
        for (int q = 0; q < 4; ++q) { stop[4 * k + q] = 0; digest[4 * k + q] = 0; }
        ihh1[k] = 0.0; ihh0[k] = 0.0;
        uint32_t minor = nc[1] < nc[0] ? nc[1] : nc[0];
        /* MAF >= num/den  <=>  den * minor >= num * n (Section 1.2) */
        if ((uint64_t)p->maf_den * minor < (uint64_t)p->maf_num * (uint64_t)n) {
            status[k] = ST_MAF_FILTERED;
            lnratio[k] = NAN;
            free(carriers[0]); free(carriers[1]);
            continue;
        }
        int worst = ST_OK;
        double ihh[2] = {0.0, 0.0}; /* indexed by allele */
        /* item order: (allele 1, down), (allele 1, up), (allele 0, down), (allele 0, up) */
        for (int q = 0; q < 4; ++q) {
            int c = q < 2 ? 1 : 0, dir = q & 1;
            strings s;
            set_members(&s, nc[c], carriers[c], NULL, NULL);
            walk_out o = walk(rows, ld, m, pos, gmap, p, &s, 1, nc[c], 0, j, dir, NULL, 0);
            strings_free(&s);
            stop[4 * k + q] = o.stop;
            digest[4 * k + q] = o.digest[0];
            if (dir == 0) ihh[c] = o.ihh[0];
            else ihh[c] = ihh[c] + o.ihh[0];      /* iHH_c = downstream + upstream */
            if (o.status > worst) worst = o.status;
        }
        ihh1[k] = ihh[1];
        ihh0[k] = ihh[0];
        if (worst == ST_OK && (ihh[1] == 0.0 || ihh[0] == 0.0)) worst = ST_UNDEFINED;
        status[k] = (int8_t)worst;
        lnratio[k] = worst == ST_OK ? log(ihh[1] / ihh[0]) : NAN;
        free(carriers[0]); free(carriers[1]);
    }
    return 0;
}

/* ---------------- XPEHH ---------------- */
int oracle_xpehh(const uint64_t *rows, int64_t ld, int32_t nA, int32_t nB, int64_t m,
                 const int64_t *pos, const double *gmap, const oracle_params *p,
                 const int64_t *cores, int64_t ncores, int nthreads, int8_t *status,
                 int32_t *n1_out, double *ihhA, double *ihhB, double *lnratio, int32_t *stop,
                 uint64_t *digest)
{
    const int64_t WA = (nA + 63) / 64, WB = (nB + 63) / 64;
    if (!rows || !pos || !gmap || nA < 2 || nB < 2 || m < 1 || ld < WA + WB || !params_ok(p))
        return -1;
    if (!cores) ncores = m;
    const int32_t nt = nA + nB;
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)nt);
    int8_t *pid = (int8_t *)malloc((size_t)nt);
    int64_t *woff = (int64_t *)malloc(sizeof(int64_t) * (size_t)nt);
    for (int32_t h = 0; h < nA; ++h) { list[h] = h; pid[h] = 0; woff[h] = 0; }
    for (int32_t h = 0; h < nB; ++h) { list[nA + h] = h; pid[nA + h] = 1; woff[nA + h] = WA; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < ncores; ++k) {
        int64_t j = cores ? cores[k] : k;
        int32_t c1 = 0;
        for (int32_t t = 0; t < nt; ++t) c1 += allele(rows, ld, j, woff[t], list[t]);
        n1_out[k] = c1;
        for (int q = 0; q < 2; ++q) stop[2 * k + q] = 0;
        for (int q = 0; q < 6; ++q) digest[6 * k + q] = 0;
        ihhA[k] = 0.0; ihhB[k] = 0.0;
        uint32_t minor = (uint32_t)(c1 < nt - c1 ? c1 : nt - c1);
        if (p->xpehh_maf_filter &&
            (uint64_t)p->maf_den * minor < (uint64_t)p->maf_num * (uint64_t)nt) {
            status[k] = ST_MAF_FILTERED;
            lnratio[k] = NAN;
            continue;
        }
        int worst = ST_OK;
        double ia = 0.0, ib = 0.0;
        for (int dir = 0; dir < 2; ++dir) {
            strings s;
            set_members(&s, nt, list, pid, woff);
            walk_out o = walk(rows, ld, m, pos, gmap, p, &s, 2, nA, nB, j, dir, NULL, 0);
            strings_free(&s);
            stop[2 * k + dir] = o.stop;
            for (int q = 0; q < 3; ++q) digest[6 * k + 3 * dir + q] = o.digest[q];
            if (dir == 0) { ia = o.ihh[0]; ib = o.ihh[1]; }
            else { ia = ia + o.ihh[0]; ib = ib + o.ihh[1]; }
            if (o.status > worst) worst = o.status;
        }
        ihhA[k] = ia;
        ihhB[k] = ib;
        if (worst == ST_OK && (ia == 0.0 || ib == 0.0)) worst = ST_UNDEFINED;
        status[k] = (int8_t)worst;
        lnratio[k] = worst == ST_OK ? log(ia / ib) : NAN;
    }
    free(list); free(pid); free(woff);
    return 0;
}

/* ---------------- single-locus EHH report ---------------- */
/*
 * Walks w = 0 (carriers of allele 1, Eq. 3), w = 1 (carriers of allele 0,
 * Eq. 3), w = 2 (whole sample, Eq. 1) in both directions from `locus`.
 * Arrays are indexed [w * 2 + dir]; S has capacity entries per walk:
 * S[(w * 2 + dir) * capacity + i].  len = number of S values the walk
 * computed (may exceed capacity; only the first capacity are stored).
 * denom[w] = C(N_w, 2).
 */
int oracle_ehh(const uint64_t *rows, int64_t ld, int32_t n, int64_t m, const int64_t *pos,
               const double *gmap, const oracle_params *p, int64_t locus, int64_t capacity,
               uint64_t *S, int64_t *len, int32_t *stop, int8_t *status, double *ihh,
               uint64_t *denom)
{
    if (!rows || !pos || !gmap || n < 2 || m < 1 || locus < 0 || locus >= m ||
        ld < (n + 63) / 64 || !params_ok(p) || capacity < 0)
        return -1;
    int32_t *carriers[3];
    int32_t nc[3] = {0, 0, n};
    for (int w = 0; w < 3; ++w) carriers[w] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t h = 0; h < n; ++h) {
        int a = allele(rows, ld, locus, 0, h);
        int w = a ? 0 : 1;
        carriers[w][nc[w]++] = h;
        carriers[2][h] = h;
    }
    for (int w = 0; w < 3; ++w) {
        denom[w] = choose2((uint64_t)nc[w]);
        for (int dir = 0; dir < 2; ++dir) {
            strings s;
            set_members(&s, nc[w], carriers[w], NULL, NULL);
            walk_out o = walk(rows, ld, m, pos, gmap, p, &s, 1, nc[w], 0, locus, dir,
                              S + (int64_t)(w * 2 + dir) * capacity, capacity);
            strings_free(&s);
            len[w * 2 + dir] = o.steps;
            stop[w * 2 + dir] = o.stop;
            status[w * 2 + dir] = (int8_t)o.status;
            ihh[w * 2 + dir] = o.ihh[0];
        }
    }
    for (int w = 0; w < 3; ++w) free(carriers[w]);
    return 0;
}
