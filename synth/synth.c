/*
 * Seeded synthetic haplotype generator (input data only; holds none of the
 * EHH / iHH arithmetic).  It stands in for the paper's simulated (ms) and
 * 1000 Genomes chromosome-22 inputs (Section 2), which are not available:
 * phased biallelic 0/1 haplotypes (0 = ancestral, 1 = derived, Section 1.1),
 * physical positions in bp and a genetic map in cM.
 *
 * Model: a Li-Stephens style mosaic of F founder haplotypes.
 *   - founders: per SNP a derived count k ~ P(k) proportional to 1/k on
 *     1..F-1, carried by a uniformly drawn k-subset of founders;
 *   - each sampled haplotype copies one founder at a time and jumps to a
 *     uniformly drawn founder at the events of a Poisson process along the
 *     genetic map with rate lambda per cM (so a jump happens between two
 *     markers with probability 1 - exp(-lambda * dg));
 *   - every allele then flips independently with probability flip_prob;
 *   - planted sweeps: a set of carriers is given allele 1 at the sweep's core
 *     marker (everyone else 0) and one identical template haplotype on every
 *     marker within +-width/2 bp of it.
 *
 * Randomness is counter based: every draw is SplitMix64's output function
 * (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) applied to a key derived from (seed, stream, index) plus a
 * counter, so the data do not depend on thread count or machine.  All
 * floating point is plain IEEE add/sub/mul/div (compile with
 * -ffp-contract=off); the only transcendental needed, a logarithm for
 * exponential / geometric draws, is computed here by a fixed series so that
 * x86-64 and aarch64 hosts produce bit-identical matrices.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* key for an independent stream (seed, stream id, index) */
static inline uint64_t sm_key(uint64_t seed, uint64_t stream, uint64_t index)
{
    return sm_mix(seed * GOLDEN ^ sm_mix(stream + GOLDEN * (index + 1)));
}

/* draw number ctr of a stream */
static inline uint64_t sm_draw(uint64_t key, uint64_t ctr)
{
    return sm_mix(key + GOLDEN * (ctr + 1));
}

/* uniform in [0, 1) with 53 random bits */
static inline double sm_unif(uint64_t key, uint64_t ctr)
{
    return (double)(sm_draw(key, ctr) >> 11) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, k) (k > 0) by multiply-shift on 32 bits */
static inline uint32_t sm_below(uint64_t key, uint64_t ctr, uint32_t k)
{
    uint64_t r = sm_draw(key, ctr) >> 32;
    return (uint32_t)((r * (uint64_t)k) >> 32);
}

/*
 * Natural logarithm of x > 0 from basic operations only:
 * x = f * 2^e with f in [sqrt(1/2), sqrt(2)), ln x = e ln 2 + 2 atanh(t),
 * t = (f-1)/(f+1), |t| < 0.172, atanh by its Taylor series (25 terms, far
 * below double rounding).  Used only to shape random draws.
 */
static double det_log(double x)
{
    int e;
    double f = frexp(x, &e); /* exact; f in [0.5, 1) */
    if (f < 0.70710678118654752) { f *= 2.0; e -= 1; }
    double t = (f - 1.0) / (f + 1.0);
    double t2 = t * t, term = t, s = 0.0;
    for (int k = 0; k < 25; ++k) {
        s += term / (double)(2 * k + 1);
        term *= t2;
    }
    return (double)e * 0.69314718055994531 + 2.0 * s;
}

/* exponential(1) draw: -ln(1 - u), u in [0,1) */
static inline double sm_exp1(uint64_t key, uint64_t ctr)
{
    return -det_log(1.0 - sm_unif(key, ctr));
}

enum { ST_POS = 1, ST_MAP = 2, ST_FOUNDER = 3, ST_SWITCH = 4, ST_FLIP = 5,
       ST_CARRIER = 6, ST_SUBSET = 7, ST_USER = 100 };

/* ------------------------------------------------------------------ */
/* public: one uniform draw for callers that need sweep / request params */
double synth_uniform(uint64_t seed, uint64_t stream, uint64_t index)
{
    return sm_unif(sm_key(seed, ST_USER + stream, index), 0);
}

/*
 * Positions: m strictly increasing integers in [1, len_bp - gap_total]
 * (sorted uniforms from normalised exponential spacings, plus rank), then
 * n_gaps planted gaps: the step into marker gap_idx[g] is set to exactly
 * gap_bp[g] bp and every later position shifts with it.
 * Map: constant rate (cM/Mb) if map_spread == 0, otherwise a rate drawn
 * per 1 Mb segment uniformly in rate*(1 +- spread); gmap = integral.
 * Returns 0, or -1 on bad arguments.
 */
int synth_positions_map(uint64_t seed, int64_t m, int64_t len_bp,
                        int32_t n_gaps, const int64_t *gap_idx,
                        const int64_t *gap_bp, double map_rate,
                        double map_spread, int64_t *pos, double *gmap)
{
    if (m < 1 || len_bp < m) return -1;
    int64_t gap_total = 0;
    for (int g = 0; g < n_gaps; ++g) {
        if (gap_idx[g] < 1 || gap_idx[g] >= m || gap_bp[g] < 1) return -1;
        gap_total += gap_bp[g];
    }
    int64_t span = len_bp - gap_total - m; /* free room for the draws */
    if (span < 0) return -1;
    uint64_t key = sm_key(seed, ST_POS, 0);
    double total = 0.0;
    double *cum = (double *)malloc(sizeof(double) * (size_t)m);
    if (!cum) return -1;
    for (int64_t k = 0; k < m; ++k) {
        total += sm_exp1(key, (uint64_t)k);
        cum[k] = total;
    }
    total += sm_exp1(key, (uint64_t)m);
    for (int64_t k = 0; k < m; ++k) {
        int64_t off = (int64_t)((cum[k] / total) * (double)span);
        if (off > span) off = span;
        pos[k] = 1 + off + k;
    }
    free(cum);
    /* planted gaps, applied in index order */
    for (int g = 0; g < n_gaps; ++g) {
        int64_t k = gap_idx[g];
        int64_t shift = pos[k - 1] + gap_bp[g] - pos[k];
        for (int64_t j = k; j < m; ++j) pos[j] += shift;
    }
    /* genetic map, cM */
    uint64_t mkey = sm_key(seed, ST_MAP, 0);
    double g = 0.0;
    int64_t prev = 0; /* bp at which g was last evaluated */
    for (int64_t k = 0; k < m; ++k) {
        int64_t p = pos[k];
        while (prev < p) {
            int64_t seg = prev / 1000000;
            int64_t seg_end = (seg + 1) * 1000000;
            int64_t upto = p < seg_end ? p : seg_end;
            double rate = map_rate;
            if (map_spread != 0.0)
                rate = map_rate * (1.0 - map_spread + 2.0 * map_spread * sm_unif(mkey, (uint64_t)seg));
            g += rate * ((double)(upto - prev) * 1e-6);
            prev = upto;
        }
        gmap[k] = g;
    }
    return 0;
}

/*
 * Founder matrix: F founders x m markers, marker-major, fw = ceil(F/64) words
 * per marker.  Derived count per marker ~ 1/k on 1..F-1; a uniform k-subset
 * is drawn by a partial Fisher-Yates shuffle.
 */
static void make_founders(uint64_t seed, uint64_t stream, int32_t F, int64_t m,
                          uint64_t *fwords)
{
    int fw = (F + 63) / 64;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)F);
    double acc = 0.0;
    for (int k = 1; k < F; ++k) { acc += 1.0 / (double)k; cdf[k] = acc; }
    #pragma omp parallel
    {
        int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)F);
        #pragma omp for schedule(static)
        for (int64_t j = 0; j < m; ++j) {
            uint64_t key = sm_key(seed, stream, (uint64_t)j);
            double u = sm_unif(key, 0) * acc;
            int k = 1;
            while (k < F - 1 && cdf[k] <= u) ++k;
            for (int f = 0; f < F; ++f) perm[f] = f;
            uint64_t *w = fwords + (size_t)j * fw;
            for (int q = 0; q < fw; ++q) w[q] = 0;
            for (int s = 0; s < k; ++s) {
                int r = s + (int)sm_below(key, (uint64_t)(1 + s), (uint32_t)(F - s));
                int32_t t = perm[s]; perm[s] = perm[r]; perm[r] = t;
                w[perm[s] >> 6] |= 1ULL << (perm[s] & 63);
            }
        }
        free(perm);
    }
    free(cdf);
}

typedef struct {
    int32_t n;              /* haplotypes of this population */
    int32_t founders;       /* F >= 2 */
    double switch_per_cM;   /* lambda */
    double flip_prob;       /* independent allele flips */
    int32_t n_sweeps;
    const double *sweep_center_bp; /* physical centre of each sweep */
    const double *sweep_width_bp;
    const double *sweep_freq;      /* carrier fraction */
} synth_pop;

/* geometric skip: number of failures before the next success, p in (0,1) */
static inline int64_t geom_skip(uint64_t key, uint64_t ctr, double log1mp)
{
    double u = sm_unif(key, ctr);
    double v = det_log(1.0 - u) / log1mp;
    if (v > 9.0e18) return (int64_t)9e18;
    return (int64_t)v;
}

/*
 * Haplotypes of one population into marker-major packed rows.  Haplotype h
 * is bit (h % 64) of word word_off + h / 64 of each row; row k starts at
 * rows + k * ld.  Pad bits above n in the last word are written as 0; words
 * outside [word_off, word_off + ceil(n/64)) are not touched.
 */
int synth_haplotypes(uint64_t seed, uint64_t pop_stream, const synth_pop *pp,
                     int64_t m, const int64_t *pos, const double *gmap,
                     uint64_t *rows, int64_t ld, int64_t word_off)
{
    const int32_t n = pp->n, F = pp->founders;
    if (n < 1 || F < 2 || m < 1 || ld < word_off + (n + 63) / 64) return -1;
    const int fw = (F + 63) / 64;
    const int W = (n + 63) / 64;
    uint64_t *fwords = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)fw * (size_t)m);
    if (!fwords) return -1;
    make_founders(seed, pop_stream * 16 + ST_FOUNDER, F, m, fwords);
    const double lam = pp->switch_per_cM;
    const double log1mp = det_log(1.0 - pp->flip_prob);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < W; ++b) {
        int nb = (n - 64 * b) < 64 ? (n - 64 * b) : 64;
        int32_t cur[64];
        double next_sw[64];
        int64_t next_flip[64];
        uint64_t ksw[64], kfl[64], csw[64], cfl[64];
        for (int t = 0; t < nb; ++t) {
            uint64_t h = (uint64_t)(64 * b + t);
            ksw[t] = sm_key(seed, pop_stream * 16 + ST_SWITCH, h);
            kfl[t] = sm_key(seed, pop_stream * 16 + ST_FLIP, h);
            csw[t] = 0; cfl[t] = 0;
            cur[t] = (int32_t)sm_below(ksw[t], csw[t]++, (uint32_t)F);
            next_sw[t] = lam > 0.0 ? gmap[0] + sm_exp1(ksw[t], csw[t]++) / lam : 1e300;
            next_flip[t] = pp->flip_prob > 0.0 ? geom_skip(kfl[t], cfl[t]++, log1mp) : INT64_MAX;
        }
        for (int64_t k = 0; k < m; ++k) {
            const double gk = gmap[k];
            const uint64_t *fk = fwords + (size_t)k * fw;
            uint64_t word = 0;
            for (int t = 0; t < nb; ++t) {
                while (gk >= next_sw[t]) {
                    cur[t] = (int32_t)sm_below(ksw[t], csw[t]++, (uint32_t)F);
                    next_sw[t] += sm_exp1(ksw[t], csw[t]++) / lam;
                }
                uint64_t bit = (fk[cur[t] >> 6] >> (cur[t] & 63)) & 1ULL;
                if (k == next_flip[t]) {
                    bit ^= 1ULL;
                    int64_t s = geom_skip(kfl[t], cfl[t]++, log1mp);
                    next_flip[t] = (s > INT64_MAX - k - 1) ? INT64_MAX : k + 1 + s;
                }
                word |= bit << t;
            }
            rows[(size_t)k * ld + word_off + b] = word;
        }
    }
    free(fwords);

    /* planted sweeps */
    for (int s = 0; s < pp->n_sweeps; ++s) {
        double c = pp->sweep_center_bp[s], half = 0.5 * pp->sweep_width_bp[s];
        /* core marker: nearest position to the centre (first on ties) */
        int64_t lo = 0, hi = m - 1;
        while (lo < hi) { /* first k with pos[k] >= c */
            int64_t mid = (lo + hi) / 2;
            if ((double)pos[mid] < c) lo = mid + 1; else hi = mid;
        }
        int64_t core = lo;
        if (core > 0 && (c - (double)pos[core - 1]) <= ((double)pos[core] - c)) core -= 1;
        int64_t ncar = (int64_t)(pp->sweep_freq[s] * (double)n + 0.5);
        if (ncar < 1) ncar = 1;
        if (ncar > n) ncar = n;
        /* carriers: uniform ncar-subset by partial Fisher-Yates */
        int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        uint64_t *cw = (uint64_t *)calloc((size_t)W, sizeof(uint64_t));
        uint64_t ckey = sm_key(seed, pop_stream * 16 + ST_CARRIER, (uint64_t)s);
        for (int i = 0; i < n; ++i) perm[i] = i;
        int32_t templ = n;
        for (int64_t i = 0; i < ncar; ++i) {
            int64_t r = i + (int64_t)sm_below(ckey, (uint64_t)i, (uint32_t)(n - i));
            int32_t t = perm[i]; perm[i] = perm[r]; perm[r] = t;
            cw[perm[i] >> 6] |= 1ULL << (perm[i] & 63);
            if (perm[i] < templ) templ = perm[i];
        }
        for (int64_t k = 0; k < m; ++k) {
            double d = (double)pos[k] - (double)pos[core];
            if (d < -half || d > half) continue;
            uint64_t *row = rows + (size_t)k * ld + word_off;
            if (k == core) {
                for (int w = 0; w < W; ++w) row[w] = cw[w];
            } else {
                uint64_t tb = (row[templ >> 6] >> (templ & 63)) & 1ULL;
                for (int w = 0; w < W; ++w)
                    row[w] = tb ? (row[w] | cw[w]) : (row[w] & ~cw[w]);
            }
        }
        free(perm);
        free(cw);
    }
    return 0;
}
