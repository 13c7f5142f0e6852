// EHH walk executed by one warp (device code, sm_103a).
//
// One walk = one core x_0, one direction and one sample (the carriers of a
// core allele for EHH_c, Eq. 3; a whole population for EHH, Eq. 1; or two
// pooled populations for XPEHH, Section 1.3).  The partition of the sample
// into distinct extended haplotypes (Section 1.1) is kept group-major:
//   pool   8-byte entries, 32-bit member mask | 32-bit word index << 32;
//          every group owns one contiguous range of entries (only words in
//          which it has members);
//   table  one row per group: start, number of entries, member count
//          (population A | population B << 16), rows in pool order.
// Groups of fewer than two haplotypes are dropped: they add nothing to any
// C(n_h, 2) and can never grow.
//
// Moving from x_{i-1} to x_i splits group g by the allele row into a members
// with allele 1 and b with allele 0; the homozygosity numerator drops by
// C(a+b,2) - C(a,2) - C(b,2) = a * b.  S is an exact integer and the stop
// test den * S < num * C(N,2) is exact.
//
// One step, one warp:
//   small groups (fewer than 32 entries): a lane owns a group and walks its
//          entries, a = sum popc(mask & row); no atomics, no reductions;
//   big groups: the whole warp takes the group's entries, one warp sum;
//   a group splits iff 0 < a < size; only split groups are rewritten: the
//          allele-1 half stays in place, the allele-0 half (if both survive)
//          goes to a new range at the pool end and a new row at the table end.
// Unused pool space and dead rows are squeezed out by compactions that keep
// pool order.  Pool entries [0, cap_s) and table rows [0, tcap_s) live in the
// warp's shared-memory slice, the rest in its global scratch slice.
#pragma once
#include <stdint.h>

#define FULLMASK 0xffffffffu

namespace selscan {

// Internal walk outcomes (the first five equal the public locus codes).
enum : int {
    WALK_OK = 0, WALK_UNDEFINED = 2, WALK_EDGE = 3, WALK_GAP = 4, WALK_UNFINISHED = 5
};


struct ScanArgs {
    const unsigned long long *hap;  // rows, row k at hap + k * ld (64-bit words)
    long long ld;
    long long m;                     // markers (walks may reach any of them)
    long long k0, k1;                // the cores of this call: [k0, k1) (a whole scan: [0, m));
                                     // per-core outputs are indexed by the global core k,
                                     // through pointers the host has offset by k0
    const long long *pos;
    const double *gmap;
    int W;                           // 64-bit words in use (iHS: W; XPEHH: W_A + W_B)
    int WA;                          // 64-bit words of population A (iHS: = W)
    int nA, nB;                      // population sizes (iHS: n, 0)
    unsigned long long lastA;        // valid bits of word WA - 1
    unsigned long long lastB;        // valid bits of word W - 1 (XPEHH)
    unsigned int cut_num, cut_den;
    long long gap_scale, max_gap;
    int crossing;
    int physical;                    // g = physical distance instead of the genetic map
};

// One warp's buffers: tier 0 on chip, tier 1 in global scratch.
struct WarpBufs {
    unsigned long long *pool_s;   // entries [0, cap_s)
    unsigned long long *pool_g;   // entries [cap_s, cap) at pool_g[e - cap_s]
    unsigned long long *tab_s, *tab_g;  // table rows: start | entries << 20 | members (A | B << 16) << 32
    unsigned short *big;          // rows of big groups this step (global)
    int cap_s, cap;               // pool capacities (on chip, total)
    int tcap_s, tcap;             // table capacities
    int *err;                     // device error word (consistency checks)
    // marker window: two buffers of R rows (+ positions and map values),
    // filled by bulk copies (TMA) ahead of the walk
    unsigned char *wrow[2];
    long long *wpos[2];
    double *wgm[2];
    unsigned long long *bar;      // one mbarrier per buffer
    int R;
    int bigt;                     // groups with at least this many entries use the whole warp
};

struct WalkOut {
    int status;
    int stop;
    double ihh[2];
    unsigned long long dig[3];
    unsigned long long D;            // C(N,2) of the walk's sample (pooled for XPEHH)
    float key;                       // EHH at the step cap (unfinished walks)
    bool abandon;                    // a bounded wait for the warp's window copies gave
                                     // up: a copy may still land in its buffers, so the
                                     // warp must not start another walk
};

// Sum of the partial sums of G consecutive lanes (a warp, or half of one),
// by a butterfly in a fixed order; every lane gets the sum, lane 0's is used.
template <int G>
__device__ __forceinline__ double lane_sum_f64(double v)
{
    const unsigned mask = G == 32 ? 0xFFFFFFFFu : (0xFFFFu << (threadIdx.x & 16));
#pragma unroll
    for (int d = G / 2; d > 0; d >>= 1) v += __shfl_xor_sync(mask, v, d);
    return v;
}

__device__ __forceinline__ unsigned int lanemask_lt()
{
    unsigned int r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned long long choose2(unsigned long long k)
{
    return k * (k - 1ull) / 2ull;
}

// EHH < num/den  <=>  den * S < num * D  (S, D < 2^31, num, den < 2^32: no overflow)
__device__ __forceinline__ bool below_cut(const ScanArgs &a, unsigned long long S,
                                          unsigned long long D)
{
    return (unsigned long long)a.cut_den * S < (unsigned long long)a.cut_num * D;
}

// valid bits of 32-bit word w32 of the row (pad bits and pad words are 0)
__device__ __forceinline__ unsigned int valid32(const ScanArgs &a, int w32)
{
    const int base = w32 < 2 * a.WA ? 0 : 2 * a.WA;
    const int n = w32 < 2 * a.WA ? a.nA : a.nB;
    const int k = w32 - base;                 // 32-bit word within the population
    const int full = n >> 5, rem = n & 31;
    if (k < full) return FULLMASK;
    if (k == full && rem) return (1u << rem) - 1u;
    return 0u;
}

__device__ __forceinline__ unsigned long long *pent(const WarpBufs &b, unsigned e)
{
    return (int)e < b.cap_s ? b.pool_s + e : b.pool_g + (e - (unsigned)b.cap_s);
}

__device__ __forceinline__ unsigned long long *trow(const WarpBufs &b, int r)
{
    return r < b.tcap_s ? b.tab_s + r : b.tab_g + r;
}

__device__ __forceinline__ unsigned long long mktab(unsigned st, unsigned ln, unsigned sz)
{
    return (unsigned long long)(st | (ln << 20)) | ((unsigned long long)sz << 32);
}
__device__ __forceinline__ unsigned tab_st(unsigned long long t) { return (unsigned)t & 0xfffffu; }
__device__ __forceinline__ unsigned tab_ln(unsigned long long t) { return ((unsigned)t >> 20) & 0xfffu; }
__device__ __forceinline__ unsigned tab_sz(unsigned long long t) { return (unsigned)(t >> 32); }

__device__ __forceinline__ unsigned lds32(unsigned addr)
{
    unsigned v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ long long lds64(unsigned addr)
{
    long long v;
    asm volatile("ld.shared.s64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ double ldsf64(unsigned addr)
{
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ unsigned long long mkent(unsigned int mask, unsigned int w)
{
    return (unsigned long long)mask | ((unsigned long long)w << 32);
}

// ---------------------------------------------------------------- TMA window
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0u;
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

constexpr long long kWaitLimit = 1ll << 22;   // try_wait rounds before a wait gives up

// One window buffer: rows [lo, hi] of the walk, positions and map values
// [plo, ...]; roff / poff / goff locate them in the buffer.
struct WinBuf {
    int lo, hi, plo;
    int roff, poff, goff;
    bool pending;
    unsigned parity;
};

// Fill buffer bi with the rows of steps [s, s + R) from `core` in direction dir.
__device__ __forceinline__ void win_issue(const ScanArgs &a, const WarpBufs &b, WinBuf &w, int bi,
                                          long long core, int dir, long long s)
{
    long long lo, hi;
    if (dir) { lo = core + s; hi = core + s + b.R - 1; if (hi > a.m - 1) hi = a.m - 1; }
    else { hi = core - s; lo = core - s - b.R + 1; if (lo < 0) lo = 0; }
    w.lo = (int)lo;
    w.hi = (int)hi;
    w.pending = false;
    if (lo > hi) return;                      // past the array end: the walk stops before
    const long long plo = lo > 0 ? lo - 1 : 0, phi = hi + 1 < a.m ? hi + 1 : a.m - 1;
    w.plo = (int)plo;
    __syncwarp();
    fence_proxy_async();                      // earlier reads of this buffer precede the copies
    const unsigned char *src[3] = {
        (const unsigned char *)a.hap + (size_t)lo * (size_t)a.ld * 8u,
        (const unsigned char *)a.pos + (size_t)plo * 8u,
        (const unsigned char *)a.gmap + (size_t)plo * 8u};
    const unsigned char *base[3] = {(const unsigned char *)a.hap, (const unsigned char *)a.pos,
                                    (const unsigned char *)a.gmap};
    const size_t total[3] = {(size_t)a.m * (size_t)a.ld * 8u, (size_t)a.m * 8u, (size_t)a.m * 8u};
    unsigned char *dst[3] = {b.wrow[bi], (unsigned char *)b.wpos[bi], (unsigned char *)b.wgm[bi]};
    const unsigned bytes[3] = {(unsigned)((hi - lo + 1) * a.ld * 8), (unsigned)((phi - plo + 1) * 8),
                               (unsigned)((phi - plo + 1) * 8)};
    int off[3];
    unsigned len[3];
    bool bulk[3];
    unsigned tx = 0u;
    // a bulk copy of the 16-byte-aligned span around each piece when that span
    // stays inside its array, else plain loads by the warp
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        off[q] = (int)((uintptr_t)src[q] & 15u);
        len[q] = (bytes[q] + (unsigned)off[q] + 15u) & ~15u;
        bulk[q] = src[q] - off[q] >= base[q] && src[q] - off[q] + len[q] <= base[q] + total[q];
        if (bulk[q]) tx += len[q];
    }
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        if (tx) mbar_expect_tx(b.bar + bi, tx);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (bulk[q]) bulk_g2s(dst[q], src[q] - off[q], len[q], b.bar + bi);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (!bulk[q])
            for (unsigned k = (unsigned)lane; k < bytes[q] / 8u; k += 32u)
                ((unsigned long long *)(dst[q] + off[q]))[k] = ((const unsigned long long *)src[q])[k];
    w.roff = off[0];
    w.poff = off[1] / 8;
    w.goff = off[2] / 8;
    w.pending = tx != 0u;
    __syncwarp();
}

// Wait (bounded) for buffer bi's copies; false if the wait gave up.
__device__ __forceinline__ bool win_wait(const WarpBufs &b, WinBuf &w, int bi)
{
    if (!w.pending) return true;
    bool done = false;
    for (long long t = 0; t < kWaitLimit && !done; ++t) done = mbar_try_wait(b.bar + bi, w.parity);
    done = __all_sync(FULLMASK, done);
    if (!done) {
        if ((threadIdx.x & 31) == 0) atomicExch(b.err, -5);   // SELSCAN_ERR_TIMEOUT
        return false;
    }
    w.parity ^= 1u;
    w.pending = false;
    return true;
}

// Per-walk mutable state (warp-uniform).
struct ListState {
    int P;        // pool end (entries in use, including unused tails)
    int live;     // entries of live groups
    int G;        // table rows (including dead ones)
    int dead;     // dead rows
};

// Split decision from the allele-1 counts `ones` (A | B << 16) and the
// member counts `sz` (A | B << 16) of one group.  Adds the numerator drops
// to d[0..2] (NPOP 1: [0]; NPOP 2: A, B, pooled) and returns whether it
// splits; k1 / k0 say which halves survive and ones/zeros their sizes.
template <int NPOP>
__device__ __forceinline__ bool decide(unsigned int ones, unsigned int sz, unsigned int d[3],
                                       bool &k1, bool &k0, unsigned int &z)
{
    const unsigned int oA = ones & 0xffffu, oB = ones >> 16;
    const unsigned int sA = sz & 0xffffu, sB = sz >> 16;
    const unsigned int zA = sA - oA, zB = sB - oB;
    const unsigned int o = oA + oB, zz = zA + zB;
    z = zA | (zB << 16);
    if (o == 0u || zz == 0u) return false;
    if (NPOP == 2) {
        d[0] += oA * zA;
        d[1] += oB * zB;
        d[2] += o * zz;
    } else {
        d[0] += o * zz;
    }
    k1 = o >= 2u;
    k0 = zz >= 2u;
    return true;
}

// Drop unused pool space: move each live group's range down, in pool order.
static __device__ __noinline__ void compact_pool(const WarpBufs &b, ListState &L)
{
    const int lane = threadIdx.x & 31;
    int out = 0;
    for (int r = 0; r < L.G; ++r) {
        unsigned long long *tp = trow(b, r);
        const unsigned long long t = *tp;
        const int ln = (int)tab_ln(t);
        if (ln == 0) continue;
        const int st = (int)tab_st(t);
        if (st != out) {
            // chunk-wise forward copy: destination <= source, each chunk read first
            for (int k0 = 0; k0 < ln; k0 += 32) {
                const int k = k0 + lane;
                unsigned long long v = 0ull;
                if (k < ln) v = *pent(b, (unsigned)(st + k));
                __syncwarp();
                if (k < ln) *pent(b, (unsigned)(out + k)) = v;
                __syncwarp();
            }
            if (lane == 0) *tp = mktab((unsigned)out, (unsigned)ln, tab_sz(t));
        }
        out += ln;
    }
    __syncwarp();
    L.P = out;
}

// Drop dead table rows (pool order kept).
static __device__ __noinline__ void compact_table(const WarpBufs &b, ListState &L)
{
    const int lane = threadIdx.x & 31;
    const unsigned ltm = lanemask_lt();
    int out = 0;
    for (int r0 = 0; r0 < L.G; r0 += 32) {
        const int r = r0 + lane;
        unsigned long long t = 0ull;
        if (r < L.G) t = *trow(b, r);
        const bool keep = tab_ln(t) != 0u;
        const unsigned bal = __ballot_sync(FULLMASK, keep);
        __syncwarp();
        if (keep) *trow(b, out + __popc(bal & ltm)) = t;
        out += __popc(bal);
        __syncwarp();
    }
    L.G = out;
    L.dead = 0;
}

// A split that removes exactly one member (the usual case once founder
// groups have formed): clear its bit in entry k of the group at row r (the
// entry's allele-`one` bit when one != 0, else its allele-0 bit); an entry
// left empty takes the group's last entry.  Returns the change in entries.
__device__ __forceinline__ int drop_one(const WarpBufs &b, unsigned row_sa, int r, unsigned st,
                                        unsigned ln, unsigned k, bool one, unsigned sz_new)
{
    unsigned long long *pe = pent(b, st + k);
    const unsigned long long v = *pe;
    const unsigned w = (unsigned)(v >> 32);
    const unsigned rr = lds32(row_sa + 4u * w);
    const unsigned nm = (unsigned)v & (one ? ~rr : rr);
    if (nm) {
        *pe = mkent(nm, w);
        *trow(b, r) = mktab(st, ln, sz_new);
        return 0;
    }
    *pe = *pent(b, st + ln - 1u);
    *trow(b, r) = mktab(st, ln - 1u, sz_new);
    return -1;
}

// Split every group by the row at shared address row_sa (32-bit words).
// d[] receives the drops of the homozygosity numerators (NPOP 1: [0];
// NPOP 2: A, B, pooled).
template <int NPOP>
__device__ __forceinline__ void split_step(const ScanArgs &a, unsigned row_sa, const WarpBufs &b,
                                           ListState &L, unsigned int dS[3])
{
    const int lane = threadIdx.x & 31;
    const unsigned ltm = lanemask_lt();
    const unsigned wsplit = 2u * (unsigned)a.WA;   // first 32-bit word of population B

    // room for this step's appends: at most one new range per live entry and
    // one new row per live group
    if (2 * L.P > b.cap || L.P > 2 * L.live + 64) compact_pool(b, L);
    if (2 * L.G > b.tcap || (L.dead > 32 && 2 * L.dead > L.G)) compact_table(b, L);

    unsigned int d[3] = {0u, 0u, 0u};
    const int G0 = L.G;
    int nbig = 0;

    // ---- small groups: one lane per group
    for (int r0 = 0; r0 < G0; r0 += 32) {
        const int r = r0 + lane;
        unsigned long long t = 0ull;
        if (r < G0) t = *trow(b, r);
        const unsigned st = tab_st(t), ln = tab_ln(t), sz = tab_sz(t);
        const bool isbig = ln >= (unsigned)b.bigt;
        const unsigned bb = __ballot_sync(FULLMASK, isbig);
        if (isbig) b.big[nbig + __popc(bb & ltm)] = (unsigned short)r;
        nbig += __popc(bb);
        const unsigned n_small = isbig ? 0u : ln;

        unsigned int ones = 0u, k1l = 0u, k0l = 0u;
        for (unsigned k = 0; k < n_small; ++k) {
            const unsigned long long v = *pent(b, st + k);
            const unsigned w = (unsigned)(v >> 32), mk = (unsigned)v;
            const unsigned rr = lds32(row_sa + 4u * w);
            const unsigned c = (unsigned)__popc(mk & rr);
            ones += (NPOP == 2 && w >= wsplit) ? (c << 16) : c;
            if (mk & rr) k1l = k;
            if (mk & ~rr) k0l = k;
        }
        bool k1 = false, k0 = false;
        unsigned int z = 0u;
        const bool split = n_small && decide<NPOP>(ones, sz, d, k1, k0, z);
        const bool both = split && k1 && k0;

        int dl = 0;
        if (split && !both) {
            if (k1) dl = drop_one(b, row_sa, r, st, ln, k0l, false, ones);       // one allele-0 member leaves
            else if (k0) dl = drop_one(b, row_sa, r, st, ln, k1l, true, z);      // one allele-1 member leaves
            else { *trow(b, r) = mktab(st, 0u, 0u); dl = -(int)ln; }             // 1 + 1: the group dies
        }

        // both halves survive: a new pool range (ln entries) and a new table row
        const unsigned bboth = __ballot_sync(FULLMASK, both);
        if (bboth) {
            unsigned int need = both ? ln : 0u, inc = need;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int tt = __shfl_up_sync(FULLMASK, inc, o);
                if (lane >= o) inc += tt;
            }
            const unsigned base0 = (unsigned)L.P + inc - need;
            const int nrow = L.G + __popc(bboth & ltm);
            L.P += (int)__shfl_sync(FULLMASK, inc, 31);
            L.G += __popc(bboth);
            if (both) {
                unsigned w1 = 0, w0 = 0;
                for (unsigned k = 0; k < ln; ++k) {
                    const unsigned long long v = *pent(b, st + k);
                    const unsigned w = (unsigned)(v >> 32), mk = (unsigned)v;
                    const unsigned rr = lds32(row_sa + 4u * w);
                    const unsigned o1 = mk & rr, o0 = mk & ~rr;
                    if (o1) *pent(b, st + w1++) = mkent(o1, w);
                    if (o0) *pent(b, base0 + w0++) = mkent(o0, w);
                }
                *trow(b, r) = mktab(st, w1, ones);
                *trow(b, nrow) = mktab(base0, w0, z);
                dl = (int)(w1 + w0) - (int)ln;
            }
        }
        L.live += (int)__reduce_add_sync(FULLMASK, (unsigned)dl);
        L.dead += __popc(__ballot_sync(FULLMASK, split && !k1 && !k0));
    }
    __syncwarp();

    // ---- big groups: the whole warp per group
    for (int t0 = 0; t0 < nbig; ++t0) {
        const int r = b.big[t0];
        const unsigned long long t = *trow(b, r);
        const unsigned st = tab_st(t), ln = tab_ln(t), sz = tab_sz(t);
        unsigned int ones = 0u, k1l = 0u, k0l = 0u;   // last entries (+1) with an allele-1 / -0 member
        for (unsigned kc = 0; kc < ln; kc += 32) {
            const unsigned k = kc + lane;
            if (k < ln) {
                const unsigned long long v = *pent(b, st + k);
                const unsigned w = (unsigned)(v >> 32), mk = (unsigned)v;
                const unsigned rr = lds32(row_sa + 4u * w);
                const unsigned c = (unsigned)__popc(mk & rr);
                ones += (NPOP == 2 && w >= wsplit) ? (c << 16) : c;
                if (mk & rr) k1l = k + 1u;
                if (mk & ~rr) k0l = k + 1u;
            }
        }
        ones = __reduce_add_sync(FULLMASK, ones);
        bool k1 = false, k0 = false;
        unsigned int z = 0u;
        unsigned int dd[3] = {0u, 0u, 0u};
        const bool split = decide<NPOP>(ones, sz, dd, k1, k0, z);
        if (lane == 0) { d[0] += dd[0]; d[1] += dd[1]; d[2] += dd[2]; }
        if (!split) continue;
        if (!(k1 && k0)) {
            k1l = __reduce_max_sync(FULLMASK, k1l);
            k0l = __reduce_max_sync(FULLMASK, k0l);
            int dl = 0;
            if (lane == 0) {
                if (k1) dl = drop_one(b, row_sa, r, st, ln, k0l - 1u, false, ones);
                else if (k0) dl = drop_one(b, row_sa, r, st, ln, k1l - 1u, true, z);
                else { *trow(b, r) = mktab(st, 0u, 0u); dl = -(int)ln; }
            }
            L.live += __shfl_sync(FULLMASK, dl, 0);
            if (!k1 && !k0) L.dead += 1;
            __syncwarp();
            continue;
        }
        const unsigned base0 = (unsigned)L.P;
        const int nrow = L.G;
        L.P += (int)ln;
        L.G += 1;
        unsigned w1 = 0, w0 = 0;
        for (unsigned kc = 0; kc < ln; kc += 32) {
            const unsigned k = kc + lane;
            unsigned o1 = 0u, o0 = 0u, w = 0u;
            if (k < ln) {
                const unsigned long long v = *pent(b, st + k);
                w = (unsigned)(v >> 32);
                const unsigned mk = (unsigned)v;
                const unsigned rr = lds32(row_sa + 4u * w);
                o1 = mk & rr;
                o0 = mk & ~rr;
            }
            const unsigned b1 = __ballot_sync(FULLMASK, o1 != 0u);
            const unsigned b0 = __ballot_sync(FULLMASK, o0 != 0u);
            __syncwarp();                        // this chunk is read before it is overwritten
            if (o1) *pent(b, st + w1 + __popc(b1 & ltm)) = mkent(o1, w);
            if (o0) *pent(b, base0 + w0 + __popc(b0 & ltm)) = mkent(o0, w);
            w1 += __popc(b1);
            w0 += __popc(b0);
            __syncwarp();
        }
        if (lane == 0) {
            *trow(b, r) = mktab(st, w1, ones);
            *trow(b, nrow) = mktab(base0, w0, z);
        }
        L.live += (int)(w1 + w0) - (int)ln;
        __syncwarp();
    }
    dS[0] = __reduce_add_sync(FULLMASK, d[0]);
    if (NPOP == 2) {
        dS[1] = __reduce_add_sync(FULLMASK, d[1]);
        dS[2] = __reduce_add_sync(FULLMASK, d[2]);
    }
    if (L.P > b.cap || L.G > b.tcap) {         // cannot happen: see the room check above
        if (lane == 0) atomicExch(b.err, -7);
    }
    __syncwarp();
}

// Walk from `core` in direction dir (0: lower indices, 1: higher).
// NPOP 1: sel 0 = carriers of allele 1, 1 = carriers of allele 0, 2 = all.
// NPOP 2: both populations pooled.  trace (optional): S(i) for i < tcap
// (NPOP 1: the sample's S; NPOP 2: the pooled S).  max_steps > 0 ends a walk
// still running after that many steps with WALK_UNFINISHED.
// win_parity: the warp's two mbarrier phase bits, carried from walk to walk.
template <int NPOP>
__device__ WalkOut walk(const ScanArgs &a, long long core, int dir, int sel, const WarpBufs &b,
                        unsigned long long *trace, long long tcap, int max_steps,
                        unsigned win_parity[2])
{
    const int lane = threadIdx.x & 31;
    WalkOut o;
    o.status = WALK_OK;
    o.stop = 0;
    o.ihh[0] = o.ihh[1] = 0.0;
    o.dig[0] = o.dig[1] = o.dig[2] = 0ull;
    o.D = 0ull;
    o.key = 0.f;
    o.abandon = false;

    // ---- the core row, staged in window buffer 0 (refilled after step 0)
    const unsigned int *row0 = (const unsigned int *)(a.hap + core * a.ld);
    const unsigned ltm = lanemask_lt();
    const int W32 = 2 * a.W;
    unsigned int *core_sm = (unsigned int *)b.wrow[0];
    for (int w = lane; w < W32; w += 32) core_sm[w] = row0[w];
    __syncwarp();
    const unsigned row0_sa = smem_u32(core_sm);

    // ---- initial state: one group (row 0) holding the selected sample
    ListState L;
    L.P = 0; L.live = 0; L.G = 1; L.dead = 0;
    unsigned int cntA = 0, cntB = 0;
    for (int base = 0; base < W32; base += 32) {
        const int w = base + lane;
        unsigned int mk = 0;
        if (w < W32) {
            const unsigned int v = valid32(a, w);
            const unsigned int r = core_sm[w];
            mk = NPOP == 2 ? v : (sel == 0 ? (r & v) : sel == 1 ? (~r & v) : v);
            if (NPOP == 2 && w >= 2 * a.WA) cntB += (unsigned int)__popc(mk);
            else cntA += (unsigned int)__popc(mk);
        }
        const unsigned int bal = __ballot_sync(FULLMASK, mk != 0u);
        if (mk != 0u) *pent(b, (unsigned)(L.P + __popc(bal & ltm))) = mkent(mk, (unsigned)w);
        L.P += __popc(bal);
    }
    cntA = __reduce_add_sync(FULLMASK, cntA);
    cntB = __reduce_add_sync(FULLMASK, cntB);
    L.live = L.P;
    if (lane == 0) *trow(b, 0) = mktab(0u, (unsigned)L.P, cntA | (cntB << 16));
    __syncwarp();

    unsigned long long D0, D1 = 0, DP = 0;
    if (NPOP == 2) {
        D0 = choose2(cntA);
        D1 = choose2(cntB);
        DP = choose2((unsigned long long)cntA + cntB);
    } else {
        D0 = choose2(cntA);
    }
    const unsigned long long Dstop = NPOP == 2 ? DP : D0;
    o.D = Dstop;
    if (Dstop == 0ull) {                   // fewer than two haplotypes: nothing to walk
        o.status = WALK_UNDEFINED;
        return o;
    }
    unsigned long long S0 = D0, S1 = D1, SP = DP;
    unsigned int dS[3] = {0, 0, 0};

    // ---- step 0: the core row itself (whole-sample walks split here, c8)
    split_step<NPOP>(a, row0_sa, b, L, dS);
    S0 -= dS[0];
    if (NPOP == 2) { S1 -= dS[1]; SP -= dS[2]; }
    o.dig[0] = S0;
    if (NPOP == 2) { o.dig[1] = S1; o.dig[2] = SP; }
    if (trace && tcap > 0 && lane == 0) trace[0] = NPOP == 2 ? SP : S0;

    double acc0 = 0.0, acc1 = 0.0;
    unsigned long long p0 = S0, p1 = S1;
    const long long step = dir ? 1 : -1;
    const int R = b.R;
    const unsigned rowbytes = (unsigned)a.ld * 8u;
    WinBuf wb[2];
    wb[0].parity = win_parity[0];
    wb[1].parity = win_parity[1];
    win_issue(a, b, wb[0], 0, core, dir, 1);
    win_issue(a, b, wb[1], 1, core, dir, 1 + R);
    int bi = 1, left = 0;                         // current buffer, steps left in it
    unsigned row_sa = 0u, pos_sa = 0u, gm_sa = 0u; // shared addresses of the current x
    for (long long i = 1;; ++i) {
        const long long x = core + step * i;
        if (x < 0 || x >= a.m) { o.status = WALK_EDGE; o.stop = (int)i; break; }
        if (max_steps > 0 && i > max_steps) {
            o.status = WALK_UNFINISHED;
            o.stop = (int)i;
            o.key = (float)((double)(NPOP == 2 ? SP : S0) / (double)Dstop);
            break;
        }
        if (left == 0) {                          // enter the next buffer
            if (i > 1) {                          // the buffer just used is done: refill it
                if (bi) win_issue(a, b, wb[1], 1, core, dir, i + R);
                else win_issue(a, b, wb[0], 0, core, dir, i + R);
            }
            bi ^= 1;
            left = R;
            if (!(bi ? win_wait(b, wb[1], 1) : win_wait(b, wb[0], 0))) {
                o.status = WALK_UNDEFINED;
                o.stop = (int)i;
                break;
            }
            const WinBuf &w = bi ? wb[1] : wb[0];
            row_sa = smem_u32(b.wrow[bi] + w.roff) + (unsigned)(x - w.lo) * rowbytes;
            pos_sa = smem_u32(b.wpos[bi]) + 8u * (unsigned)(w.poff + (int)(x - w.plo));
            gm_sa = smem_u32(b.wgm[bi]) + 8u * (unsigned)(w.goff + (int)(x - w.plo));
        }
        --left;
        // positions / map of x and of the previous marker (one slot away in the window)
        const unsigned prev_off = dir ? (unsigned)-8 : 8u;
        const long long bp = dir ? lds64(pos_sa) - lds64(pos_sa + prev_off)
                                 : lds64(pos_sa + prev_off) - lds64(pos_sa);
        if (bp > a.max_gap) { o.status = WALK_GAP; o.stop = (int)i; break; }
        double g = a.physical ? (double)bp
                 : (dir ? ldsf64(gm_sa) - ldsf64(gm_sa + prev_off) : ldsf64(gm_sa + prev_off) - ldsf64(gm_sa));
        if (bp > a.gap_scale) g = g * ((double)a.gap_scale / (double)bp);

        split_step<NPOP>(a, row_sa, b, L, dS);
        // advance to the next marker inside the buffer
        if (dir) { row_sa += rowbytes; pos_sa += 8u; gm_sa += 8u; }
        else { row_sa -= rowbytes; pos_sa -= 8u; gm_sa -= 8u; }
        S0 -= dS[0];
        if (NPOP == 2) { S1 -= dS[1]; SP -= dS[2]; }
        const unsigned long long ii = (unsigned long long)(i + 1);
        o.dig[0] += ii * S0;
        if (NPOP == 2) { o.dig[1] += ii * S1; o.dig[2] += ii * SP; }
        if (trace && i < tcap && lane == 0) trace[i] = NPOP == 2 ? SP : S0;

        const bool stop = below_cut(a, NPOP == 2 ? SP : S0, Dstop);
        if (stop && !a.crossing) { o.stop = (int)i; break; }
        // trapezoid (Eq. 4 / Eq. 5): (EHH(i-1) + EHH(i)) / 2 * g, with the
        // common 1 / (2 C(N,2)) applied once at the end.  Lane (i - 1) % 32
        // keeps the term of step i in its partial sum; the partial sums are
        // added by a fixed butterfly when the walk ends.  The sorted-sweep
        // walk sums in the same order, so both give the same bits.
        if (lane == (int)((i - 1) & 31)) {
            acc0 += (double)(p0 + S0) * g;
            if (NPOP == 2) acc1 += (double)(p1 + S1) * g;
        }
        if (stop) { o.stop = (int)i; break; }
        p0 = S0;
        p1 = S1;
    }
    // drain copies still in flight before the buffers serve the next walk
    const bool d0 = win_wait(b, wb[0], 0);
    const bool d1 = win_wait(b, wb[1], 1);
    o.abandon = !d0 || !d1;
    if (o.abandon) o.status = WALK_UNDEFINED;
    win_parity[0] = wb[0].parity;
    win_parity[1] = wb[1].parity;
    acc0 = lane_sum_f64<32>(acc0);
    if (NPOP == 2) acc1 = lane_sum_f64<32>(acc1);
    if (NPOP == 2) {
        o.ihh[0] = D0 ? acc0 / (2.0 * (double)D0) : 0.0;
        o.ihh[1] = D1 ? acc1 / (2.0 * (double)D1) : 0.0;
    } else {
        o.ihh[0] = acc0 / (2.0 * (double)D0);
    }
    return o;
}

}  // namespace selscan
