// EHH walk executed by one warp (device code, sm_103a).
//
// One walk = one core x_0, one direction and one sample (the carriers of a
// core allele for EHH_c, Eq. 3; a whole population for EHH, Eq. 1; or two
// pooled populations for XPEHH, Section 1.3).  The partition of the sample
// into distinct extended haplotypes (Section 1.1) is held as a list of
// "group words": (word index w, 64-bit mask, group id).  A group is the set of
// its words; only words where the group has members are stored, groups of
// fewer than two haplotypes are dropped (they add nothing to any C(n_h, 2)
// and can never grow).  Moving from x_{i-1} to x_i splits every group g by the
// allele row: a = popc(g & row), b = popc(g & ~row) summed over its words, and
// the homozygosity numerator drops by C(a+b,2) - C(a,2) - C(b,2) = a * b.
// S is an exact integer; the stop test den * S < num * C(N,2) is exact.
//
// Per step the warp runs three phases over its lists:
//   A  lanes take group words, count (a, b) per group with one shared/L1
//      atomic each (one warp reduction when all 32 words share a group);
//   M  lanes take groups: S update, survivor flags, new ids by warp scan;
//   B  lanes take group words again and write the surviving halves to the
//      other buffer, compacted with ballots.
// Lists live in the warp's shared-memory slice while they fit and spill to
// the warp's global scratch slice when they do not; both are used through
// generic pointers so one code path serves both.
#pragma once
#include <stdint.h>

#define FULLMASK 0xffffffffu

namespace selscan {

// Internal walk outcomes (the first five equal the public locus codes).
enum : int {
    W_OK = 0, W_UNDEFINED = 2, W_EDGE = 3, W_GAP = 4, W_UNFINISHED = 5
};

struct ScanArgs {
    const unsigned long long *hap;  // rows, row k at hap + k * ld
    long long ld;
    long long m;
    const long long *pos;
    const double *gmap;
    int W;                           // words in use (iHS: W; XPEHH: W_A + W_B)
    int WA;                          // words of population A (iHS: = W)
    int nA, nB;                      // population sizes (iHS: n, 0)
    unsigned long long lastA;        // valid bits of word WA - 1
    unsigned long long lastB;        // valid bits of word W - 1 (XPEHH)
    unsigned int cut_num, cut_den;
    long long gap_scale, max_gap;
    int crossing;
};

struct WarpBufs {
    unsigned long long *mask[4];     // [0], [1] on chip; [2], [3] global
    unsigned int *meta[4];           // w | group << 16
    unsigned int *cnt[2];            // counts (a | b << 16) per group: [on chip, global]
    unsigned int *cntB[2];           // population B counts (pooled walks)
    unsigned int *nid[2];            // new ids: id1 | id0 << 16
    int cap_s, gcap_s;               // on-chip capacities (entries, groups)
};

struct WalkOut {
    int status;
    int stop;
    double ihh[2];
    unsigned long long dig[3];
    float key;                       // EHH at the step cap (unfinished walks)
};

__device__ __forceinline__ unsigned long long valid_word(const ScanArgs &a, int w)
{
    if (w == a.WA - 1) return a.lastA;
    if (w == a.W - 1) return a.lastB;
    return ~0ull;
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

// Split every group of the current list by `row`.  On return the other
// buffer holds the new list; E, G, cur are updated; dS[] receives the drops
// of the homozygosity numerators (NPOP 1: [0]; NPOP 2: A, B, pooled).
template <int NPOP>
__device__ __forceinline__ void split_step(const ScanArgs &a, const unsigned long long *row,
                                           WarpBufs &b, int &cur, int &E, int &G,
                                           unsigned int dS[3])
{
    const int lane = threadIdx.x & 31;
    const int gl = G <= b.gcap_s ? 0 : 1;
    unsigned int *cnt = b.cnt[gl];
    unsigned int *cntB = b.cntB[gl];
    unsigned int *nid = b.nid[gl];
    const unsigned long long *cm = b.mask[cur];
    const unsigned int *ct = b.meta[cur];

    // ---- phase A: per-group allele counts
    for (int base = 0; base < E; base += 32) {
        const int e = base + lane;
        unsigned int g = 0, val = 0;
        int pop = 0;
        if (e < E) {
            const unsigned int mt = ct[e];
            const int w = (int)(mt & 0xffffu);
            g = mt >> 16;
            const unsigned long long mk = cm[e];
            const unsigned long long r = __ldg(row + w);
            val = (unsigned int)__popcll(mk & r) | ((unsigned int)__popcll(mk & ~r) << 16);
            if (NPOP == 2) pop = w >= a.WA;
        }
        const unsigned int key = (g << 1) | (unsigned int)pop;
        const unsigned int key0 = __shfl_sync(FULLMASK, key, 0);
        if (__all_sync(FULLMASK, e >= E || key == key0)) {
            const unsigned int tot = __reduce_add_sync(FULLMASK, val);
            if (lane == 0) {
                unsigned int *dst = (NPOP == 2 && (key0 & 1u)) ? cntB : cnt;
                atomicAdd(dst + (key0 >> 1), tot);
            }
        } else if (e < E) {
            unsigned int *dst = (NPOP == 2 && pop) ? cntB : cnt;
            atomicAdd(dst + g, val);
        }
    }
    __syncwarp();

    // ---- phase M: S update, survivors, new ids; consumed counts reset to 0
    unsigned int s0 = 0, s1 = 0, s2 = 0;
    int Gn = 0;
    for (int base = 0; base < G; base += 32) {
        const int g = base + lane;
        unsigned int k1 = 0, k0 = 0;
        if (g < G) {
            // read-and-reset at L2 / shared memory (never a stale L1 line)
            const unsigned int v = atomicExch(cnt + g, 0u);
            unsigned int x1 = v & 0xffffu, x0 = v >> 16;
            if (NPOP == 2) {
                const unsigned int vb = atomicExch(cntB + g, 0u);
                const unsigned int y1 = vb & 0xffffu, y0 = vb >> 16;
                s0 += x1 * x0;                       // population A
                s1 += y1 * y0;                       // population B
                x1 += y1;
                x0 += y0;
                s2 += x1 * x0;                       // pooled
            } else {
                s0 += x1 * x0;
            }
            k1 = x1 >= 2u;
            k0 = x0 >= 2u;
        }
        unsigned int k = k1 + k0, inc = k;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(FULLMASK, inc, o);
            if (lane >= o) inc += t;
        }
        const unsigned int ex = (unsigned int)Gn + inc - k;
        if (g < G) {
            const unsigned int id1 = k1 ? ex : 0xffffu;
            const unsigned int id0 = k0 ? ex + k1 : 0xffffu;
            nid[g] = id1 | (id0 << 16);
        }
        Gn += (int)__shfl_sync(FULLMASK, inc, 31);
    }
    dS[0] = __reduce_add_sync(FULLMASK, s0);
    if (NPOP == 2) {
        dS[1] = __reduce_add_sync(FULLMASK, s1);
        dS[2] = __reduce_add_sync(FULLMASK, s2);
    }
    __syncwarp();

    // ---- phase B: write the surviving halves to the other buffer
    int nxt;
    if (2 * E <= b.cap_s) nxt = cur == 0 ? 1 : 0;        // stays (or moves) on chip
    else nxt = cur == 2 ? 3 : 2;                          // global scratch
    unsigned long long *nm = b.mask[nxt];
    unsigned int *nt = b.meta[nxt];
    int out = 0;
    const unsigned int ltm = lanemask_lt();
    for (int base = 0; base < E; base += 32) {
        const int e = base + lane;
        bool e1 = false, e0 = false;
        unsigned long long m1 = 0, m0 = 0;
        unsigned int w = 0, ids = 0;
        if (e < E) {
            const unsigned int mt = ct[e];
            w = mt & 0xffffu;
            const unsigned long long mk = cm[e];
            const unsigned long long r = __ldg(row + w);
            m1 = mk & r;
            m0 = mk & ~r;
            ids = nid[mt >> 16];
            e1 = m1 != 0ull && (ids & 0xffffu) != 0xffffu;
            e0 = m0 != 0ull && (ids >> 16) != 0xffffu;
        }
        const unsigned int b1 = __ballot_sync(FULLMASK, e1);
        const unsigned int b0 = __ballot_sync(FULLMASK, e0);
        const int p = out + __popc(b1 & ltm) + __popc(b0 & ltm);
        if (e1) { nm[p] = m1; nt[p] = w | ((ids & 0xffffu) << 16); }
        if (e0) { nm[p + (int)e1] = m0; nt[p + (int)e1] = w | (ids & 0xffff0000u); }
        out += __popc(b1) + __popc(b0);
    }
    __syncwarp();
    cur = nxt;
    E = out;
    G = Gn;
}

// Walk from `core` in direction dir (0: lower indices, 1: higher).
// NPOP 1: sel 0 = carriers of allele 1, 1 = carriers of allele 0, 2 = all.
// NPOP 2: both populations pooled.  trace (optional): S(i) for i < tcap
// (NPOP 1: the sample's S; NPOP 2: the pooled S).  max_steps > 0 ends a walk
// still running after that many steps with W_UNFINISHED.
template <int NPOP>
__device__ WalkOut walk(const ScanArgs &a, long long core, int dir, int sel, WarpBufs &b,
                        unsigned long long *trace, long long tcap, int max_steps)
{
    const int lane = threadIdx.x & 31;
    WalkOut o;
    o.status = W_OK;
    o.stop = 0;
    o.ihh[0] = o.ihh[1] = 0.0;
    o.dig[0] = o.dig[1] = o.dig[2] = 0ull;
    o.key = 0.f;

    // ---- initial list: one group holding the selected sample
    const unsigned long long *row0 = a.hap + core * a.ld;
    int cur = a.W <= b.cap_s ? 0 : 2;
    unsigned long long *im = b.mask[cur];
    unsigned int *it = b.meta[cur];
    int E = 0;
    unsigned int cntA = 0, cntB = 0;
    const unsigned int ltm = lanemask_lt();
    for (int base = 0; base < a.W; base += 32) {
        const int w = base + lane;
        unsigned long long mk = 0;
        if (w < a.W) {
            const unsigned long long v = valid_word(a, w);
            const unsigned long long r = __ldg(row0 + w);
            mk = NPOP == 2 ? v : (sel == 0 ? (r & v) : sel == 1 ? (~r & v) : v);
            if (NPOP == 2 && w >= a.WA) cntB += (unsigned int)__popcll(mk);
            else cntA += (unsigned int)__popcll(mk);
        }
        const unsigned int bal = __ballot_sync(FULLMASK, mk != 0ull);
        if (mk != 0ull) {
            const int p = E + __popc(bal & ltm);
            im[p] = mk;
            it[p] = (unsigned int)w;           // group 0
        }
        E += __popc(bal);
    }
    cntA = __reduce_add_sync(FULLMASK, cntA);
    cntB = __reduce_add_sync(FULLMASK, cntB);
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
    if (Dstop == 0ull) {                   // fewer than two haplotypes: nothing to walk
        o.status = W_UNDEFINED;
        return o;
    }
    if (E == 0) { /* unreachable with Dstop > 0 */ }
    int G = 1;
    unsigned long long S0 = D0, S1 = D1, SP = DP;
    unsigned int dS[3] = {0, 0, 0};

    // ---- step 0: the core row itself (whole-sample walks split here, c8)
    split_step<NPOP>(a, row0, b, cur, E, G, dS);
    S0 -= dS[0];
    if (NPOP == 2) { S1 -= dS[1]; SP -= dS[2]; }
    o.dig[0] = S0;
    if (NPOP == 2) { o.dig[1] = S1; o.dig[2] = SP; }
    if (trace && tcap > 0 && lane == 0) trace[0] = NPOP == 2 ? SP : S0;

    double acc0 = 0.0, acc1 = 0.0;
    unsigned long long p0 = S0, p1 = S1;
    const long long step = dir ? 1 : -1;
    for (long long i = 1;; ++i) {
        const long long x = core + step * i;
        if (x < 0 || x >= a.m) { o.status = W_EDGE; o.stop = (int)i; break; }
        if (max_steps > 0 && i > max_steps) {
            o.status = W_UNFINISHED;
            o.stop = (int)i;
            o.key = (float)((double)(NPOP == 2 ? SP : S0) / (double)Dstop);
            break;
        }
        const long long xp = x - step;
        const long long lo = dir ? xp : x, hi = dir ? x : xp;
        const long long bp = __ldg(a.pos + hi) - __ldg(a.pos + lo);
        if (bp > a.max_gap) { o.status = W_GAP; o.stop = (int)i; break; }
        double g = __ldg(a.gmap + hi) - __ldg(a.gmap + lo);
        if (bp > a.gap_scale) g = g * ((double)a.gap_scale / (double)bp);

        split_step<NPOP>(a, a.hap + x * a.ld, b, cur, E, G, dS);
        S0 -= dS[0];
        if (NPOP == 2) { S1 -= dS[1]; SP -= dS[2]; }
        const unsigned long long ii = (unsigned long long)(i + 1);
        o.dig[0] += ii * S0;
        if (NPOP == 2) { o.dig[1] += ii * S1; o.dig[2] += ii * SP; }
        if (trace && i < tcap && lane == 0) trace[i] = NPOP == 2 ? SP : S0;

        const bool stop = below_cut(a, NPOP == 2 ? SP : S0, Dstop);
        if (stop && !a.crossing) { o.stop = (int)i; break; }
        // trapezoid (Eq. 4 / Eq. 5): (EHH(i-1) + EHH(i)) / 2 * g, with the
        // common 1 / (2 C(N,2)) applied once at the end
        acc0 += (double)(p0 + S0) * g;
        if (NPOP == 2) acc1 += (double)(p1 + S1) * g;
        if (stop) { o.stop = (int)i; break; }
        p0 = S0;
        p1 = S1;
    }
    if (NPOP == 2) {
        o.ihh[0] = D0 ? acc0 / (2.0 * (double)D0) : 0.0;
        o.ihh[1] = D1 ? acc1 / (2.0 * (double)D1) : 0.0;
    } else {
        o.ihh[0] = acc0 / (2.0 * (double)D0);
    }
    return o;
}

}  // namespace selscan
