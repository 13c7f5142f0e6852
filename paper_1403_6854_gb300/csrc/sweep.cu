// Sorted-sweep form of the EHH walks (iHS Eq. 3-5, XPEHH Eq. 6-7).
//
// Every statistic of a walk is a function of S(i), the number of pairs of the
// walk's sample that are identical over the markers between the core and
// x_i (Section 1.2: EHH(x_i) = S(i) / C(N, 2)).  If the haplotypes are kept
// sorted by their sequence read outward from the core (the prefix order of a
// positional Burrows-Wheeler sweep), the haplotypes identical over
// [core, x_i] are contiguous runs of that order, and two neighbours t-1, t
// part at the first marker where they differ, i.e. at walk step M[t] = the
// length of their common run ending at the core.  So S(0) = C(n_c, 2) per
// core class, and step i only has to apply the boundaries t with M[t] = i:
// splitting a run [l, r) at t lowers S by (t - l)(r - t).  The cost of a walk
// becomes the number of boundaries it crosses, not the number of groups it
// carries at every step.
//
// Two kernels per stage:
//  * sweep_kernel: one CTA per chunk of cores and direction keeps the order A
//    and the run lengths M of all haplotypes in shared memory and advances them
//    marker by marker (a stable partition by allele; the new run length of a
//    neighbour pair is 1 + the minimum over the old pairs it spans).  At every
//    core of the stage it writes M, the class boundary n0 (and, for XPEHH, the
//    population of each sorted position) to a slot, with the boundaries of
//    the first walk steps already grouped by step.  A chunk starts `warmup`
//    markers before its first core, so its sort is exact for walks that stay
//    within that history.
//  * split_walk_kernel: one warp per slot runs the walk steps of that core
//    (both allele classes of iHS, or the pooled XPEHH walk): gaps, the map,
//    the cutoff and the trapezoid exactly as the per-step walk does, with S(i)
//    from the boundaries of step i (from the slot's first window, then from
//    64-step windows it finds in M).  A walk that would step beyond its
//    chunk's history is handed to the per-step walk kernel (second pass).
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>
#include <limits.h>

#include "../../include/selscan.h"
#include "device_common.cuh"
#include "internal.h"

namespace selscan {

namespace {

constexpr unsigned kInf16 = 0xFFFFu;
constexpr int kRowRing = 4;                 // rows in flight ahead of the sort (cp.async)
constexpr int kSlotListCap = 1024;          // first-window boundaries kept per slot
constexpr int kSplitListSmem = 1024;        // window list entries a walking warp keeps on chip
constexpr int kWin = 64;                    // steps of a window the walker groups itself (a power of 2)

__host__ __device__ inline int sweep_e(int n, int T)
{
    int e = (n + T - 1) / T;
    return (e + 3) & ~3;                    // a multiple of 4: elements are read 4 at a time
}
__host__ __device__ inline int sweep_npad(int n, int T) { return sweep_e(n, T) * T; }
__host__ __device__ inline int split_nw(int n) { return (n + 32) >> 5; }   // bits 0..n

// ---- prefix-state algebra of the stable partition --------------------------
// A segment of the current order summarised as: the running minimum of the
// run lengths since its last allele-0 / allele-1 element (or over the whole
// segment if it has none) -- the "tails" -- the minimum over the segment, the
// number of allele-0 elements, and whether each allele occurs.  Three words:
// A = tail0 | tail1 << 16; B = the minimum in both halves; C = zeros |
// seen0 << 15 | seen1 << 31 (zeros < 2^14; the flags sit on byte sign bits,
// so one byte permute in sign-replicate mode turns them into the halfword
// mask of the tails that R decides).  compose(L, R) replaces R by the summary
// of L followed by R: both tails are continued through R with one 16-bit
// SIMD minimum.
__device__ __forceinline__ unsigned seen_mask(unsigned c)
{
    unsigned r;   // bytes 0, 1 <- sign of byte 1 (seen0); bytes 2, 3 <- sign of byte 3 (seen1)
    asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(r) : "r"(c));
    return r;
}
__device__ __forceinline__ void compose(unsigned lA, unsigned lB, unsigned lC, unsigned &rA,
                                        unsigned &rB, unsigned &rC)
{
    const unsigned cont = __vminu2(lA, rB);                        // L's tails continued through R
    const unsigned keep = seen_mask(rC);                           // the tails R decides
    rA = (rA & keep) | (cont & ~keep);
    rB = __vminu2(lB, rB);
    rC = ((lC + rC) & 0x3FFFu) | ((lC | rC) & 0x80008000u);
}
constexpr unsigned kIdA = 0xFFFFFFFFu;
constexpr unsigned kIdB = 0xFFFFFFFFu;
constexpr unsigned kIdC = 0u;

// Asynchronous global -> shared copies of 8 bytes (rows start on 8-byte
// boundaries whatever their stride), in per-thread commit groups.
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ unsigned bit_index(const SweepArgs &w, int h)
{
    // position of haplotype h (pooled numbering, A first) in the row's bits
    return h < w.a.nA ? (unsigned)h : (unsigned)(64 * w.a.WA + (h - w.a.nA));
}

}  // namespace

// Slot of one core: header {n0, history horizon, W1, 0}, the run lengths M
// (u16 per sorted position), for XPEHH the population-A flags of the sorted
// positions, then the first window: W1 + 1 step offsets (u16) and its
// boundaries ordered by step (u16 positions).  The window is the longest run
// of steps 1..W1 (W1 <= 64) whose boundaries fit slot_list_cap(n) entries.
namespace {
__host__ __device__ inline int slot_list_cap(int n) { return n < kSlotListCap ? n : kSlotListCap; }
__host__ __device__ inline size_t slot_isa_at(int n) { return 16 + (((size_t)n * 2 + 15) & ~(size_t)15); }
__host__ __device__ inline size_t slot_off_at(int n, int xpehh)
{
    return slot_isa_at(n) + (xpehh ? (((size_t)split_nw(n) * 4 + 15) & ~(size_t)15) : 0);
}
__host__ __device__ inline size_t slot_list_at(int n, int xpehh) { return slot_off_at(n, xpehh) + 144; }
}  // namespace

size_t sweep_smem_bytes(int n, int W, int T, int R)
{
    const int W32 = ((2 * W) + 4) & ~3;
    return (size_t)sweep_npad(n, T) * 4 * 2 + (size_t)W32 * 4 * kRowRing + T / 32 * 12 + 2 * 65 * 4 +
           (size_t)((R + 31) / 32) * 4;
}

size_t sweep_slot_bytes(int n, int xpehh)
{
    // a multiple of 16 bytes: every slot's M region is read and written in 16-byte units
    return slot_list_at(n, xpehh) + (((size_t)slot_list_cap(n) * 2 + 15) & ~(size_t)15);
}

size_t sweep_state_bytes(int n, int T) { return (size_t)sweep_npad(n, T) * 4; }
size_t sweep_elements(int n, int T) { return (size_t)sweep_npad(n, T); }


// ---- the sweep ---------------------------------------------------------------
// Shared memory: two buffers of np packed elements (bit index of the haplotype
// in the row | run length with its predecessor << 16), a ring of kRowRing row
// buffers (filled by cp.async, each with one extra all-ones word), the warp
// totals, a core's first-window counts and offsets, and the stage's core
// bitmap.  Positions n..np-1 hold padding elements whose allele is that
// all-ones word: they sort after every real haplotype and never touch a real
// element's run length.  T threads (32 to 512); EMAX bounds the elements per
// thread (at most 32, one allele bit each in a 32-bit mask), up to 24 stay in
// registers between the two passes.
template <int T, int EMAX, bool EXACT = false>
__global__ void __launch_bounds__(T, T == 512 ? 2 : (T == 256 ? 3 : 512 / T)) sweep_kernel(SweepArgs w)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool CACHE = EMAX <= 24;
    const int n = w.n;
    // EXACT: every thread holds exactly EMAX elements (no per-element guards)
    const int E = EXACT ? EMAX : sweep_e(n, T);
    const int np = E * T;
    const int W32 = 2 * w.a.W;
    const int W32r = (W32 + 4) & ~3;             // >= W32 + 1
    const unsigned pad_bi = 32u * (unsigned)W32; // bit index of the padding elements
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = T / 32;
    unsigned *P0 = (unsigned *)smem;             // buffer b at P0 + b * np
    unsigned *R0 = P0 + 2 * np;                  // row ring: slot r at R0 + r * W32r
    unsigned *wsum = R0 + kRowRing * W32r;
    unsigned *hcnt = wsum + 3 * NW;              // a core's first window: per-step counts,
    unsigned *hoff = hcnt + 65;                  // then cursors and (at [64]) W1
    unsigned *cbits = hoff + 65;                 // the stage's cores that pass the filter

    const int dir = blockIdx.x / w.nch;          // 0: walks toward lower indices
    const int c = blockIdx.x % w.nch;
    const long long m = w.a.m;
    const long long c0 = w.a.k0 + (long long)c * w.B;   // chunk c covers cores [c0, c1) of [k0, k1)
    if (c0 >= w.a.k1) return;
    const long long c1 = c0 + w.B < w.a.k1 ? c0 + w.B : w.a.k1;
    long long klo, khi;                          // this stage's cores [klo, khi)
    if (dir == 0) {
        klo = c0 + (long long)w.stage * w.R;
        khi = klo + w.R < c1 ? klo + w.R : c1;
        if (klo >= c1) return;
    } else {
        khi = c1 - (long long)w.stage * w.R;
        klo = khi - w.R > c0 ? khi - w.R : c0;
        if (khi <= c0) return;
    }
    // history origin of the chunk: the sort is exact for runs inside it
    const long long s0 = c0 - w.L > 0 ? c0 - w.L : 0;
    const long long e0 = c1 - 1 + w.L < m - 1 ? c1 - 1 + w.L : m - 1;
    long long xfirst, xlast;                     // markers of this launch, in sweep order
    if (dir == 0) {
        xfirst = w.stage == 0 ? s0 : klo;
        xlast = khi - 1;
    } else {
        xfirst = w.stage == 0 ? e0 : khi - 1;
        xlast = klo;
    }
    const long long step = dir == 0 ? 1 : -1;
    unsigned *st = (unsigned *)w.st + (size_t)blockIdx.x * np;

    if (blockIdx.x == 0 && tid == 0) *w.walk_head = 0ull;   // the next walk launch's slot counter
    // ---- state in
    if (w.stage == 0) {
        for (int t = tid; t < np; t += T) P0[t] = t < n ? bit_index(w, t) : pad_bi;
    } else {
        for (int t = tid; t < np; t += T) P0[t] = st[t];
    }
    const unsigned long long *hap64 = (const unsigned long long *)w.a.hap;
    const long long ld = w.a.ld;
    const int W = w.a.W;
    const long long nq = (xlast - xfirst) * step + 1;   // markers of this launch
    // row q (in sweep order) goes to ring slot q % kRowRing, kRowRing - 1 rows ahead
    auto fetch_row = [&](long long q) {
        if (q < nq) {
            unsigned *dst = R0 + (q & (kRowRing - 1)) * W32r;
            const unsigned long long *src = hap64 + (xfirst + q * step) * ld;
            for (int t = tid; t < W; t += T) cp_async8(dst + 2 * t, src + t);
        }
        cp_async_commit();
    };
    for (int q = 0; q < kRowRing; ++q) fetch_row(q);
    for (int t = tid; t < 64; t += T) hcnt[t] = 0u;
    for (int r = 0; r < kRowRing; ++r)          // the padding elements' all-ones word
        if (tid < W32r - W32) R0[r * W32r + W32 + tid] = 0xFFFFFFFFu;
    {
        const int nrc = (int)(khi - klo);
        for (int r0 = 0; r0 < nrc; r0 += T) {
            const int r = r0 + tid;
            const bool v = r < nrc && w.sk.core_status[klo + r] != (int8_t)SELSCAN_LOCUS_MAF_FILTERED;
            const unsigned bits = __ballot_sync(FULLMASK, v);
            if (lane == 0 && r0 + warp * 32 < nrc) cbits[(r0 >> 5) + warp] = bits;
        }
    }
    cp_async_wait<kRowRing - 1>();               // row 0
    __syncthreads();

    int cur = 0;
    const int base = tid * E;
    unsigned val[CACHE ? EMAX : 1];
    long long q = 0;
    for (long long x = xfirst;; x += step, ++q) {
        const bool more = x != xlast;
        const bool is_core = x >= klo && x < khi;
        const bool wr = is_core && ((cbits[(x - klo) >> 5] >> ((x - klo) & 31)) & 1u);

        const unsigned *Pc = P0 + cur * np;
        const unsigned *row = R0 + (q & (kRowRing - 1)) * W32r;
        // pass 1: alleles, the new run lengths as far as this segment decides
        // them, and the segment summary.  Both tails live in one word (allele
        // 0 low, 1 high).  Run lengths stay at most 65,000 (a chunk plus its
        // warm-up spans at most 65,000 markers), so adding one to each half
        // never carries.  The first element of each allele in the segment gets
        // its prefix tail after placement.
        unsigned vmask = 0u, allw = 0xFFFFFFFFu, mn01 = 0xFFFFFFFFu;
#pragma unroll
        for (int e = 0; e < EMAX; e += 4) {
            if (e < E) {
                // 16-byte loads: a thread's segment starts at 16 E bytes, and
                // eight lanes at that stride cover distinct banks
                const uint4 q = *(const uint4 *)(Pc + base + e);
                const unsigned q4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const unsigned pv = q4[h];
                    // the word of bit index pv & 0xFFFF, (pv & 0xFFFF) >> 5, by multiplies
                    const unsigned wd = row[__umulhi(pv * 65536u, 2048u)];
                    const unsigned v = __funnelshift_r(wd, wd, pv) & 1u;   // bit pv % 32
                    vmask = vmask + vmask + v;            // element e at bit E - 1 - e
                    allw = min(allw, pv);                 // high half: the segment minimum
                    mn01 = __vminu2(mn01, __byte_perm(pv, 0u, 0x3232u));
                    // the selector by multiply-add (v ? 0x7610 : 0x5410), and the tail
                    // of allele v restarted by a 16x2 maximum with 0xFFFF in its half
                    if (CACHE) val[e + h] = __byte_perm(pv, mn01 + 0x00010001u, 0x5410u + v * 0x2200u);
                    mn01 = __vmaxu2(mn01, 0x0000FFFFu + v * 0xFFFE0001u);
                }
            }
        }
        const unsigned ones = (unsigned)__popc(vmask);
        vmask <<= 32 - E;                         // element e at bit 31 - e
        const unsigned zeros = (unsigned)E - ones;
        const unsigned hp0 = zeros != 0u, hp1 = ones != 0u;
        unsigned p0 = mn01;
        unsigned p1 = (allw >> 16) * 0x00010001u;
        unsigned p2 = zeros | (hp0 << 15) | (hp1 << 31);
        // warp inclusive scan
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o0 = __shfl_up_sync(FULLMASK, p0, d);
            const unsigned o1 = __shfl_up_sync(FULLMASK, p1, d);
            const unsigned o2 = __shfl_up_sync(FULLMASK, p2, d);
            if (lane >= d) compose(o0, o1, o2, p0, p1, p2);
        }
        unsigned x0 = __shfl_up_sync(FULLMASK, p0, 1), x1 = __shfl_up_sync(FULLMASK, p1, 1);
        unsigned x2 = __shfl_up_sync(FULLMASK, p2, 1);
        if (lane == 0) { x0 = kIdA; x1 = kIdB; x2 = kIdC; }
        if (lane == 31) { wsum[3 * warp] = p0; wsum[3 * warp + 1] = p1; wsum[3 * warp + 2] = p2; }
        __syncthreads();
        fetch_row(q + kRowRing);                  // every thread is done with this row's slot
        // every warp scans the warp totals: its own prefix and the block total
        unsigned q0 = lane < NW ? wsum[3 * lane] : kIdA;
        unsigned q1 = lane < NW ? wsum[3 * lane + 1] : kIdB;
        unsigned q2 = lane < NW ? wsum[3 * lane + 2] : kIdC;
#pragma unroll
        for (int d = 1; d < NW; d <<= 1) {
            const unsigned o0 = __shfl_up_sync(FULLMASK, q0, d);
            const unsigned o1 = __shfl_up_sync(FULLMASK, q1, d);
            const unsigned o2 = __shfl_up_sync(FULLMASK, q2, d);
            if (lane >= d) compose(o0, o1, o2, q0, q1, q2);
        }
        unsigned w0 = __shfl_sync(FULLMASK, q0, (warp + 31) & 31);
        unsigned w1 = __shfl_sync(FULLMASK, q1, (warp + 31) & 31);
        unsigned w2 = __shfl_sync(FULLMASK, q2, (warp + 31) & 31);
        if (warp == 0) { w0 = kIdA; w1 = kIdB; w2 = kIdC; }
        const unsigned tot2 = __shfl_sync(FULLMASK, q2, NW - 1);
        const unsigned n0 = tot2 & 0x3FFFu;
        compose(w0, w1, w2, x0, x1, x2);          // this thread's exclusive prefix
        // pass 2: place the elements; the first allele-0 / allele-1 element of
        // the segment takes its run length from the prefix (0 if it is the
        // first of its allele overall)
        const unsigned zs = x2 & 0x3FFFu;
        const unsigned os = n0 + (unsigned)base - zs;
        unsigned z = zs, o = os;
        unsigned *Pn = P0 + (cur ^ 1) * np;
        if (CACHE) {
            // allele-0 elements go to zs + (elements so far) - (ones so far)
            const unsigned zk = zs + os;
#pragma unroll
            for (int e = 0; e < EMAX; ++e) {
                if (e < E) {
                    const unsigned one = (vmask >> (31 - e)) & 1u;
                    Pn[one ? o : zk + (unsigned)e - o] = val[CACHE ? e : 0];
                    o += one;
                }
            }
        }
        if (!CACHE) {
            // second sweep over the segment for the run lengths (large samples)
            unsigned a0 = x0 & 0xFFFFu, a1 = x0 >> 16;
            unsigned h0 = (x2 >> 15) & 1u, h1 = x2 >> 31;
            z = zs;
            o = os;
            for (int e = 0; e < E; ++e) {
                const unsigned q = Pc[base + e];
                const unsigned mv = q >> 16;
                a0 = min(a0, mv);
                a1 = min(a1, mv);
                const unsigned one = (vmask >> (31 - e)) & 1u;
                const unsigned mnv = one ? a1 : a0;
                const unsigned hpv = one ? h1 : h0;
                const unsigned out = hpv ? min(mnv + 1u, kInf16) : 0u;
                const unsigned p = one ? o : z;
                o += one;
                z += one ^ 1u;
                a1 = one ? kInf16 : a1;
                a0 = one ? a0 : kInf16;
                h1 |= one;
                h0 |= one ^ 1u;
                Pn[p] = (q & 0xFFFFu) | (out << 16);
            }
        } else {
            // the first allele-0 / allele-1 element of the segment (placed at zs
            // / os): 1 + the minimum over the prefix tail and its own span
            if (hp0) {
                const unsigned u = Pn[zs];
                const unsigned out = ((x2 >> 15) & 1u) ? min((x0 & 0xFFFFu) + 1u, u >> 16) : 0u;
                Pn[zs] = (u & 0xFFFFu) | (out << 16);
            }
            if (hp1) {
                const unsigned u = Pn[os];
                const unsigned out = (x2 >> 31) ? min((x0 >> 16) + 1u, u >> 16) : 0u;
                Pn[os] = (u & 0xFFFFu) | (out << 16);
            }
        }
        cp_async_wait<kRowRing - 1>();           // row q + 1 has landed
        __syncthreads();
        cur ^= 1;

        // ---- a core of this stage: hand its sorted state to the walk
        if (wr) {
            const int r = dir == 0 ? (int)(x - klo) : (int)(khi - 1 - x);
            unsigned char *slot = w.slots + ((size_t)(dir * w.nch + c) * w.R + r) * w.slot_bytes;
            const int xp = w.a.nB > 0;
            if (tid == 0) {
                int *hdr = (int *)slot;
                hdr[0] = (int)n0;
                long long hz;
                if (dir == 0) hz = s0 == 0 ? INT_MAX : x - s0;
                else hz = e0 == m - 1 ? INT_MAX : e0 - x;
                hdr[1] = (int)hz;
            }
            const unsigned *Ps = P0 + cur * np;
            // run lengths, 4 per 8-byte store (four elements per item: finer
            // items even out the threads' shares; the slot's M region is a
            // multiple of 16 bytes, values past n are never read), counting the
            // boundaries of each of steps 1..64 (M in [1, 64])
            const uint4 *P4 = (const uint4 *)Ps;
            uint2 *M2 = (uint2 *)(slot + 16);
            for (int t = tid; t < (n + 3) / 4; t += T) {
                const uint4 a = P4[t];
                M2[t] = make_uint2(__byte_perm(a.x, a.y, 0x7632u), __byte_perm(a.z, a.w, 0x7632u));
                const unsigned e4[4] = {a.x, a.y, a.z, a.w};
                if (4 * t + 4 <= n) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (e4[j] - 0x10000u < 0x400000u) atomicAdd(hcnt + (e4[j] >> 16) - 1, 1u);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (e4[j] - 0x10000u < 0x400000u && 4 * t + j < n) atomicAdd(hcnt + (e4[j] >> 16) - 1, 1u);
                }
            }
            if (xp) {                            // population of each sorted position
                // one 32-position word per warp iteration: a ballot over the lanes
                const unsigned limA = 64u * (unsigned)w.a.WA;
                unsigned *isA = (unsigned *)(slot + slot_isa_at(n));
                const int nw = split_nw(n);
                for (int q = warp; q < nw; q += NW) {
                    const int t = q * 32 + lane;
                    const unsigned word = __ballot_sync(FULLMASK, t < n && (Ps[t] & 0xFFFFu) < limA);
                    if (lane == 0) isA[q] = word;
                }
            }
            __syncthreads();
            // the first window: the longest run of steps from step 1 on whose
            // boundaries fit the slot's list
            unsigned short *soff = (unsigned short *)(slot + slot_off_at(n, xp));
            if (warp == 0) {
                const unsigned c0 = hcnt[2 * lane], c1 = hcnt[2 * lane + 1];
                unsigned incl = c0 + c1;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const unsigned v = __shfl_up_sync(FULLMASK, incl, d);
                    if (lane >= d) incl += v;
                }
                const unsigned ex = incl - c0 - c1;
                const unsigned cap = (unsigned)slot_list_cap(n);
                // steps 2 lane + 1 and 2 lane + 2 end at offsets ex + c0 and incl
                const unsigned w1 = __popc(__ballot_sync(FULLMASK, ex + c0 <= cap)) +
                                    __popc(__ballot_sync(FULLMASK, incl <= cap));
                soff[2 * lane] = (unsigned short)min(ex, 0xFFFFu);
                soff[2 * lane + 1] = (unsigned short)min(ex + c0, 0xFFFFu);
                if (lane == 31) soff[64] = (unsigned short)min(incl, 0xFFFFu);
                hoff[2 * lane] = ex;
                hoff[2 * lane + 1] = ex + c0;
                hcnt[2 * lane] = 0u;
                hcnt[2 * lane + 1] = 0u;
                if (lane == 0) {
                    hoff[64] = w1;
                    ((int *)slot)[2] = (int)w1;
                    ((int *)slot)[3] = 0;
                }
            }
            __syncthreads();
            // place the window's boundaries by step
            const unsigned lim = hoff[64] << 16;
            unsigned short *slist = (unsigned short *)(slot + slot_list_at(n, xp));
            for (int t = tid; t < (n + 3) / 4; t += T) {
                const uint4 a = P4[t];
                const unsigned e4[4] = {a.x, a.y, a.z, a.w};
                if (4 * t + 4 <= n) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (e4[j] - 0x10000u < lim)
                            slist[atomicAdd(hoff + (e4[j] >> 16) - 1, 1u)] = (unsigned short)(4 * t + j);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (e4[j] - 0x10000u < lim && 4 * t + j < n)
                            slist[atomicAdd(hoff + (e4[j] >> 16) - 1, 1u)] = (unsigned short)(4 * t + j);
                }
            }
        }
        if (!more) break;
    }
    // ---- state out for the next stage
    if (w.stage + 1 < w.nstages) {
        const unsigned *Ps = P0 + cur * np;
        for (int t = tid; t < np; t += T) st[t] = Ps[t];
    }
}

// ---- the split walk ----------------------------------------------------------
namespace {

// Per-warp shared memory: run starts before this step (O) and all run starts
// including this step's (A) as bitmaps over positions 0..n, one summary bit
// per non-zero word (SO, SA), step counts / offsets of the current window, and
// for XPEHH the population-A flags of the sorted positions with their
// per-word prefix counts.
struct SplitSmem {
    unsigned *O, *A, *SO, *SA;
    unsigned *cnt, *off;
    unsigned short *lst;                  // the current window's list, when it fits
    unsigned *isA, *PA;
    int nw, ns;
};

__device__ inline SplitSmem split_smem(unsigned char *base, int n, int xpehh)
{
    SplitSmem s;
    s.nw = split_nw(n);
    s.ns = (s.nw + 31) >> 5;
    unsigned *p = (unsigned *)base;
    s.O = p; p += s.nw;
    s.A = p; p += s.nw;
    s.SO = p; p += s.ns;
    s.SA = p; p += s.ns;
    s.cnt = p; p += kWin;
    s.off = p; p += kWin + 1;
    s.isA = xpehh ? p : nullptr;
    s.PA = xpehh ? p + s.nw : nullptr;
    s.lst = (unsigned short *)(p + (xpehh ? 2 * s.nw : 0));
    return s;
}

__device__ __forceinline__ int c2i(unsigned k) { return (int)(k * (k - 1u) / 2u); }

// Bitmap searches with a third level: `sup` has bit q set when summary word q
// is non-zero (at most 16 summary words: n <= 16383), so neither search loops.
// last set position < b (b > 0; position 0 is always set)
__device__ __forceinline__ int prev_start(const unsigned *B, const unsigned *S, unsigned sup, int b)
{
    const int wd = b >> 5;
    const unsigned bits = B[wd] & ((1u << (b & 31)) - 1u);
    if (bits) return (wd << 5) + 31 - __clz(bits);
    const int sw = wd - 1;                       // >= 0: word 0 holds position 0
    int q = sw >> 5;
    unsigned sb = S[q] & (0xFFFFFFFFu >> (31 - (sw & 31)));
    if (!sb) {                                   // q > 0 here: summary word 0 has bit 0
        q = 31 - __clz(sup & ((1u << q) - 1u));
        sb = S[q];
    }
    const int ww = (q << 5) + 31 - __clz(sb);
    return (ww << 5) + 31 - __clz(B[ww]);
}

// first set position > b (b < n; position n is always set)
__device__ __forceinline__ int next_start(const unsigned *B, const unsigned *S, unsigned sup, int b)
{
    const int wd = b >> 5;
    const unsigned bits = B[wd] & ~((2u << (b & 31)) - 1u);
    if (bits) return (wd << 5) + __ffs(bits) - 1;
    const int sw = wd + 1;                       // a word up to the one of position n
    int q = sw >> 5;
    unsigned sb = S[q] & (0xFFFFFFFFu << (sw & 31));
    if (!sb) {
        q = __ffs(sup & ~((2u << q) - 1u)) - 1;
        sb = S[q];
    }
    const int ww = (q << 5) + __ffs(sb) - 1;
    return (ww << 5) + __ffs(B[ww]) - 1;
}

__device__ __forceinline__ unsigned count_a(const SplitSmem &s, int x)
{
    return s.PA[x >> 5] + (unsigned)__popc(s.isA[x >> 5] & ((1u << (x & 31)) - 1u));
}

// Offsets of the kWin step counts and placement of the K staged boundaries
// (position | step in window << 16 | rank in step << 32) by step.
template <int G, typename Tile>
__device__ const unsigned short *place_window(const Tile &tile, const SplitSmem &s, unsigned K,
                                             const unsigned long long *stage, unsigned short *list)
{
    const int lane = tile.thread_rank();
    tile.sync();
    constexpr int C = kWin / G;
    unsigned own = 0;
#pragma unroll
    for (int j = 0; j < C; ++j) own += s.cnt[C * lane + j];
    unsigned incl = own;
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
        const unsigned v = tile.shfl_up(incl, d);
        if (lane >= d) incl += v;
    }
    unsigned run = incl - own;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const unsigned c = s.cnt[C * lane + j];
        s.off[C * lane + j] = run;
        run += c;
    }
    if (lane == G - 1) s.off[kWin] = incl;
    tile.sync();
    // the list goes to shared memory when it fits, else to the global scratch
    unsigned short *dst = K <= (unsigned)kSplitListSmem ? s.lst : list;
    for (unsigned j = lane; j < K; j += G) {
        const unsigned long long e = stage[j];
        dst[s.off[(unsigned)(e >> 16) & (kWin - 1u)] + (unsigned)(e >> 32)] = (unsigned short)(e & 0xFFFFu);
    }
    tile.sync();
    return dst;
}

// Group the boundaries t with lo <= M[t] < lo + kWin by step: one pass over M
// (8 values per 16-byte load, four loads in flight per lane) marks the values
// in the window with two integer operations per 16-bit half; only the marked
// ones are ranked inside their step and staged, then placed by step.  Done by
// one tile of G lanes.  Window starts stay below 65,001 (run lengths are at
// most 65,000), so the all-ones fill past the slot's end is never marked.
template <int G, typename Tile>
__device__ const unsigned short *build_window(const Tile &tile, const SplitSmem &s, const unsigned *M32,
                                              int n, int lo, unsigned long long *stage,
                                              unsigned short *list)
{
    const int lane = tile.thread_rank();
    const uint4 *M4 = (const uint4 *)M32;
    const unsigned short *M16 = (const unsigned short *)M32;
    for (int q = lane; q < kWin; q += G) s.cnt[q] = 0u;
    tile.sync();
    const int n4 = (n + 7) >> 3;
    constexpr unsigned kOut = 0xFFFFu & ~(kWin - 1u);      // a 16-bit difference is in the window
    const unsigned ulo = (unsigned)lo, uhi = (unsigned)lo << 16;
    unsigned K = 0;
    for (int base = 0; base < n4; base += 4 * G) {
        uint4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = base + u * G + lane;
            q[u] = idx < n4 ? __ldg(M4 + idx) : make_uint4(~0u, ~0u, ~0u, ~0u);
        }
        // bit 8u + v: value v of this lane's u-th group of eight is in the window
        unsigned hit = 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const unsigned wv[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (((wv[j] - ulo) & kOut) == 0u) hit |= 1u << (8 * u + 2 * j);
                if (((wv[j] - uhi) & (kOut << 16)) == 0u) hit |= 1u << (8 * u + 2 * j + 1);
            }
        }
        if (base + 4 * G > n4 && (n & 7)) {      // the last group holds values past n
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (base + u * G + lane == n4 - 1) hit &= ~(((0xFFu << (n & 7)) & 0xFFu) << (8 * u));
        }
        if (tile.ballot(hit != 0u) == 0u) continue;
        const unsigned c = (unsigned)__popc(hit);
        unsigned incl = c;
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const unsigned v = tile.shfl_up(incl, d);
            if (lane >= d) incl += v;
        }
        unsigned at = K + incl - c;
        while (hit) {
            const int bb = __ffs(hit) - 1;
            hit &= hit - 1u;
            const int t = (base + (bb >> 3) * G + lane) * 8 + (bb & 7);
            const unsigned d = (unsigned)__ldg(M16 + t) - ulo;
            const unsigned r = atomicAdd(s.cnt + d, 1u);
            stage[at++] = (unsigned long long)t | ((unsigned long long)d << 16) | ((unsigned long long)r << 32);
        }
        K += tile.shfl(incl, G - 1);
    }
    return place_window<G>(tile, s, K, stage, list);
}


// Pair counts fit 32 bits (C(16383, 2) < 2^32); the digest and the cutoff
// product are 64-bit.
// The trapezoid sum (Eq. 4 / Eq. 5) is kept per lane: the lane that owns
// step i of the current G-step block (the lane whose map step it computed)
// records that step's integer term S(i-1) + S(i) in `rec`, and once per
// block every lane adds rec * g to its FP64 partial sum; the partial sums are
// added over the tile by a fixed butterfly when the walk ends.  One FP64
// multiply-add per lane and block instead of one per step (FP64 is a narrow
// pipe on this GPU); with 32-lane tiles the additions are exactly those of the
// per-step walk, so a walk handed over to it gives the same bits.
struct ClassWalk {
    unsigned D, S;
    unsigned rec;                   // this lane's step term of the current block (0: none)
    unsigned long long dig;
    unsigned thr;                   // stop at the first S < thr, i.e. cut_den * S < cut_num * D
    double acc;                     // this lane's partial trapezoid sum
    int stop;                       // the step the walk stopped at (status: at the end)
    bool active;
};

// Reductions of S caused by the boundaries b that part at this step
// (iHS: d0 class 0, d1 class 1; XPEHH: d0 A, d1 B, d2 pooled).  The pairs
// whose common run ends exactly at step i are counted once, at the leftmost
// boundary b of their span with M[b] = i: the first member lies in [p, b),
// p the last run start before b with M <= i (the bitmap A, this step's
// starts included), the second in [b, e), e the first old start after b
// (M < i, the bitmap O).  So boundary b removes (b - p)(e - b) pairs, and
// per population the products of its members on either side.
template <int NPOP>
__device__ __forceinline__ void split_terms(const SplitSmem &s, int b, int n0, unsigned supA,
                                            unsigned supO, int &d0, int &d1, int &d2)
{
    const int p = prev_start(s.A, s.SA, supA, b);
    const int e = next_start(s.O, s.SO, supO, b);
    if (NPOP == 2) {
        const unsigned ap = count_a(s, p), ab = count_a(s, b), ae = count_a(s, e);
        const unsigned l1a = ab - ap, l2a = ae - ab;
        const unsigned l1b = (unsigned)(b - p) - l1a, l2b = (unsigned)(e - b) - l2a;
        d0 -= (int)(l1a * l2a);
        d1 -= (int)(l1b * l2b);
        d2 -= (b - p) * (e - b);
    } else {
        const int dd = (b - p) * (e - b);
        if (b < n0) d0 -= dd;
        else d1 -= dd;
    }
}

// Steps that part more than G pairs (a few per walk): kept out of line so
// that the common one-round path stays small in the instruction cache.
template <int NPOP, int G, typename Tile>
__device__ __noinline__ unsigned split_many(const Tile &tile, const SplitSmem &s,
                                            const unsigned short *list, unsigned j0, unsigned j1,
                                            int n0, unsigned supA, unsigned supO, int &d0, int &d1,
                                            int &d2)
{
    const int lane = tile.thread_rank();
    unsigned r = 0u;
    for (unsigned j = j0 + lane; j < j1; j += G) {
        const int b = list[j];
        atomicOr(s.A + (b >> 5), 1u << (b & 31));
        atomicOr(s.SA + (b >> 10), 1u << ((b >> 5) & 31));
        r |= 1u << (b >> 10);
    }
    r = __reduce_or_sync(G == 32 ? 0xFFFFFFFFu : (0xFFFFu << (threadIdx.x & 16)), r);
    tile.sync();
    for (unsigned j = j0 + lane; j < j1; j += G)
        split_terms<NPOP>(s, (int)list[j], n0, supA | r, supO, d0, d1, d2);
    tile.sync();
    for (unsigned j = j0 + lane; j < j1; j += G) {
        const int b = list[j];
        atomicOr(s.O + (b >> 5), 1u << (b & 31));
        atomicOr(s.SO + (b >> 10), 1u << ((b >> 5) & 31));
    }
    return r;                                    // summary words that gained a start
}

}  // namespace

size_t split_smem_per_warp(int n, int xpehh)
{
    const int nw = split_nw(n), ns = (nw + 31) >> 5;
    size_t b = (size_t)nw * 4 * 2 + (size_t)ns * 4 * 2 + (size_t)(2 * kWin + 1) * 4;
    if (xpehh) b += (size_t)nw * 4 * 2;
    b += (size_t)kSplitListSmem * 2;
    return (b + 15) & ~(size_t)15;
}

size_t split_scratch_per_warp(int n) { return (((size_t)n * 10) + 255) & ~(size_t)255; }

// Persistent: each tile of G lanes (a warp, or half a warp so that one warp
// walks two cores at once) takes slots of this stage (both directions) from a
// counter and walks the cores in them.  iHS walks run four CTAs per SM at 64
// registers; the XPEHH walk (three pair counts per boundary, the population
// prefix table) spills more at that cap and runs three at 80 (1M XPEHH scan:
// 51.35 ms against 51.82).
#ifndef SPLIT_MIN_CTAS
#define SPLIT_MIN_CTAS 4
#endif
template <int NPOP, int G>
__global__ void __launch_bounds__(kSplitWarps * 32, NPOP == 2 ? 3 : SPLIT_MIN_CTAS) split_walk_kernel(SweepArgs w)
{
    extern __shared__ __align__(16) unsigned char smem[];
    namespace cg = cooperative_groups;
    const cg::thread_block_tile<G> tile = cg::tiled_partition<G>(cg::this_thread_block());
    constexpr int TPC = kSplitWarps * 32 / G;            // tiles per CTA
    const int lane = tile.thread_rank(), tix = threadIdx.x / G;
    const int n = w.n;
    SplitSmem s = split_smem(smem + (size_t)tix * w.split_bytes, n, NPOP == 2);
    unsigned char *scr = w.wscratch + ((size_t)blockIdx.x * TPC + tix) * w.wscratch_bytes;
    unsigned long long *stage = (unsigned long long *)scr;
    unsigned short *list = (unsigned short *)(scr + (size_t)n * 8);
    const long long per_dir = (long long)w.nch * w.R;
    const long long m = w.a.m;
    for (;;) {
        unsigned long long gs = 0;
        if (lane == 0) gs = atomicAdd(w.walk_head, 1ull);
        gs = tile.shfl(gs, 0);
        if (gs >= (unsigned long long)(2 * per_dir)) break;
        // slot counts are below 2^31 (2 x chunks x stage cores): 32-bit decode
        const unsigned gsl = (unsigned)gs;
        const long long gslot = (long long)gs;
        const unsigned cr = gsl / (unsigned)w.R;
        const int r = (int)(gsl - cr * (unsigned)w.R);
        const int dir = cr >= (unsigned)w.nch ? 1 : 0;
        const int c = (int)(cr - (unsigned)dir * (unsigned)w.nch);
        const long long c0 = w.a.k0 + (long long)c * w.B;
        if (c0 >= w.a.k1) continue;
        const long long c1 = c0 + w.B < w.a.k1 ? c0 + w.B : w.a.k1;
        long long k;
        if (dir == 0) {
            const long long klo = c0 + (long long)w.stage * w.R;
            const long long khi = klo + w.R < c1 ? klo + w.R : c1;
            k = klo + r;
            if (k >= khi) continue;
        } else {
            const long long khi = c1 - (long long)w.stage * w.R;
            const long long klo = khi - w.R > c0 ? khi - w.R : c0;
            k = khi - 1 - r;
            if (k < klo) continue;
        }
        if (w.sk.core_status[k] == (int8_t)SELSCAN_LOCUS_MAF_FILTERED) continue;

        const unsigned char *slot = w.slots + (size_t)gslot * w.slot_bytes;
        const int n0 = ((const int *)slot)[0];
        const int hz = ((const int *)slot)[1];
        const int w1 = ((const int *)slot)[2];
        const unsigned *M32 = (const unsigned *)(slot + 16);

        for (int q = lane; q < s.nw; q += G) { s.O[q] = 0u; s.A[q] = 0u; }
        for (int q = lane; q < s.ns; q += G) { s.SO[q] = 0u; s.SA[q] = 0u; }
        if (NPOP == 2) {
            const unsigned *isA = (const unsigned *)(slot + slot_isa_at(n));
            unsigned carry = 0u;
            for (int base = 0; base < s.nw; base += G) {
                const int q = base + lane;
                const unsigned v = q < s.nw ? __ldg(isA + q) : 0u;
                const unsigned pc = (unsigned)__popc(v);
                unsigned incl = pc;
#pragma unroll
                for (int d = 1; d < G; d <<= 1) {
                    const unsigned u = tile.shfl_up(incl, d);
                    if (lane >= d) incl += u;
                }
                if (q < s.nw) { s.isA[q] = v; s.PA[q] = carry + incl - pc; }
                carry += tile.shfl(incl, G - 1);
            }
        }
        tile.sync();
        if (lane < 3) {                           // run starts before step 1: 0, n0, n
            const int mk = lane == 0 ? 0 : (lane == 1 ? n0 : n);
            atomicOr(s.O + (mk >> 5), 1u << (mk & 31));
            atomicOr(s.SO + (mk >> 10), 1u << ((mk >> 5) & 31));
            atomicOr(s.A + (mk >> 5), 1u << (mk & 31));
            atomicOr(s.SA + (mk >> 10), 1u << ((mk >> 5) & 31));
        }
        tile.sync();
        // summary words with a start (third level of both bitmaps)
        unsigned supA = 1u | (1u << (n0 >> 10)) | (1u << (n >> 10)), supO = supA;

        // ---- step 0 (the core marker splits the sample into its allele classes)
        constexpr int NWK = NPOP == 2 ? 1 : 2;    // walks handled by this warp
        ClassWalk cw[NWK];
        unsigned SA = 0, SB = 0, pA = 0, pB = 0, DA = 0, DB = 0;
        unsigned long long dA = 0, dB = 0;
        double accB = 0.0;                  // XPEHH: population B's partial sum (A's in cw[0])
        unsigned recB = 0;
        if (NPOP == 2) {
            const unsigned nA = (unsigned)w.a.nA, nB = (unsigned)w.a.nB;
            const unsigned a0 = count_a(s, n0), a1 = nA - a0;
            const unsigned b0 = (unsigned)n0 - a0, b1 = nB - b0;
            SA = (unsigned)(c2i(a0) + c2i(a1));
            SB = (unsigned)(c2i(b0) + c2i(b1));
            DA = (unsigned)c2i(nA);
            DB = (unsigned)c2i(nB);
            cw[0].D = (unsigned)c2i((unsigned)n);
            cw[0].S = (unsigned)(c2i((unsigned)n0) + c2i((unsigned)(n - n0)));
            pA = SA; pB = SB;
            dA = SA; dB = SB;
        } else {
            cw[0].D = (unsigned)c2i((unsigned)n0);             // allele 0: positions [0, n0)
            cw[1].D = (unsigned)c2i((unsigned)(n - n0));       // allele 1: positions [n0, n)
            cw[0].S = cw[0].D;
            cw[1].S = cw[1].D;
        }
        bool any = false;
#pragma unroll
        for (int q = 0; q < NWK; ++q) {
            {
                const unsigned long long t =
                    ((unsigned long long)w.a.cut_num * cw[q].D + w.a.cut_den - 1u) / w.a.cut_den;
                cw[q].thr = t < 0xFFFFFFFFull ? (unsigned)t : 0xFFFFFFFFu;
            }
            cw[q].dig = cw[q].S;
            cw[q].acc = 0.0;
            cw[q].rec = 0u;
            cw[q].stop = 0;
            cw[q].active = cw[q].D != 0u;
            any |= cw[q].active;
        }

        const long long step = dir ? 1 : -1;
        double gq = 0.0;        // this lane's step of the current G-step block: the map step g
        int gk = 0;             // its kind: 0 a step, WALK_EDGE past the array end, WALK_GAP a gap abort
        // steps [lo, lo + wlen) are grouped in cl: first the slot's window
        // (steps 1..w1), then windows of kWin steps found in M
        int lo = 1, wlen = w1 > 0 ? w1 : kWin;
        const unsigned short *cl = s.lst;
        if (any) {
            if (w1 > 0) {                        // the slot's list, copied on chip
                const unsigned short *so = (const unsigned short *)(slot + slot_off_at(n, NPOP == 2));
                const unsigned *sl = (const unsigned *)(slot + slot_list_at(n, NPOP == 2));
                for (int q = lane; q <= w1; q += G) s.off[q] = so[q];
                const int kw = ((int)so[w1] + 1) >> 1;
#pragma unroll 4
                for (int q = lane; q < kw; q += G) ((unsigned *)s.lst)[q] = __ldg(sl + q);
                tile.sync();
            } else {
                cl = build_window<G>(tile, s, M32, n, lo, stage, list);
            }
        }
        int fin = WALK_OK;                           // how the still-active walks end
        int i = 1;                              // walks stay below 2^31 steps (a chunk history)
        for (; any; ++i) {
            const int own_step = (int)((i - 1) & (G - 1));   // the lane that owns step i
            if (own_step == 0) {                  // gaps and map steps of the next G steps
                if (i > 1) {                      // the previous block's terms
#pragma unroll
                    for (int q = 0; q < NWK; ++q) { cw[q].acc += (double)cw[q].rec * gq; cw[q].rec = 0u; }
                    if (NPOP == 2) { accB += (double)recB * gq; recB = 0u; }
                }
                const long long xl = k + step * (i + lane), xp = xl - step;
                gq = 0.0;
                gk = 0;
                if (xl < 0 || xl >= m) gk = WALK_EDGE;
                else {
                    const long long p1 = __ldg(w.a.pos + xl), p0 = __ldg(w.a.pos + xp);
                    const long long bp = dir ? p1 - p0 : p0 - p1;
                    if (bp > w.a.max_gap) gk = WALK_GAP;
                    else {
                        double gg;
                        if (w.a.physical) gg = (double)bp;
                        else {
                            const double g1 = __ldg(w.a.gmap + xl), g0 = __ldg(w.a.gmap + xp);
                            gg = dir ? g1 - g0 : g0 - g1;
                        }
                        if (bp > w.a.gap_scale) gg = gg * ((double)w.a.gap_scale / (double)bp);
                        gq = gg;
                    }
                }
            }
            const int kind = tile.shfl(gk, own_step);
            if (kind != 0) { fin = kind; break; }
            const bool own = lane == own_step;
            if (i > hz) { fin = WALK_UNFINISHED; break; }
            if (i >= lo + wlen) {
                lo += wlen;
                wlen = kWin;
                cl = build_window<G>(tile, s, M32, n, lo, stage, list);
            }
            // ---- the boundaries that part at this step
            const unsigned j0 = s.off[i - lo], j1 = s.off[i - lo + 1];
            int d0 = 0, d1 = 0, d2 = 0;
            if (j1 > j0) {
                // new run starts first, then their reductions, then merge
                if (j1 - j0 <= (unsigned)G) {     // one boundary per lane, loaded once
                    bool has = lane < (int)(j1 - j0);
                    const int b = has ? (int)cl[j0 + lane] : 0;
                    // an iHS class whose walk has ended needs its runs no more
                    if (NPOP == 1) has = has && (b < n0 ? cw[0].active : cw[NWK - 1].active);
                    const unsigned bw = 1u << (b & 31), sw = 1u << ((b >> 5) & 31);
                    if (tile.ballot(has) != 0u) {
                    if (has) {
                        atomicOr(s.A + (b >> 5), bw);
                        atomicOr(s.SA + (b >> 10), sw);
                    }
                    const unsigned r = __reduce_or_sync(G == 32 ? 0xFFFFFFFFu : (0xFFFFu << (threadIdx.x & 16)),
                                                        has ? 1u << (b >> 10) : 0u);
                    supA |= r;
                    tile.sync();
                    if (has) split_terms<NPOP>(s, b, n0, supA, supO, d0, d1, d2);
                    tile.sync();
                    // this step's starts become old ones; the next step reads O
                    // only after its own sync
                    if (has) {
                        atomicOr(s.O + (b >> 5), bw);
                        atomicOr(s.SO + (b >> 10), sw);
                    }
                    supO |= r;
                    }
                } else {
                    const unsigned r = split_many<NPOP, G>(tile, s, cl, j0, j1, n0, supA, supO, d0, d1, d2);
                    supA |= r;
                    supO |= r;
                }
                d0 = cg::reduce(tile, d0, cg::plus<int>());
                d1 = cg::reduce(tile, d1, cg::plus<int>());
                if (NPOP == 2) d2 = cg::reduce(tile, d2, cg::plus<int>());
            }
            const unsigned ii = (unsigned)(i + 1);
            if (NPOP == 2) {
                SA += (unsigned)d0;                  // the decrements are negative: S stays >= 0
                SB += (unsigned)d1;
                ClassWalk &q = cw[0];
                q.S += (unsigned)d2;
                dA += (unsigned long long)ii * SA;
                dB += (unsigned long long)ii * SB;
                q.dig += (unsigned long long)ii * q.S;
                const bool stop = q.S < q.thr;
                if (stop && !w.a.crossing) { q.stop = (int)i; q.active = false; }
                else {
                    if (own) {
                        q.rec = pA + SA;
                        recB = pB + SB;
                    }
                    if (stop) { q.stop = (int)i; q.active = false; }
                    pA = SA;
                    pB = SB;
                }
            } else {
#pragma unroll
                for (int c_ = 0; c_ < 2; ++c_) {
                    ClassWalk &q = cw[c_];
                    if (!q.active) continue;
                    q.S += (unsigned)(c_ ? d1 : d0);
                    q.dig += (unsigned long long)ii * q.S;
                    const bool stop = q.S < q.thr;
                    if (stop && !w.a.crossing) { q.stop = (int)i; q.active = false; continue; }
                    if (own) q.rec = 2u * q.S - (unsigned)(c_ ? d1 : d0);   // S(i - 1) + S(i)
                    if (stop) { q.stop = (int)i; q.active = false; continue; }
                }
            }
            any = false;
#pragma unroll
            for (int q = 0; q < NWK; ++q) any |= cw[q].active;
        }
        // ---- the last block's terms, then the tile's sum of the partial sums
#pragma unroll
        for (int q = 0; q < NWK; ++q) {
            cw[q].acc += (double)cw[q].rec * gq;
            cw[q].acc = lane_sum_f64<G>(cw[q].acc);
        }
        if (NPOP == 2) {
            accB += (double)recB * gq;
            accB = lane_sum_f64<G>(accB);
        }
        // ---- results (lane 0)
        if (lane == 0) {
            const ItemSink &sk = w.sk;
#pragma unroll
            for (int q_ = 0; q_ < NWK; ++q_) {
                ClassWalk &q = cw[q_];
                // iHS items: (allele 1, down), (allele 1, up), (allele 0, down), (allele 0, up)
                const uint32_t item = NPOP == 2 ? (uint32_t)(k * 2 + dir)
                                                : (uint32_t)(k * 4 + (q_ == 1 ? 0 : 2) + dir);
                int status = q.D == 0u ? WALK_UNDEFINED : WALK_OK;
                if (q.active) {
                    if (fin == WALK_UNFINISHED) {
                        const unsigned long long slot2 = atomicAdd(&sk.q->n2, 1ull);
                        sk.list2[slot2] = item;
                        sk.key2[slot2] = bucket_of((float)((double)q.S / (double)q.D));
                        continue;
                    }
                    status = fin;
                    q.stop = (int)i;
                }
                sk.item_status[item] = (int8_t)status;
                sk.stop[item] = q.stop;
                if (NPOP == 2) {
                    sk.item_ihh[2 * (size_t)item] = DA ? q.acc / (2.0 * (double)DA) : 0.0;
                    sk.item_ihh[2 * (size_t)item + 1] = DB ? accB / (2.0 * (double)DB) : 0.0;
                    sk.digest[3 * (size_t)item] = dA;
                    sk.digest[3 * (size_t)item + 1] = dB;
                    sk.digest[3 * (size_t)item + 2] = q.dig;
                } else {
                    sk.item_ihh[item] = q.D ? q.acc / (2.0 * (double)q.D) : 0.0;
                    sk.digest[item] = q.D ? q.dig : 0ull;
                }
            }
        }
        tile.sync();
    }
}

template <int G>
static void (*walk_kernel_for(int xpehh))(SweepArgs)
{
    return xpehh ? split_walk_kernel<2, G> : split_walk_kernel<1, G>;
}

static void (*walk_kernel(int xpehh, int tile))(SweepArgs)
{
    return tile == 16 ? walk_kernel_for<16>(xpehh) : walk_kernel_for<32>(xpehh);
}

int split_walk_ctas(int n, int xpehh, int tile)
{
    // resident CTAs of the persistent walker
    int per_sm = 0;
    const size_t smem = split_smem_per_warp(n, xpehh) * (kSplitWarps * 32 / tile);
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, walk_kernel(xpehh, tile), kSplitWarps * 32, smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * (sms > 0 ? sms : 1);
}

cudaError_t launch_sweep_path(const SweepArgs &w0, cudaStream_t s)
{
    SweepArgs w = w0;
    const size_t ssm = sweep_smem_bytes(w.n, w.a.W, w.threads, w.R);
    const int E = sweep_e(w.n, w.threads);
    void (*sweep)(SweepArgs);
    if (w.threads == 256)
        sweep = E == 4 ? sweep_kernel<256, 4, true> : E == 8 ? sweep_kernel<256, 8, true>
              : E == 12 ? sweep_kernel<256, 12, true> : E == 16 ? sweep_kernel<256, 16, true>
              : E == 20 ? sweep_kernel<256, 20, true> : E == 24 ? sweep_kernel<256, 24, true>
              : sweep_kernel<256, 32>;
    else if (w.threads == 512)
        sweep = E <= 4 ? sweep_kernel<512, 4> : E <= 8 ? sweep_kernel<512, 8>
              : E <= 16 ? sweep_kernel<512, 16> : E <= 24 ? sweep_kernel<512, 24>
              : sweep_kernel<512, 32>;
    else if (w.threads == 128)
        sweep = E <= 8 ? sweep_kernel<128, 8> : E <= 16 ? sweep_kernel<128, 16> : sweep_kernel<128, 32>;
    else if (w.threads == 64)
        sweep = E <= 8 ? sweep_kernel<64, 8> : E <= 16 ? sweep_kernel<64, 16> : sweep_kernel<64, 32>;
    else
        sweep = E <= 8 ? sweep_kernel<32, 8> : E <= 16 ? sweep_kernel<32, 16> : sweep_kernel<32, 32>;
    cudaError_t e = cudaFuncSetAttribute(sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm);
    if (e != cudaSuccess) return e;
    const size_t wsm = (size_t)w.split_bytes * (kSplitWarps * 32 / w.split_tile);
    void (*walk)(SweepArgs) = walk_kernel(w.a.nB > 0, w.split_tile);
    if ((e = cudaFuncSetAttribute(walk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm)) !=
        cudaSuccess)
        return e;
    for (int st = 0; st < w.nstages; ++st) {
        w.stage = st;
        sweep<<<2 * w.nch, w.threads, ssm, s>>>(w);
        if (st == 0 && w.sweep_done_event &&
            (e = cudaEventRecord((cudaEvent_t)w.sweep_done_event, s)) != cudaSuccess)
            return e;
        walk<<<w.walk_ctas, kSplitWarps * 32, wsm, s>>>(w);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace selscan
