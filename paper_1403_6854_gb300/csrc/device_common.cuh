// Device helpers shared by the walk kernels (kernels.cu, batch.cu).
#pragma once
#include "internal.h"

namespace selscan {

__device__ __forceinline__ WarpBufs make_bufs(unsigned char *sm, unsigned char *gm,
                                              const Scratch &sc)
{
    WarpBufs b;
    b.cap_s = sc.cap_s;
    b.cap = sc.cap;
    b.tcap_s = sc.tcap_s;
    b.tcap = sc.tcap;
    b.pool_s = (unsigned long long *)sm;
    b.tab_s = (unsigned long long *)(sm + (size_t)sc.cap_s * 8);
    b.pool_g = (unsigned long long *)gm;
    b.tab_g = (unsigned long long *)(gm + (size_t)sc.cap * 8);
    b.big = (unsigned short *)(b.tab_g + sc.tcap);
    b.err = sc.err;
    unsigned char *w = sm + (size_t)sc.cap_s * 8 + (size_t)sc.tcap_s * 8;
    b.wrow[0] = w; w += sc.rowcap;
    b.wrow[1] = w; w += sc.rowcap;
    b.wpos[0] = (long long *)w; w += sc.poscap;
    b.wpos[1] = (long long *)w; w += sc.poscap;
    b.wgm[0] = (double *)w; w += sc.poscap;
    b.wgm[1] = (double *)w; w += sc.poscap;
    b.bar = (unsigned long long *)w;
    b.R = sc.R;
    b.bigt = sc.bigt;
    return b;
}

// one-time set-up of the warp's two window mbarriers (fresh shared memory)
__device__ __forceinline__ void init_window(const WarpBufs &b)
{
    if ((threadIdx.x & 31) == 0) {
        mbar_init(b.bar, 1u);
        mbar_init(b.bar + 1, 1u);
    }
    fence_proxy_async();
    __syncwarp();
}

__host__ __device__ __forceinline__ size_t slice_bytes(const Scratch &sc)
{
    return smem_per_warp(sc.cap_s, sc.tcap_s, sc.rowcap, sc.poscap);
}

__device__ __forceinline__ uint32_t bucket_of(float ehh)
{
    // longer expected walks (higher EHH at the probe cap) get lower buckets
    if (!(ehh > 0.f)) return NBUCKET - 1;
    float b = -__log2f(ehh) * 16.f;
    if (b < 0.f) b = 0.f;
    if (b > (float)(NBUCKET - 1)) b = (float)(NBUCKET - 1);
    return (uint32_t)b;
}

// Runs one walk and stores its result.  Returns false if the warp must stop
// taking walks: a bounded wait for its window copies gave up (the error word
// holds SELSCAN_ERR_TIMEOUT), so a copy may still land in its buffers.  The
// launch's results are then invalid as a whole (every scan of a batch tick).
template <int NPOP>
__device__ __forceinline__ bool run_item(const ScanArgs &a, const ItemSink &sk, WarpBufs &b,
                                         uint32_t item, int max_steps, unsigned wpar[2])
{
    const int lane = threadIdx.x & 31;
    const int ipc = NPOP == 2 ? 2 : 4;
    const long long core = item / ipc;
    const int q = (int)(item % ipc);
    const int dir = q & 1;
    const int sel = NPOP == 2 ? 0 : (q < 2 ? 0 : 1);
    WalkOut o = walk<NPOP>(a, core, dir, sel, b, nullptr, 0, max_steps, wpar);
    const bool go_on = !o.abandon;
    if (lane != 0) return go_on;
    if (o.status == WALK_UNFINISHED) {
        const unsigned long long slot = atomicAdd(&sk.q->n2, 1ull);
        sk.list2[slot] = item;
        sk.key2[slot] = bucket_of(o.key);
        return go_on;
    }
    sk.item_status[item] = (int8_t)o.status;
    sk.stop[item] = o.stop;
    if (NPOP == 2) {
        sk.item_ihh[2 * (size_t)item] = o.ihh[0];
        sk.item_ihh[2 * (size_t)item + 1] = o.ihh[1];
        sk.digest[3 * (size_t)item] = o.dig[0];
        sk.digest[3 * (size_t)item + 1] = o.dig[1];
        sk.digest[3 * (size_t)item + 2] = o.dig[2];
    } else {
        sk.item_ihh[item] = o.ihh[0];
        sk.digest[item] = o.dig[0];
    }
    return go_on;
}

}  // namespace selscan
