// Host stand-ins for the CUDA constructs the sorting and split-walk kernels
// use, so that their source runs on the CPU: one OS thread per CUDA thread,
// a spinning barrier for __syncthreads, per-warp exchange buffers for
// shuffles, ballots and reductions, and the integer intrinsics written from
// their documented semantics.  Test infrastructure only (the library never
// includes it).
#pragma once
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>
#include <sched.h>

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __noinline__
#define __launch_bounds__(...)
#define __align__(x)

struct uint2 { unsigned x, y; };
struct uint4 { unsigned x, y, z, w; };
inline uint2 make_uint2(unsigned a, unsigned b) { return uint2{a, b}; }
inline uint4 make_uint4(unsigned a, unsigned b, unsigned c, unsigned d) { return uint4{a, b, c, d}; }
struct dim3e { unsigned x = 0, y = 0, z = 0; };
extern thread_local dim3e threadIdx;
extern dim3e blockIdx;
extern unsigned char *g_smem;

// a reusable barrier of n threads; gives up (and exits) after 60 s so that a
// divergent barrier shows as a failure, not a hang
struct SpinBarrier {
    std::atomic<int> count{0}, gen{0};
    int n;
    explicit SpinBarrier(int n_) : n(n_) {}
    void arrive_and_wait()
    {
        const int g = gen.load(std::memory_order_acquire);
        if (count.fetch_add(1, std::memory_order_acq_rel) == n - 1) {
            count.store(0, std::memory_order_relaxed);
            gen.fetch_add(1, std::memory_order_acq_rel);
            return;
        }
        const auto t0 = std::chrono::steady_clock::now();
        long k = 0;
        while (gen.load(std::memory_order_acquire) == g) {
            sched_yield();
            if ((++k & 4095) == 0 && std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60)) {
                fprintf(stderr, "barrier: threads never met\n");
                std::_Exit(3);
            }
        }
    }
};
struct WarpCtx {
    SpinBarrier bar{32};
    unsigned long long v[32];
};
extern thread_local WarpCtx *g_warp;
extern SpinBarrier *g_block;
#define __syncthreads() (g_block->arrive_and_wait())


template <typename T> inline unsigned long long to_u64(T v) { unsigned long long r = 0; memcpy(&r, &v, sizeof(T)); return r; }
template <typename T> inline T from_u64(unsigned long long r) { T v; memcpy(&v, &r, sizeof(T)); return v; }
// every lane of the warp publishes a value, then reads lane src's
template <typename T> inline T shfl_idx(T v, int src)
{
    const int lane = threadIdx.x & 31;
    g_warp->v[lane] = to_u64(v);
    g_warp->bar.arrive_and_wait();
    T r = from_u64<T>(g_warp->v[src & 31]);
    g_warp->bar.arrive_and_wait();
    return r;
}
template <typename T> inline T __shfl_sync(unsigned, T v, int src) { return shfl_idx(v, src); }
template <typename T> inline T __shfl_up_sync(unsigned, T v, int d)
{
    const int lane = threadIdx.x & 31;
    return shfl_idx(v, lane - d < 0 ? lane : lane - d);
}
template <typename T> inline T __shfl_xor_sync(unsigned, T v, int d) { return shfl_idx(v, (threadIdx.x & 31) ^ d); }
inline unsigned __ballot_sync(unsigned, int pred)
{
    const int lane = threadIdx.x & 31;
    g_warp->v[lane] = pred ? 1 : 0;
    g_warp->bar.arrive_and_wait();
    unsigned r = 0;
    for (int l = 0; l < 32; ++l) r |= (unsigned)g_warp->v[l] << l;
    g_warp->bar.arrive_and_wait();
    return r;
}
inline unsigned __reduce_or_sync(unsigned, unsigned v)
{
    g_warp->v[threadIdx.x & 31] = v;
    g_warp->bar.arrive_and_wait();
    unsigned r = 0;
    for (int l = 0; l < 32; ++l) r |= (unsigned)g_warp->v[l];
    g_warp->bar.arrive_and_wait();
    return r;
}
inline int __reduce_add_sync(unsigned, int v)
{
    g_warp->v[threadIdx.x & 31] = (unsigned)v;
    g_warp->bar.arrive_and_wait();
    unsigned r = 0;
    for (int l = 0; l < 32; ++l) r += (unsigned)g_warp->v[l];
    g_warp->bar.arrive_and_wait();
    return (int)r;
}
inline unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }
inline int __popc(unsigned x) { return __builtin_popcount(x); }
inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }
inline int __ffs(unsigned x) { return x ? __builtin_ctz(x) + 1 : 0; }
inline unsigned __umulhi(unsigned a, unsigned b) { return (unsigned)(((unsigned long long)a * b) >> 32); }
// 16-bit SIMD minimum / maximum of the two halves
inline unsigned __vminu2(unsigned a, unsigned b)
{
    return std::min(a & 0xFFFFu, b & 0xFFFFu) | (std::min(a >> 16, b >> 16) << 16);
}
inline unsigned __vmaxu2(unsigned a, unsigned b)
{
    return std::max(a & 0xFFFFu, b & 0xFFFFu) | (std::max(a >> 16, b >> 16) << 16);
}
// byte permute: result byte i = byte (s >> 4i) & 7 of the pair (y:x)
inline unsigned __byte_perm(unsigned x, unsigned y, unsigned s)
{
    unsigned char b[8];
    memcpy(b, &x, 4);
    memcpy(b + 4, &y, 4);
    unsigned r = 0;
    for (int i = 0; i < 4; ++i) r |= (unsigned)b[(s >> (4 * i)) & 7] << (8 * i);
    return r;
}
// right funnel shift of the 64-bit pair (hi:lo) by sh mod 32
inline unsigned __funnelshift_r(unsigned lo, unsigned hi, unsigned sh)
{
    const unsigned long long v = ((unsigned long long)hi << 32) | lo;
    return (unsigned)(v >> (sh & 31));
}
inline unsigned atomicAdd(unsigned *p, unsigned v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline unsigned atomicOr(unsigned *p, unsigned v) { return __atomic_fetch_or(p, v, __ATOMIC_SEQ_CST); }
template <typename T> inline T __ldg(const T *p) { return *p; }
inline float __log2f(float x) { return std::log2(x); }
using std::max;
using std::min;

// the cooperative-groups calls of the split walk, for whole-warp tiles
namespace cooperative_groups {
struct thread_block {};
inline thread_block this_thread_block() { return {}; }
template <int G> struct thread_block_tile {
    static_assert(G == 32, "host emulation: whole-warp tiles only");
    int thread_rank() const { return threadIdx.x & 31; }
    template <class T> T shfl(T v, int src) const { return shfl_idx(v, src & 31); }
    template <class T> T shfl_up(T v, int d) const
    {
        const int l = threadIdx.x & 31;
        return shfl_idx(v, l >= d ? l - d : l);
    }
    unsigned ballot(int p) const { return __ballot_sync(0xFFFFFFFFu, p); }
    void sync() const { g_warp->bar.arrive_and_wait(); }
};
template <int G> thread_block_tile<G> tiled_partition(thread_block) { return {}; }
template <class T> struct plus { T operator()(T a, T b) const { return a + b; } };
template <class Tile, class T, class Op> T reduce(const Tile &, T v, Op op)
{
    for (int d = 1; d < 32; d <<= 1) v = op(v, shfl_idx(v, (threadIdx.x & 31) ^ d));
    return v;
}
}  // namespace cooperative_groups
