// Runs the sorted sweep (all chunks and stages) and the split walk (one warp
// taking every slot) of one scan on the host, from the kernels' own source
// (kernels_host.h, written by extract.py), and writes the per-item results.
// Test infrastructure only.
//   args: n nA nB W WA m L R T nch B rows status pos gmap out
//   T is 32, 64 (up to 8 haplotypes a thread) or 256 (4 a thread).
#include "kernels_host.h"
thread_local dim3e threadIdx;
dim3e blockIdx;
unsigned char *g_smem;
thread_local WarpCtx *g_warp;
SpinBarrier *g_block;
using namespace selscan;

template <typename T> std::vector<T> readf(const char *path, size_t n)
{
    std::vector<T> v(n);
    FILE *f = fopen(path, "rb");
    if (!f || fread(v.data(), sizeof(T), n, f) != n) { fprintf(stderr, "read %s\n", path); exit(2); }
    fclose(f);
    return v;
}

// one CTA of T threads; each thread runs `body` with its threadIdx
template <class F> void run_threads(int T, size_t smem, F body)
{
    std::vector<unsigned char> sm(smem, 0xA5);
    g_smem = sm.data();
    SpinBarrier blk(T);
    g_block = &blk;
    std::vector<WarpCtx *> warps;
    for (int i = 0; i < (T + 31) / 32; ++i) warps.push_back(new WarpCtx());
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t)
        th.emplace_back([&, t] {
            threadIdx.x = t;
            g_warp = warps[t / 32];
            body();
        });
    for (auto &x : th) x.join();
    for (auto *p : warps) delete p;
}

int main(int argc, char **argv)
{
    if (argc < 17) { fprintf(stderr, "args\n"); return 2; }
    const int n = atoi(argv[1]), nA = atoi(argv[2]), nB = atoi(argv[3]), W = atoi(argv[4]),
              WA = atoi(argv[5]);
    const long long m = atoll(argv[6]);
    const int L = atoi(argv[7]), R = atoi(argv[8]), T = atoi(argv[9]), nch = atoi(argv[10]);
    const long long B = atoll(argv[11]);
    const int xp = nB > 0;
    std::vector<unsigned long long> hap = readf<unsigned long long>(argv[12], (size_t)m * W);
    std::vector<int8_t> cs = readf<int8_t>(argv[13], (size_t)m);
    std::vector<long long> pos = readf<long long>(argv[14], (size_t)m);
    std::vector<double> gm = readf<double>(argv[15], (size_t)m);
    const int E = sweep_e(n, T);
    const size_t ssm = sweep_smem_bytes(n, W, T, R);
    std::vector<unsigned> state((size_t)2 * nch * E * T);
    const size_t slot_bytes = sweep_slot_bytes(n, xp);
    std::vector<unsigned char> slots((size_t)2 * nch * R * slot_bytes, 0);
    unsigned long long head = 0;
    int32_t err = 0;
    const long long items = m * (xp ? 2 : 4);
    std::vector<int8_t> istat(items, 0x7F);
    std::vector<double> ihh(items * 2, 0.0);
    std::vector<int32_t> stop(items, 0);
    std::vector<unsigned long long> dig(items * 3, 0);
    std::vector<uint32_t> list2(items), key2(items);
    Queue qq;
    memset(&qq, 0, sizeof(qq));
    SweepArgs w;
    memset(&w, 0, sizeof(w));
    w.a.hap = hap.data(); w.a.ld = W; w.a.m = m; w.a.k0 = 0; w.a.k1 = m; w.a.W = W; w.a.WA = WA;
    w.a.nA = nA; w.a.nB = nB; w.a.pos = pos.data(); w.a.gmap = gm.data();
    w.a.cut_num = 1; w.a.cut_den = 20; w.a.gap_scale = 20000; w.a.max_gap = 200000;
    w.sk.mode = xp; w.sk.core_status = cs.data(); w.sk.item_status = istat.data();
    w.sk.item_ihh = ihh.data(); w.sk.stop = stop.data(); w.sk.digest = dig.data();
    w.sk.list2 = list2.data(); w.sk.key2 = key2.data(); w.sk.q = &qq;
    w.n = n; w.threads = T; w.nch = nch; w.B = B; w.L = L; w.R = R;
    w.nstages = (int)((B + R - 1) / R);
    w.st = (unsigned short *)state.data(); w.slots = slots.data(); w.slot_bytes = slot_bytes;
    w.walk_head = &head; w.err = &err;
    w.split_bytes = (int)split_smem_per_warp(n, xp);
    w.split_tile = 32;
    w.wscratch_bytes = split_scratch_per_warp(n);
    std::vector<unsigned char> wscr(w.wscratch_bytes * kSplitWarps);
    w.wscratch = wscr.data();
    w.walk_ctas = 1;
    for (int s = 0; s < w.nstages; ++s) {
        w.stage = s;
        for (int b = 0; b < 2 * nch; ++b) {
            blockIdx.x = b;
            if (T == 32 && E <= 8) run_threads(32, ssm, [&] { sweep_kernel<32, 8>(w); });
            else if (T == 64 && E <= 8) run_threads(64, ssm, [&] { sweep_kernel<64, 8>(w); });
            else if (T == 256 && E == 4) run_threads(256, ssm, [&] { sweep_kernel<256, 4, true>(w); });
            else { fprintf(stderr, "unsupported shape T %d E %d\n", T, E); return 2; }
        }
        blockIdx.x = 0;                          // one warp takes every slot of the stage
        const size_t wsm = (size_t)w.split_bytes * kSplitWarps;
        if (xp) run_threads(32, wsm, [&] { split_walk_kernel<2, 32>(w); });
        else run_threads(32, wsm, [&] { split_walk_kernel<1, 32>(w); });
    }
    FILE *f = fopen(argv[16], "wb");
    fwrite(istat.data(), 1, items, f);
    fwrite(stop.data(), 4, items, f);
    fwrite(ihh.data(), 8, items * 2, f);
    fwrite(dig.data(), 8, items * 3, f);
    fwrite(&qq.n2, 8, 1, f);
    fclose(f);
    printf("err %d handed-off %llu\n", err, (unsigned long long)qq.n2);
    return err != 0;
}
