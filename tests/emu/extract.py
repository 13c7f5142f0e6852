"""Build a host-compilable copy of the sorting kernel and the split walk.

The kernels' own source (paper_1403_6854_gb300/csrc/sweep.cu) is taken as
it stands; the argument structs, walk outcomes and small device helpers it
needs come from the library's headers by name; the few device-only lines
(inline PTX of the byte permute in sign-replicate mode, cp.async copies, the
dynamic shared-memory declaration) are replaced by host equivalents.  The
result runs under tests/emu/cuda_host.h (one OS thread per CUDA thread).
Test infrastructure only."""
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "..", "paper_1403_6854_gb300", "csrc")


def _block(text, start):
    """From the first occurrence of `start` to the end of its brace block (and a
    trailing ';' if there is one)."""
    i = text.index(start)
    j = text.index("{", i)
    depth = 0
    for k in range(j, len(text)):
        if text[k] == "{":
            depth += 1
        elif text[k] == "}":
            depth -= 1
            if depth == 0:
                end = k + 1
                if text[end:end + 1] == ";":
                    end += 1
                return text[i:end]
    raise ValueError(start)


def _line(text, start):
    i = text.index(start)
    return text[i:text.index("\n", i)]


def build(out_path):
    sweep = open(os.path.join(CSRC, "sweep.cu")).read()
    walk = open(os.path.join(CSRC, "walk.cuh")).read()
    internal = open(os.path.join(CSRC, "internal.h")).read()
    common = open(os.path.join(CSRC, "device_common.cuh")).read()
    pre = ["#include \"cuda_host.h\"", "#include \"selscan.h\"",
           "#define FULLMASK 0xffffffffu",
           "inline void cp_async8(void *dst, const void *src) { memcpy(dst, src, 8); }",
           "inline void cp_async_commit() {}",
           "template <int N> inline void cp_async_wait() {}",
           "namespace selscan {",
           _block(walk, "enum : int {"),
           _block(walk, "struct ScanArgs {"),
           _block(internal, "struct Queue {"),
           _block(internal, "struct ItemSink {"),
           _line(internal, "constexpr int NBUCKET"),
           _line(internal, "constexpr int kSplitWarps"),
           _block(internal, "struct SweepArgs {"),
           "template <int G>",
           _block(walk, "__device__ __forceinline__ double lane_sum_f64(double v)"),
           _block(common, "__device__ __forceinline__ uint32_t bucket_of(float ehh)"),
           "}  // namespace selscan", ""]
    a = sweep.index("namespace selscan {")
    b = sweep.index("template <int G>\nstatic void (*walk_kernel_for(int xpehh))(SweepArgs)")
    body = sweep[a:b]
    # device-only helpers with host equivalents in the preamble
    for sig in ("__device__ __forceinline__ void cp_async8(",
                "__device__ __forceinline__ void cp_async_commit(",
                "template <int N>\n__device__ __forceinline__ void cp_async_wait("):
        i = body.index(sig)
        j = body.index("}\n", i) + 2
        body = body[:i] + body[j:]
    body = re.sub(r'asm\("prmt\.b32 %0, %1, 0, 0xBB99;" : "=r"\(r\) : "r"\(c\)\);',
                  "r = ((c & 0x8000u) ? 0x0000FFFFu : 0u) | ((c & 0x80000000u) ? 0xFFFF0000u : 0u);",
                  body)
    body = body.replace("extern __shared__ __align__(16) unsigned char smem[];",
                        "unsigned char *smem = g_smem;")
    body = body.replace("namespace cg = cooperative_groups;", "namespace cg = ::cooperative_groups;")
    if "asm(" in body or "asm volatile" in body:
        raise ValueError("device-only inline assembly left in the kernel source")
    open(out_path, "w").write("\n".join(pre) + body + "\n}  // namespace selscan\n")
    return out_path


if __name__ == "__main__":
    import sys
    print(build(sys.argv[1]))
