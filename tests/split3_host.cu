// Host build of the split-BF16 operand split (split3.cuh): reads FP64 values from stdin
// (raw little-endian doubles) and writes, per value, its three BF16 terms widened to FP32
// (raw floats) to stdout.  Built and run by test_split3_host.py; no GPU is involved.
#include <cstdio>

#include "../paper_2205_08941_gb300/csrc/split3.cuh"

int main()
{
    double x;
    while (std::fread(&x, sizeof x, 1, stdin) == 1) {
        __nv_bfloat16 b0, b1, b2;
        split3(x, b0, b1, b2);
        const float f[3] = {__bfloat162float(b0), __bfloat162float(b1), __bfloat162float(b2)};
        if (std::fwrite(f, sizeof f[0], 3, stdout) != 3) return 1;
    }
    return 0;
}
