// Host build of the emulated-FP64 digit planes (emu_digits.cuh): reads records of one FP64
// value and one int32 group exponent E from stdin (raw little-endian; E = 99999 asks for the
// value's own exponent), and writes per record the exponent used (int32) and the eight
// planes d_p 2^(-8p) widened to FP32 (raw floats).  Built and run by test_emu_digits_host.py;
// no GPU is involved.
#include <cstdio>

#include "../paper_2205_08941_gb300/csrc/emu_digits.cuh"

int main()
{
    double x;
    int E;
    while (std::fread(&x, sizeof x, 1, stdin) == 1 && std::fread(&E, sizeof E, 1, stdin) == 1) {
        if (E == 99999) E = emu_exponent(x);
        __nv_bfloat16 d[EMU_P];
        emu_digits(x, E, d);
        float f[EMU_P];
        for (int p = 0; p < EMU_P; ++p) f[p] = __bfloat162float(d[p]);
        if (std::fwrite(&E, sizeof E, 1, stdout) != 1) return 1;
        if (std::fwrite(f, sizeof f[0], EMU_P, stdout) != (size_t)EMU_P) return 1;
    }
    return 0;
}
