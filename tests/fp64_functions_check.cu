// Host program for tests/test_fp64_functions.py: evaluates the library's
// binary64 erfcx and exp (fabf_device.cuh, host build of the same code and
// tables), or its bit-level binary64 -> binary32 rounding, on the arguments
// read from stdin and prints them as hex floats.
#include <cstdio>
#include <cstring>

#include "../paper_1811_02308_gb300/csrc/fabf_device.cuh"

static const double h_erfcx[] = {FABF_ERFCX_TABLE, FABF_ERFCX_P0_LO};
static const double h_exp[] = {FABF_EXP2_TABLE};

int main()
{
    char kind[8];
    double x;
    while (std::scanf("%7s %la", kind, &x) == 2) {
        if (kind[0] == 'd') {   // "d2f": the bit-level binary64 -> binary32 rounding
            std::printf("%a\n", (double)fabf::double_to_float_rn(x));
            continue;
        }
        const double v = kind[0] == 'e' && kind[1] == 'r' ? fabf::erfcx_fp64_with(x, h_erfcx)
                                                          : fabf::exp_fp64_with(x, h_exp);
        std::printf("%a\n", v);
    }
    return 0;
}
