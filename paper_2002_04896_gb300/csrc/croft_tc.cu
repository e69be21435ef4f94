// croft_tc.cu - instantiations of the tensor-core pass kernel and the DFT-16 operand.
#include <math.h>
#include <string.h>

#include "croft_tc_kernel.cuh"

namespace croft {

pass_fn tc_pass_kernel_for(int layout, int n) {
    switch (n) {
        case 256: return layout == LAYOUT_ROW ? croft_pass_kernel_tc<LAYOUT_ROW, 256> : croft_pass_kernel_tc<LAYOUT_COL, 256>;
        case 512: return layout == LAYOUT_ROW ? croft_pass_kernel_tc<LAYOUT_ROW, 512> : croft_pass_kernel_tc<LAYOUT_COL, 512>;
        default: return nullptr;
    }
}

static unsigned short bf16_bits_rn(float x) {
    unsigned int u;
    memcpy(&u, &x, 4);
    const unsigned int lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;  // round to nearest even (inputs are finite)
    return (unsigned short)(u >> 16);
}

static float bf16_value(unsigned short b) {
    unsigned int u = (unsigned int)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// B operand of the radix-16 GEMM, B[n][k] (n = output, k = input; re parts then im parts):
//   n < 16 : B[n][j] = C[n][j],  B[n][16+j] = -S[n][j]
//   n >= 16: B[n][j] = S[n-16][j], B[n][16+j] = C[n-16][j]
// with C + iS = exp(-2 pi i n j / 16), evaluated in float64 with (n j) mod 16 reduced
// in integers; split into bf16 hi = rn(B) and lo = rn(B - hi).  Layout: K-major,
// no-swizzle core matrices (tc_cm_offset), hi in bytes [0, 2048), lo in [2048, 4096).
void tc_dft16_matrix(unsigned char* out) {
    memset(out, 0, 4096);
    for (int n = 0; n < 32; ++n)
        for (int k = 0; k < 32; ++k) {
            const int on = n & 15, ik = k & 15;
            const int r = (on * ik) % 16;
            const double ang = 2.0 * M_PI * (double)r / 16.0;
            const double C = (r % 4 == 0) ? (r == 0 ? 1.0 : (r == 8 ? -1.0 : 0.0)) : cos(ang);
            const double Sv = (r % 4 == 0) ? (r == 4 ? -1.0 : (r == 12 ? 1.0 : 0.0)) : -sin(ang);
            double v;
            if (n < 16) v = (k < 16) ? C : -Sv;
            else v = (k < 16) ? Sv : C;
            const unsigned short hi = bf16_bits_rn((float)v);
            const unsigned short lo = bf16_bits_rn((float)(v - (double)bf16_value(hi)));
            const int off = tc_cm_offset(n, k);
            memcpy(out + off, &hi, 2);
            memcpy(out + 2048 + off, &lo, 2);
        }
}

}  // namespace croft
