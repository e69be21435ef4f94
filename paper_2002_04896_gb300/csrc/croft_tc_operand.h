// croft_tc_operand.h - the B operand of the tensor-core radix-16 stage (host code, plain C++:
// compiled into the library and, by a CPU test, with the host compiler).
//
// Round-to-nearest-even conversions of float64 values to bfloat16 and IEEE binary16 bits,
// written from the formats' definitions, and the 32 x 32 real form of the 16-point DFT matrix
// split into hi + lo halves in the tensor-core layout.
#pragma once
#include <math.h>
#include <string.h>

// Byte offset of element (row r, k) of a K = 32, 16-bit, K-major operand in the no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix; core matrices adjacent in K are 128 B
// apart, 8-row groups 512 B apart).
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int tc_cm_offset(int r, int k) {
    return (r / 8) * 512 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2;
}

// Nearest value (ties to even) to a finite v with a p-bit significand and smallest normal
// exponent emin (below it the spacing stays 2^(emin - p + 1): subnormals).  One rounding of
// the float64 value, no intermediate format.
static inline double tc_round_format(double v, int p, int emin) {
    if (v == 0.0) return v;  // keeps the sign of zero
    int e = 0;
    frexp(fabs(v), &e);  // |v| = f * 2^e, f in [0.5, 1): the leading bit has weight 2^(e-1)
    int ex = e - 1;
    if (ex < emin) ex = emin;
    const double ulp = ldexp(1.0, ex - (p - 1));
    return nearbyint(v / ulp) * ulp;  // exact scaling by a power of two; ties to even
}

// bfloat16 bits of a finite value (8-bit significand, float32's exponent range).
static inline unsigned short bf16_bits_rn(double v) {
    const float f = (float)tc_round_format(v, 8, -126);  // exact: the rounded value is a float
    unsigned int u;
    memcpy(&u, &f, 4);
    return (unsigned short)(u >> 16);
}
static inline double bf16_value(unsigned short b) {
    const unsigned int u = (unsigned int)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

// IEEE binary16 bits of a finite |v| < 65504 (11-bit significand, normal exponents -14..15).
static inline unsigned short f16_bits_rn(double v) {
    const double r = tc_round_format(v, 11, -14);
    const unsigned short sign = (r < 0 || (r == 0 && signbit(v))) ? 0x8000 : 0;
    const double a = fabs(r);
    if (a == 0.0) return sign;
    int e = 0;
    frexp(a, &e);
    const int ex = e - 1;
    if (ex < -14) return (unsigned short)(sign | (unsigned)(a / ldexp(1.0, -24)));  // subnormal
    const unsigned m = (unsigned)(a / ldexp(1.0, ex - 10)) - 1024u;                  // stored fraction
    return (unsigned short)(sign | ((unsigned)(ex + 15) << 10) | m);
}
static inline double f16_value(unsigned short b) {
    const int ex = (b >> 10) & 0x1f, m = b & 0x3ff;
    const double mag = ex == 0 ? ldexp((double)m, -24) : ldexp((double)(1024 + m), ex - 25);
    return (b & 0x8000) ? -mag : mag;
}

// B operand of the radix-16 GEMM, B[n][k] (n = output, k = input; re parts then im parts):
//   n < 16 : B[n][j] = C[n][j],  B[n][16+j] = -S[n][j]
//   n >= 16: B[n][j] = S[n-16][j], B[n][16+j] = C[n-16][j]
// with C + iS = exp(-2 pi i n j / 16), evaluated in float64 with (n j) mod 16 reduced
// in integers; split into hi = rn(B) and lo = rn(B - hi) in the operand precision (bf16 or
// fp16).  Layout: K-major, no-swizzle core matrices (tc_cm_offset), hi in bytes [0, 2048),
// lo in [2048, 4096).
static inline void tc_dft16_operand(unsigned char* out, bool fp16) {
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
            unsigned short hi, lo;
            if (fp16) {
                hi = f16_bits_rn(v);
                lo = f16_bits_rn(v - f16_value(hi));
            } else {
                hi = bf16_bits_rn(v);
                lo = bf16_bits_rn(v - bf16_value(hi));
            }
            const int off = tc_cm_offset(n, k);
            memcpy(out + off, &hi, 2);
            memcpy(out + 2048 + off, &lo, 2);
        }
}

