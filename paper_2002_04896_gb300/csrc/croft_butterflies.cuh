// croft_butterflies.cuh - in-register radix-R DFT butterflies (forward sign).
//
// dft<R>(v) overwrites v[0..R-1] with y[k] = sum_j v[j] exp(-2 pi i j k / R),
// output in natural order.  These are the serial 1D FFT building blocks that
// replace the FFTW codelets of the paper (Sec. 4, Sec. 5).  The backward
// transform reuses them through conj(F(conj(x))), applied at the global load
// and store of each pass.
//
// Radix 8 and 16 are split Cooley-Tukey (2x4 and 4x4) with the inner twiddles
// as compile-time constants; 3 and 5 use the symmetric cos/sin form.  The
// constants are the exact mathematical values rounded to float.
#pragma once
#include <cuda_runtime.h>

namespace croft {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * (-i)
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }
// a * (c + i s) for constants
__device__ __forceinline__ float2 mul_cs(float2 a, float c, float s) {
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
}

// cos(pi/8), sin(pi/8), sqrt(2)/2, sqrt(3)/2
#define CROFT_C8 0.92387953251128675613f
#define CROFT_S8 0.38268343236508977173f
#define CROFT_R2 0.70710678118654752440f
#define CROFT_R3 0.86602540378443864676f
// cos(2pi/5), cos(4pi/5), sin(2pi/5), sin(4pi/5)
#define CROFT_C51 0.30901699437494742410f
#define CROFT_C52 (-0.80901699437494742410f)
#define CROFT_S51 0.95105651629515357212f
#define CROFT_S52 0.58778525229247312917f

template <int R> __device__ __forceinline__ void dft(float2* v);

template <> __device__ __forceinline__ void dft<2>(float2* v) {
    float2 t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
}

__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
    float2 a = cadd(x0, x2), b = csub(x0, x2);
    float2 c = cadd(x1, x3), d = mul_mi(csub(x1, x3));
    x0 = cadd(a, c);
    x2 = csub(a, c);
    x1 = cadd(b, d);
    x3 = csub(b, d);
}

template <> __device__ __forceinline__ void dft<4>(float2* v) { dft4(v[0], v[1], v[2], v[3]); }

template <> __device__ __forceinline__ void dft<8>(float2* v) {
    // j = 4*j1 + j2: length-2 DFTs over j1, twiddle W8^(j2*k1), length-4 DFTs over j2.
    float2 a0[4], a1[4];
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2) {
        a0[j2] = cadd(v[j2], v[4 + j2]);
        a1[j2] = csub(v[j2], v[4 + j2]);
    }
    a1[1] = mul_cs(a1[1], CROFT_R2, -CROFT_R2);   // W8^1
    a1[2] = mul_mi(a1[2]);                        // W8^2 = -i
    a1[3] = mul_cs(a1[3], -CROFT_R2, -CROFT_R2);  // W8^3
    dft4(a0[0], a0[1], a0[2], a0[3]);
    dft4(a1[0], a1[1], a1[2], a1[3]);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
        v[2 * k2] = a0[k2];
        v[2 * k2 + 1] = a1[k2];
    }
}

template <> __device__ __forceinline__ void dft<16>(float2* v) {
    // j = 4*j1 + j2: length-4 DFTs over j1, twiddle W16^(j2*k1), length-4 DFTs over j2.
    float2 a[4][4];  // a[k1][j2]
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2) {
        float2 x0 = v[j2], x1 = v[4 + j2], x2 = v[8 + j2], x3 = v[12 + j2];
        dft4(x0, x1, x2, x3);
        a[0][j2] = x0;
        a[1][j2] = x1;
        a[2][j2] = x2;
        a[3][j2] = x3;
    }
    a[1][1] = mul_cs(a[1][1], CROFT_C8, -CROFT_S8);    // W16^1
    a[1][2] = mul_cs(a[1][2], CROFT_R2, -CROFT_R2);    // W16^2
    a[1][3] = mul_cs(a[1][3], CROFT_S8, -CROFT_C8);    // W16^3
    a[2][1] = mul_cs(a[2][1], CROFT_R2, -CROFT_R2);    // W16^2
    a[2][2] = mul_mi(a[2][2]);                         // W16^4
    a[2][3] = mul_cs(a[2][3], -CROFT_R2, -CROFT_R2);   // W16^6
    a[3][1] = mul_cs(a[3][1], CROFT_S8, -CROFT_C8);    // W16^3
    a[3][2] = mul_cs(a[3][2], -CROFT_R2, -CROFT_R2);   // W16^6
    a[3][3] = mul_cs(a[3][3], -CROFT_C8, CROFT_S8);    // W16^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        dft4(a[k1][0], a[k1][1], a[k1][2], a[k1][3]);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = a[k1][k2];
    }
}

template <> __device__ __forceinline__ void dft<3>(float2* v) {
    float2 t = cadd(v[1], v[2]);
    float2 d = csub(v[1], v[2]);
    float2 m = make_float2(fmaf(-0.5f, t.x, v[0].x), fmaf(-0.5f, t.y, v[0].y));
    // -i * (sqrt3/2) * d
    float2 r = make_float2(CROFT_R3 * d.y, -CROFT_R3 * d.x);
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
}

template <> __device__ __forceinline__ void dft<5>(float2* v) {
    float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    float2 x0 = v[0];
    float2 a1 = make_float2(fmaf(CROFT_C51, t1.x, fmaf(CROFT_C52, t2.x, x0.x)),
                            fmaf(CROFT_C51, t1.y, fmaf(CROFT_C52, t2.y, x0.y)));
    float2 a2 = make_float2(fmaf(CROFT_C52, t1.x, fmaf(CROFT_C51, t2.x, x0.x)),
                            fmaf(CROFT_C52, t1.y, fmaf(CROFT_C51, t2.y, x0.y)));
    float2 b1 = make_float2(fmaf(CROFT_S51, d1.x, CROFT_S52 * d2.x), fmaf(CROFT_S51, d1.y, CROFT_S52 * d2.y));
    float2 b2 = make_float2(fmaf(CROFT_S52, d1.x, -CROFT_S51 * d2.x), fmaf(CROFT_S52, d1.y, -CROFT_S51 * d2.y));
    v[0] = make_float2(x0.x + t1.x + t2.x, x0.y + t1.y + t2.y);
    // y1 = a1 - i b1, y4 = a1 + i b1, y2 = a2 - i b2, y3 = a2 + i b2
    v[1] = make_float2(a1.x + b1.y, a1.y - b1.x);
    v[4] = make_float2(a1.x - b1.y, a1.y + b1.x);
    v[2] = make_float2(a2.x + b2.y, a2.y - b2.x);
    v[3] = make_float2(a2.x - b2.y, a2.y + b2.x);
}

}  // namespace croft
