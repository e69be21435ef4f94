// croft_butterflies.cuh - in-register radix-R DFT butterflies (forward sign).
//
// dft<R>(v) overwrites v[0..R-1] with y[k] = sum_j v[j] exp(-2 pi i j k / R),
// output in natural order.  These are the serial 1D FFT building blocks that
// replace the FFTW codelets of the paper (Sec. 4, Sec. 5).  The backward
// transform reuses them through conj(F(conj(x))), applied at the global load
// and store of each pass.
//
// Radix 8, 9, 15 and 16 are split Cooley-Tukey (2x4, 3x3, 5x3 and 4x4) with the
// inner twiddles as compile-time constants; 3 and 5 use the symmetric cos/sin form.  The
// constants are the exact mathematical values rounded to the working precision
// (float for complex64, double for complex128).
#pragma once
#include <cuda_runtime.h>

namespace croft {

// Complex helpers for float2 (complex64) and double2 (complex128).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

template <class C> struct CxScalar;
template <> struct CxScalar<float2> { using T = float; };
template <> struct CxScalar<double2> { using T = double; };

template <class C> __device__ __forceinline__ C mkc(typename CxScalar<C>::T re, typename CxScalar<C>::T im) {
    C c;
    c.x = re;
    c.y = im;
    return c;
}
// a * (-i)
template <class C> __device__ __forceinline__ C mul_mi(C a) { return mkc<C>(a.y, -a.x); }
// a * (c + i s) for constants
template <class C>
__device__ __forceinline__ C mul_cs(C a, typename CxScalar<C>::T c, typename CxScalar<C>::T s) {
    return mkc<C>(fma(a.x, c, -a.y * s), fma(a.x, s, a.y * c));
}

// cos(pi/8), sin(pi/8), sqrt(2)/2, sqrt(3)/2, cos(2pi/5), cos(4pi/5), sin(2pi/5), sin(4pi/5):
// the exact values, rounded to the working precision.
#define CROFT_C8 0.92387953251128675613
#define CROFT_S8 0.38268343236508977173
#define CROFT_R2 0.70710678118654752440
#define CROFT_R3 0.86602540378443864676
#define CROFT_C51 0.30901699437494742410
#define CROFT_C52 (-0.80901699437494742410)
#define CROFT_S51 0.95105651629515357212
#define CROFT_S52 0.58778525229247312917
// cos and sin of 2 pi m / 9 (m = 1, 2, 4) and of 2 pi m / 15 (m = 1, 2, 4, 8; m = 3 and
// 6 are the radix-5 constants above), exact values rounded to the working precision.
#define CROFT_C9_1 0.7660444431189780352024
#define CROFT_S9_1 0.6427876096865393263226
#define CROFT_C9_2 0.1736481776669303488517
#define CROFT_S9_2 0.9848077530122080593667
#define CROFT_C9_4 (-0.9396926207859083840541)
#define CROFT_S9_4 0.3420201433256687330441
#define CROFT_C15_1 0.9135454576426008955021
#define CROFT_S15_1 0.4067366430758002077540
#define CROFT_C15_2 0.6691306063588582138263
#define CROFT_S15_2 0.7431448254773942350147
#define CROFT_C15_4 (-0.1045284632676534713998)
#define CROFT_S15_4 0.9945218953682733369227
#define CROFT_C15_8 (-0.9781476007338056379286)
#define CROFT_S15_8 (-0.2079116908177593371017)

template <int R, class C> __device__ __forceinline__ void dft(C* v);

template <class C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
    C a = cadd(x0, x2), b = csub(x0, x2);
    C c = cadd(x1, x3), d = mul_mi(csub(x1, x3));
    x0 = cadd(a, c);
    x2 = csub(a, c);
    x1 = cadd(b, d);
    x3 = csub(b, d);
}

template <int R, class C> struct Dft;

template <class C> struct Dft<2, C> {
    __device__ __forceinline__ static void run(C* v) {
        C t = v[0];
        v[0] = cadd(t, v[1]);
        v[1] = csub(t, v[1]);
    }
};

template <class C> struct Dft<4, C> {
    __device__ __forceinline__ static void run(C* v) { dft4(v[0], v[1], v[2], v[3]); }
};

template <class C> struct Dft<8, C> {
    __device__ __forceinline__ static void run(C* v) {
        using T = typename CxScalar<C>::T;
        const T r2 = (T)CROFT_R2;
        // j = 4*j1 + j2: length-2 DFTs over j1, twiddle W8^(j2*k1), length-4 DFTs over j2.
        C a0[4], a1[4];
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) {
            a0[j2] = cadd(v[j2], v[4 + j2]);
            a1[j2] = csub(v[j2], v[4 + j2]);
        }
        a1[1] = mul_cs(a1[1], r2, -r2);   // W8^1
        a1[2] = mul_mi(a1[2]);            // W8^2 = -i
        a1[3] = mul_cs(a1[3], -r2, -r2);  // W8^3
        dft4(a0[0], a0[1], a0[2], a0[3]);
        dft4(a1[0], a1[1], a1[2], a1[3]);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            v[2 * k2] = a0[k2];
            v[2 * k2 + 1] = a1[k2];
        }
    }
};

template <class C> struct Dft<16, C> {
    __device__ __forceinline__ static void run(C* v) {
        using T = typename CxScalar<C>::T;
        const T c8 = (T)CROFT_C8, s8 = (T)CROFT_S8, r2 = (T)CROFT_R2;
        // j = 4*j1 + j2: length-4 DFTs over j1, twiddle W16^(j2*k1), length-4 DFTs over j2.
        C a[4][4];  // a[k1][j2]
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) {
            C x0 = v[j2], x1 = v[4 + j2], x2 = v[8 + j2], x3 = v[12 + j2];
            dft4(x0, x1, x2, x3);
            a[0][j2] = x0;
            a[1][j2] = x1;
            a[2][j2] = x2;
            a[3][j2] = x3;
        }
        a[1][1] = mul_cs(a[1][1], c8, -s8);   // W16^1
        a[1][2] = mul_cs(a[1][2], r2, -r2);   // W16^2
        a[1][3] = mul_cs(a[1][3], s8, -c8);   // W16^3
        a[2][1] = mul_cs(a[2][1], r2, -r2);   // W16^2
        a[2][2] = mul_mi(a[2][2]);            // W16^4
        a[2][3] = mul_cs(a[2][3], -r2, -r2);  // W16^6
        a[3][1] = mul_cs(a[3][1], s8, -c8);   // W16^3
        a[3][2] = mul_cs(a[3][2], -r2, -r2);  // W16^6
        a[3][3] = mul_cs(a[3][3], -c8, s8);   // W16^9
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            dft4(a[k1][0], a[k1][1], a[k1][2], a[k1][3]);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = a[k1][k2];
        }
    }
};

template <class C> struct Dft<3, C> {
    __device__ __forceinline__ static void run(C* v) {
        using T = typename CxScalar<C>::T;
        const T r3 = (T)CROFT_R3;
        C t = cadd(v[1], v[2]);
        C d = csub(v[1], v[2]);
        C m = mkc<C>(fma((T)-0.5, t.x, v[0].x), fma((T)-0.5, t.y, v[0].y));
        C r = mkc<C>(r3 * d.y, -r3 * d.x);  // -i * (sqrt3/2) * d
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};

template <class C> struct Dft<5, C> {
    __device__ __forceinline__ static void run(C* v) {
        using T = typename CxScalar<C>::T;
        const T c1 = (T)CROFT_C51, c2 = (T)CROFT_C52, s1 = (T)CROFT_S51, s2 = (T)CROFT_S52;
        C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        C d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
        C x0 = v[0];
        C a1 = mkc<C>(fma(c1, t1.x, fma(c2, t2.x, x0.x)), fma(c1, t1.y, fma(c2, t2.y, x0.y)));
        C a2 = mkc<C>(fma(c2, t1.x, fma(c1, t2.x, x0.x)), fma(c2, t1.y, fma(c1, t2.y, x0.y)));
        C b1 = mkc<C>(fma(s1, d1.x, s2 * d2.x), fma(s1, d1.y, s2 * d2.y));
        C b2 = mkc<C>(fma(s2, d1.x, -s1 * d2.x), fma(s2, d1.y, -s1 * d2.y));
        v[0] = mkc<C>(x0.x + t1.x + t2.x, x0.y + t1.y + t2.y);
        // y1 = a1 - i b1, y4 = a1 + i b1, y2 = a2 - i b2, y3 = a2 + i b2
        v[1] = mkc<C>(a1.x + b1.y, a1.y - b1.x);
        v[4] = mkc<C>(a1.x - b1.y, a1.y + b1.x);
        v[2] = mkc<C>(a2.x + b2.y, a2.y - b2.x);
        v[3] = mkc<C>(a2.x - b2.y, a2.y + b2.x);
    }
};

template <class C> struct Dft<9, C> {
    __device__ __forceinline__ static void run(C* v) {
        using T = typename CxScalar<C>::T;
        // j = 3*j1 + j2: length-3 DFTs over j1, twiddle W9^(j2*k1), length-3 DFTs over j2.
        C a[3][3];  // a[k1][j2]
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2) {
            C t[3] = {v[j2], v[3 + j2], v[6 + j2]};
            Dft<3, C>::run(t);
            a[0][j2] = t[0];
            a[1][j2] = t[1];
            a[2][j2] = t[2];
        }
        a[1][1] = mul_cs(a[1][1], (T)CROFT_C9_1, -(T)CROFT_S9_1);  // W9^1
        a[1][2] = mul_cs(a[1][2], (T)CROFT_C9_2, -(T)CROFT_S9_2);  // W9^2
        a[2][1] = mul_cs(a[2][1], (T)CROFT_C9_2, -(T)CROFT_S9_2);  // W9^2
        a[2][2] = mul_cs(a[2][2], (T)CROFT_C9_4, -(T)CROFT_S9_4);  // W9^4
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            Dft<3, C>::run(a[k1]);
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) v[k1 + 3 * k2] = a[k1][k2];
        }
    }
};

template <class C> struct Dft<15, C> {
    __device__ __forceinline__ static void run(C* v) {
        using T = typename CxScalar<C>::T;
        // j = 3*j1 + j2 (j1 < 5, j2 < 3): length-5 DFTs over j1, twiddle W15^(j2*k1),
        // length-3 DFTs over j2; output k1 + 5*k2.
        C a[5][3];  // a[k1][j2]
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2) {
            C t[5] = {v[j2], v[3 + j2], v[6 + j2], v[9 + j2], v[12 + j2]};
            Dft<5, C>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < 5; ++k1) a[k1][j2] = t[k1];
        }
        a[1][1] = mul_cs(a[1][1], (T)CROFT_C15_1, -(T)CROFT_S15_1);  // W15^1
        a[2][1] = mul_cs(a[2][1], (T)CROFT_C15_2, -(T)CROFT_S15_2);  // W15^2
        a[3][1] = mul_cs(a[3][1], (T)CROFT_C51, -(T)CROFT_S51);      // W15^3 = W5^1
        a[4][1] = mul_cs(a[4][1], (T)CROFT_C15_4, -(T)CROFT_S15_4);  // W15^4
        a[1][2] = mul_cs(a[1][2], (T)CROFT_C15_2, -(T)CROFT_S15_2);  // W15^2
        a[2][2] = mul_cs(a[2][2], (T)CROFT_C15_4, -(T)CROFT_S15_4);  // W15^4
        a[3][2] = mul_cs(a[3][2], (T)CROFT_C52, -(T)CROFT_S52);      // W15^6 = W5^2
        a[4][2] = mul_cs(a[4][2], (T)CROFT_C15_8, -(T)CROFT_S15_8);  // W15^8
#pragma unroll
        for (int k1 = 0; k1 < 5; ++k1) {
            Dft<3, C>::run(a[k1]);
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) v[k1 + 5 * k2] = a[k1][k2];
        }
    }
};

template <int R, class C> __device__ __forceinline__ void dft(C* v) { Dft<R, C>::run(v); }

}  // namespace croft
