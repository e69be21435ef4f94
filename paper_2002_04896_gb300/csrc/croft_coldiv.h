// croft_coldiv.h - the column split col -> (col / M, col % M) of the column passes as a
// multiply-high and two shifts instead of a 64-bit division (which costs a few dozen
// instructions per thread, a few per transformed point at 16 points per thread).
//
// Division by an invariant integer (T. Granlund and P. L. Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994, Sec. 4): for a divisor 1 <= d < 2^32, with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1 (which fits in 32 bits), every
// 32-bit n has
//     floor(n / d) = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0),   t = floor(m n / 2^32).
// Host and device share this header.
#pragma once

#ifdef __CUDACC__
#define CROFT_COLDIV_HD __host__ __device__
#else
#define CROFT_COLDIV_HD
#endif

struct CroftColDiv {
    unsigned m;  // 0: not set up (the divisor or the dividends do not fit in 32 bits)
    unsigned char s1, s2;
};

// The divider of d, for dividends below `limit` (both must fit in 32 bits).
inline CroftColDiv croft_coldiv_make(long long d, long long limit) {
    CroftColDiv v{0, 0, 0};
    if (d < 1 || d > 0xffffffffLL || limit < 0 || limit > 0x100000000LL) return v;
    int l = 0;
    while ((1ULL << l) < (unsigned long long)d) ++l;
    const unsigned long long ud = (unsigned long long)d;
    v.m = (unsigned)((((1ULL << l) - ud) << 32) / ud + 1);
    v.s1 = (unsigned char)(l > 0 ? 1 : 0);
    v.s2 = (unsigned char)(l > 0 ? l - 1 : 0);
    return v;
}

CROFT_COLDIV_HD inline unsigned croft_coldiv_q(unsigned m, unsigned s1, unsigned s2, unsigned n) {
#ifdef __CUDA_ARCH__
    const unsigned t = __umulhi(m, n);
#else
    const unsigned t = (unsigned)(((unsigned long long)m * n) >> 32);
#endif
    return (t + ((n - t) >> s1)) >> s2;
}
