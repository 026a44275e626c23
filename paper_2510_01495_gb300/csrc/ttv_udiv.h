// ttv_udiv.h -- exact unsigned 64-bit division by an invariant divisor with
// one multiply-high (T. Granlund and P. Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994, unsigned algorithm of Fig. 4.1):
//   l = ceil(log2 d),  m' = floor(2^64 (2^l - d) / d) + 1,
//   sh1 = min(l, 1),   sh2 = max(l - 1, 0),
//   q = (t + ((n - t) >> sh1)) >> sh2   with t = mulhi(m', n).
// Used to turn linear keys back into subscripts without 64-bit divides.
// Plain C++ (host and device), so the host test can check it exhaustively.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define TTV_HD __host__ __device__ __forceinline__
#else
#define TTV_HD inline
#endif

inline void udiv_magic(uint64_t d, uint64_t& magic, uint32_t& shifts) {
    int l = 0;
    while (l < 64 && ((unsigned __int128)1 << l) < d) ++l;
    const unsigned __int128 two64 = (unsigned __int128)1 << 64;
    const unsigned __int128 num = two64 * ((((unsigned __int128)1) << l) - d);
    magic = (uint64_t)(num / d + 1);
    const uint32_t sh1 = l < 1 ? (uint32_t)l : 1u;
    const uint32_t sh2 = l >= 1 ? (uint32_t)(l - 1) : 0u;
    shifts = sh1 | (sh2 << 8);
}

TTV_HD uint64_t udiv_mulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

TTV_HD uint64_t udiv_invariant(uint64_t n, uint64_t magic, uint32_t shifts) {
    const uint64_t t = udiv_mulhi(magic, n);
    return (t + ((n - t) >> (shifts & 0xFF))) >> (shifts >> 8);
}
