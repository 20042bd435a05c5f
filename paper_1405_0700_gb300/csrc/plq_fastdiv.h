// Division of non-negative 32-bit integers by a run-time invariant divisor
// through a multiply-high and a shift (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, the round-up method).
//
// For a divisor d >= 1 let s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d)
// + 1, which fits in 32 bits because 2^s - d < d.  Then for every n with
// 0 <= n < 2^31
//     n / d = (mulhi(n, m) + n) >> s,
// where mulhi is the high 32 bits of the 64-bit product; the sum cannot
// overflow because mulhi(n, m) < n < 2^31.  The lattice kernels divide
// checkerboard site indices (< 2^30) by the lattice extents, so every use is
// inside that range.
//
// The header is plain C++ (usable by host compilers and nvcc alike).
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define PLQ_HD __host__ __device__ __forceinline__
#else
#define PLQ_HD inline
#endif

namespace plq {

struct FastDiv {
    uint32_t d = 1;  // divisor
    uint32_t m = 0;  // magic multiplier
    uint32_t s = 0;  // shift
};

inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d ? d : 1;
    uint32_t s = 0;
    while (s < 31 && (1u << s) < f.d) ++s;
    f.s = s;
    const uint64_t two_s = 1ull << s;
    f.m = (uint32_t)(((two_s - f.d) << 32) / f.d + 1ull);
    return f;
}

PLQ_HD uint32_t fd_mulhi(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

// n / f.d for 0 <= n < 2^31
PLQ_HD uint32_t fd_div(uint32_t n, const FastDiv &f) { return (fd_mulhi(n, f.m) + n) >> f.s; }

// quotient and remainder of n by f.d
PLQ_HD uint32_t fd_divmod(uint32_t n, const FastDiv &f, uint32_t *rem) {
    const uint32_t q = fd_div(n, f);
    *rem = n - q * f.d;
    return q;
}

}  // namespace plq
