// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
// as easy as 1, 2, 3", SC'11), usable from host and device code of the library.
//
// Ten rounds; each round multiplies counter words 0 and 2 by the Philox constants, mixes the
// high halves with words 1 and 3 and the key, and the key advances by the Weyl increments
// between rounds. A 53-bit uniform takes all 32 bits of output word 0 and the top 21 bits of
// word 1.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define PTSBE_HD __host__ __device__ __forceinline__
#else
#define PTSBE_HD inline
#endif

namespace ptsbe {

struct Philox4 { uint32_t x[4]; };

PTSBE_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

PTSBE_HD Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hiA = mulhi32(kMulA, c0), loA = kMulA * c0;
        const uint32_t hiB = mulhi32(kMulB, c2), loB = kMulB * c2;
        const uint32_t n0 = hiB ^ c1 ^ k0, n2 = hiA ^ c3 ^ k1;
        c0 = n0; c1 = loB; c2 = n2; c3 = loA;
        k0 += kWeylA; k1 += kWeylB;
    }
    Philox4 o;
    o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
    return o;
}

// Raw 53-bit integer of a uniform draw (the uniform is this value times 2^-53).
PTSBE_HD uint64_t u53_bits(uint32_t x0, uint32_t x1) { return ((uint64_t)x0 << 21) | (uint64_t)(x1 >> 11); }

PTSBE_HD double u53(uint32_t x0, uint32_t x1) { return (double)u53_bits(x0, x1) * (1.0 / 9007199254740992.0); }

PTSBE_HD double uniform53(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
    const Philox4 o = philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    return u53(o.x[0], o.x[1]);
}

// Counter domains (low byte of counter word 3).
enum : uint32_t { kDomPts = 1, kDomShot = 2, kDomPershotKraus = 3, kDomLiteral = 4, kDomPershotRead = 5 };

}  // namespace ptsbe
