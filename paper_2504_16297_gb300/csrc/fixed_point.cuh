// Outcome probabilities in 2^-62 fixed point, shared by every shot sampler of the library (the
// stand-alone samplers and the sampling fused into the last evolve stage), so that all of them
// draw the same outcome for the same state, seed and shot index.
//
// P = |psi_i|^2 (an FP32 product) becomes floor(P * 2^62) as an unsigned 64-bit integer: prefix
// sums are exact integer additions (no rounding, the same result in any summation order) on the
// integer pipe (the FP64 pipe runs at 1/64 of the FP32 rate on GB300); the resolution (2.2e-19
// absolute) is finer than an FP64 running sum near C = 1 (1.1e-16). A state's total must stay
// below 4 (normalised states: 1).
//
// Shot j of a state with inclusive prefix C and total T draws the 53-bit integer m of a Philox
// uniform u = m / 2^53 and returns the smallest i with floor(u T) < C[i]; floor(u T) =
// floor(m T / 2^53) is computed exactly.
#pragma once
#include <cstdint>

namespace ptsbe {

using fx = unsigned long long;
constexpr int kFxBits = 62;

__device__ __forceinline__ fx fx_of(float p) {          // p >= 0 finite; P >= 2 saturates at 2^63
    const uint32_t u = __float_as_uint(p);
    const uint32_t e = u >> 23;
    const fx m = e ? (fx)((u & 0x7FFFFFu) | 0x800000u) : (fx)(u & 0x7FFFFFu);
    const int sh = (int)(e ? e : 1u) - 150 + kFxBits;    // P = m 2^(e - 150)
    if (sh >= 0) return sh > 39 ? (fx)1 << 63 : m << sh;
    return sh <= -24 ? 0ull : m >> (-sh);
}
__device__ __forceinline__ fx fx_prob(float2 a) { return fx_of(fmaf(a.x, a.x, a.y * a.y)); }

// floor(u T) for the uniform u = m / 2^53 (m its 53-bit integer): exact.
__device__ __forceinline__ fx fx_target(uint64_t m53, fx T) { return __umul64hi(m53 << 11, T); }

}  // namespace ptsbe
