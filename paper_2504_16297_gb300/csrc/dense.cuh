// Dense tile passes for large states (Sec. 3, batched execution: one O(2^n) preparation per Kraus
// set, the dominant cost of PTSBE). Shared by the CUDA kernel (dense.cu), the host planner
// (dense_plan.cpp) and the CPU harness of the tests, which runs the same per-thread code.
//
// A pass streams a state through HBM once: the 2^n amplitudes are cut into 2^(n-T) tiles of 2^T
// amplitudes (T = kT tile bits); the tile bits are a set of physical index bits that always
// contains the kC lowest ones, so a tile is made of contiguous 2^kC-amplitude (128-byte) runs.
// Inside the tile, the pass applies every operator of its part of the circuit -- gates, and at each
// noise site the Kraus operator the set selects -- fused into 1- and 2-qubit blocks. The blocks
// run in register groups: each of the 2^(T-kR) threads holds 2^kR amplitudes whose tile index
// varies in the group's kR register bits, applies the group's blocks in registers and hands the
// tile on through shared memory (XOR-swizzled so that a warp's accesses spread over the banks).
// Between passes the logical-to-physical qubit map may change: a pass writes its tile bits back
// in another order, which is how qubits that the next pass needs reach the low bits.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#ifdef __CUDACC__
#define PTSBE_HD __host__ __device__ __forceinline__
#else
#define PTSBE_HD inline
#endif

namespace ptsbe {
namespace dense {

constexpr int kT = 12;                          // tile bits: 2^12 complex64 = 32 KiB of shared memory
constexpr int kC = 4;                           // contiguous low bits of every tile (16 amplitudes)
constexpr int kR = 4;                           // register bits per thread (16 amplitudes)
constexpr int kTB = kT - kR;                    // thread-index bits
constexpr int kThreads = 1 << kTB;              // 256 threads per CTA
constexpr int kAmps = 1 << kR;                  // amplitudes per thread
constexpr int kCodes1 = kR;                     // block codes 0 .. kR-1: 2x2 on one register bit
constexpr int kCodeDR = 10;                     // offset of the diagonal-times-real variant of a code
constexpr int kStageMax = 24 * 1024;            // shared memory for a pass's groups, blocks and matrices
                                                // (the planner keeps every pass within it)
constexpr int kHi = 1 << (kT - kC);             // entries of a pass's high-offset table
constexpr int kMaxQ = 32;

// One fused operator of a pass. code 0..3: 2x2 on register bit `code`; code 4..9: 4x4 on the
// register pair number code - 4 = (lo, hi) of (0,1) (0,2) (0,3) (1,2) (1,3) (2,3), local index
// bit(lo) + 2 bit(hi). Codes kCodeDR + 0..9: the same operator in diagonal-times-real form, M = R D
// with D diagonal (its entry 0 is 1) and R real: the amplitudes are multiplied by D, then by R
// (matrix layout: D entries 1.. as float2, padded to an even count, then R row-major as floats).
struct Block {
    uint8_t code;
    uint8_t pad[3];
    uint32_t mat;                               // default matrix: float2 pool offset (4 or 16 entries)
    uint32_t id;                                // plan-wide index, increasing in execution order
};

// Consecutive blocks of a pass that act on the same kR tile bits. Thread t holds the amplitudes at
// tile addresses base(t) ^ roff[j], j = 0 .. 15, with base(t) the XOR of toff[k] over the set bits k
// of t; both tables hold swizzled addresses (the swizzle is linear over GF(2)).
struct Group {
    uint16_t toff[kTB];
    uint16_t roff[kAmps];
    uint32_t blk_begin, blk_end;                // blocks (indices into the plan's block array)
};

// One pass. Tile bit i is physical index bit pos[i] (pos ascending, pos[i] = i for i < kC) on the
// way in; on the way out the tile is written in another order: the amplitude at output-local index
// L (whose bit j is physical bit pos[j] again) comes from tile address omap[L >> kC] ^ olow[L & 15].
struct Pass {
    uint32_t group_begin, group_end;
    uint32_t blk_begin, blk_end;                // plan-wide block ids of this pass
    uint32_t hi_off;                            // hi pool: kHi amplitude offsets of tile bits [kC, kT)
    uint32_t omap_off;                          // omap pool: kHi tile addresses
    uint16_t olow[1 << kC];
    uint8_t opos[kMaxQ];                        // outer bit k -> physical position (ascending)
    uint32_t nouter;
    uint32_t nops;                              // circuit operations this pass applies
    uint32_t mat_begin, mat_end;                // the pass's default matrices (float2 pool range)
    uint32_t stage_bytes;                       // groups + blocks + matrices staged in shared memory
};

// A (set, pass) launch entry: where the tile comes from and goes to, and the set's override blocks.
struct Node {
    const float2* src;                          // nullptr: the state starts from |0...0> in this pass
    float2* dst;
    uint32_t ov_begin, ov_end;                  // overrides (sorted by block id) of this set
    uint32_t part;                              // row of the norm partials (last pass)
    uint32_t pad;
};

struct Override {
    uint32_t block;                             // plan-wide block id
    uint32_t mat;                               // float2 offset into the override pool (4 or 16 entries)
    uint32_t code;                              // its block code (a general 2x2 or 4x4)
};


// Shared-memory staging of a pass (groups, then blocks, then default matrices, each 16-byte aligned).
PTSBE_HD uint32_t dense_align16(uint32_t x) { return (x + 15u) & ~15u; }
PTSBE_HD uint32_t dense_stage_blocks_off(const Pass& p) { return dense_align16((p.group_end - p.group_begin) * (uint32_t)sizeof(Group)); }
PTSBE_HD uint32_t dense_stage_mats_off(const Pass& p) {
    return dense_stage_blocks_off(p) + dense_align16((p.blk_end - p.blk_begin) * (uint32_t)sizeof(Block));
}
PTSBE_HD uint32_t dense_stage_bytes(const Pass& p) {
    return dense_stage_mats_off(p) + (p.mat_end - p.mat_begin) * (uint32_t)sizeof(float2);
}

// XOR swizzle of a tile address (kT = 12): the float2 bank pair of address t is bits 0..3 of the
// result, and tile bit p contributes unit vector p mod 4 to them.
PTSBE_HD uint32_t swz(uint32_t t) { return t ^ ((t >> 4) & 15u) ^ ((t >> 8) & 15u); }

// Block matrices come from shared memory (a staged pass) or from global memory (override blocks,
// unstaged passes): a plain generic load serves both (the read-only global path must not be used
// on a shared-memory address).
PTSBE_HD float4 ldm(const float2* p) { return *reinterpret_cast<const float4*>(p); }

// out = a * x + b * y (complex)
PTSBE_HD float2 cmac2(float2 a, float2 x, float2 b, float2 y) {
    float2 r;
    r.x = a.x * x.x - a.y * x.y + b.x * y.x - b.y * y.y;
    r.y = a.x * x.y + a.y * x.x + b.x * y.y + b.y * y.x;
    return r;
}

// 2x2 matrix m (row-major, 4 float2, 16-byte aligned) on register bit A of v[16].
template <int A>
PTSBE_HD void apply1(float2* v, const float2* m) {
    const float4 r0 = ldm(m), r1 = ldm(m + 2);
    const float2 m00 = make_float2(r0.x, r0.y), m01 = make_float2(r0.z, r0.w);
    const float2 m10 = make_float2(r1.x, r1.y), m11 = make_float2(r1.z, r1.w);
#pragma unroll
    for (int j = 0; j < kAmps; ++j) {
        if (j & (1 << A)) continue;
        const float2 x = v[j], y = v[j | (1 << A)];
        v[j] = cmac2(m00, x, m01, y);
        v[j | (1 << A)] = cmac2(m10, x, m11, y);
    }
}

// 4x4 matrix m (row-major, 16 float2) on register bits (L, H), local index bit(L) + 2 bit(H).
template <int L, int H>
PTSBE_HD void apply2(float2* v, const float2* m) {
    float2 M[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 r = ldm(m + 2 * i);
        M[2 * i] = make_float2(r.x, r.y);
        M[2 * i + 1] = make_float2(r.z, r.w);
    }
#pragma unroll
    for (int j = 0; j < kAmps; ++j) {
        if (j & ((1 << L) | (1 << H))) continue;
        const int i1 = j | (1 << L), i2 = j | (1 << H), i3 = j | (1 << L) | (1 << H);
        const float2 x[4] = {v[j], v[i1], v[i2], v[i3]};
        float2 o[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            // one multiply-add chain per component: 16 operations per output
            float re = M[4 * r].x * x[0].x, im = M[4 * r].x * x[0].y;
            re -= M[4 * r].y * x[0].y;
            im += M[4 * r].y * x[0].x;
#pragma unroll
            for (int l = 1; l < 4; ++l) {
                re += M[4 * r + l].x * x[l].x;
                im += M[4 * r + l].x * x[l].y;
                re -= M[4 * r + l].y * x[l].y;
                im += M[4 * r + l].y * x[l].x;
            }
            o[r] = make_float2(re, im);
        }
        v[j] = o[0]; v[i1] = o[1]; v[i2] = o[2]; v[i3] = o[3];
    }
}

PTSBE_HD float2 cmul(float2 a, float2 d) {
    float2 r;
    r.x = a.x * d.x - a.y * d.y;
    r.y = a.x * d.y + a.y * d.x;
    return r;
}

// Diagonal-times-real 2x2 on register bit A: amplitude 1 of each pair times d1, then R.
template <int A>
PTSBE_HD void apply1dr(float2* v, const float2* m) {
    const float4 a = ldm(m), r = ldm(m + 2);
    const float2 d1 = make_float2(a.x, a.y);
#pragma unroll
    for (int j = 0; j < kAmps; ++j) {
        if (j & (1 << A)) continue;
        const float2 x = v[j], y = cmul(v[j | (1 << A)], d1);
        v[j] = make_float2(r.x * x.x + r.y * y.x, r.x * x.y + r.y * y.y);
        v[j | (1 << A)] = make_float2(r.z * x.x + r.w * y.x, r.z * x.y + r.w * y.y);
    }
}

// Diagonal-times-real 4x4 on register bits (L, H): amplitudes 1, 2, 3 of each quad times d1, d2, d3,
// then the real matrix R (12 multiply-adds of the diagonal and 32 of R per quad, against 64).
template <int L, int H>
PTSBE_HD void apply2dr(float2* v, const float2* m) {
    const float4 a = ldm(m), b = ldm(m + 2);
    const float2 d1 = make_float2(a.x, a.y), d2 = make_float2(a.z, a.w), d3 = make_float2(b.x, b.y);
    float R[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 r = ldm(m + 4 + 2 * i);
        R[4 * i] = r.x; R[4 * i + 1] = r.y; R[4 * i + 2] = r.z; R[4 * i + 3] = r.w;
    }
#pragma unroll
    for (int j = 0; j < kAmps; ++j) {
        if (j & ((1 << L) | (1 << H))) continue;
        const int i1 = j | (1 << L), i2 = j | (1 << H), i3 = j | (1 << L) | (1 << H);
        const float2 x[4] = {v[j], cmul(v[i1], d1), cmul(v[i2], d2), cmul(v[i3], d3)};
        float2 o[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float re = R[4 * r] * x[0].x, im = R[4 * r] * x[0].y;
#pragma unroll
            for (int l = 1; l < 4; ++l) {
                re += R[4 * r + l] * x[l].x;
                im += R[4 * r + l] * x[l].y;
            }
            o[r] = make_float2(re, im);
        }
        v[j] = o[0]; v[i1] = o[1]; v[i2] = o[2]; v[i3] = o[3];
    }
}

PTSBE_HD void apply_block(float2* v, int code, const float2* m) {
    switch (code) {
    case 0: apply1<0>(v, m); break;
    case 1: apply1<1>(v, m); break;
    case 2: apply1<2>(v, m); break;
    case 3: apply1<3>(v, m); break;
    case 4: apply2<0, 1>(v, m); break;
    case 5: apply2<0, 2>(v, m); break;
    case 6: apply2<0, 3>(v, m); break;
    case 7: apply2<1, 2>(v, m); break;
    case 8: apply2<1, 3>(v, m); break;
    case 9: apply2<2, 3>(v, m); break;
    case kCodeDR + 0: apply1dr<0>(v, m); break;
    case kCodeDR + 1: apply1dr<1>(v, m); break;
    case kCodeDR + 2: apply1dr<2>(v, m); break;
    case kCodeDR + 3: apply1dr<3>(v, m); break;
    case kCodeDR + 4: apply2dr<0, 1>(v, m); break;
    case kCodeDR + 5: apply2dr<0, 2>(v, m); break;
    case kCodeDR + 6: apply2dr<0, 3>(v, m); break;
    case kCodeDR + 7: apply2dr<1, 2>(v, m); break;
    case kCodeDR + 8: apply2dr<1, 3>(v, m); break;
    default: apply2dr<2, 3>(v, m); break;
    }
}

// float2 entries of a block matrix in the pool: general 2x2 4, 4x4 16; diagonal-times-real 2x2 4,
// 4x4 12 (all even, so matrices stay 16-byte aligned).
PTSBE_HD uint32_t code_mat_count(int code) {
    return code < kCodes1 ? 4u : code < kCodeDR ? 16u : code < kCodeDR + kCodes1 ? 4u : 12u;
}

// Swizzled tile address of thread t's register base in group g.
PTSBE_HD uint32_t group_base(const Group& g, uint32_t t) {
    uint32_t b = 0;
#pragma unroll
    for (int k = 0; k < kTB; ++k)
        if ((t >> k) & 1u) b ^= g.toff[k];
    return b;
}

// Amplitude offset of outer index tau (bits -> physical positions opos).
PTSBE_HD uint64_t outer_offset(const Pass& p, uint64_t tau) {
    uint64_t o = 0;
    for (uint32_t k = 0; k < p.nouter; ++k)
        if ((tau >> k) & 1u) o |= 1ull << p.opos[k];
    return o;
}

}  // namespace dense
}  // namespace ptsbe
