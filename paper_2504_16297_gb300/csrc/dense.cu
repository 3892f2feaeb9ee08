// Dense tile passes (dense.cuh): batched state preparation (Sec. 3) for states too large, or too
// densely mixed, for the deferred-frame kernel -- every amplitude streams through HBM once per pass
// and every gate and Kraus operator of the pass is applied on chip.
//
// One launch runs one pass for a list of nodes (a node = one Kraus set's state: where its tiles are
// read from, where they go, and the set's override blocks -- the fused blocks that contain one of
// its Kraus entries). Persistent CTAs walk the (node, tile) work items: a tile is loaded with
// 16-byte loads into XOR-swizzled shared memory, every register group of the pass loads its 16
// amplitudes per thread, applies its blocks in registers and writes them back, and the tile is
// stored in the pass's output order. The last pass also leaves each tile's FP64 squared norm.
#include <algorithm>

#include "dense.cuh"
#include "internal.h"
#include "tile_ops.cuh"

namespace ptsbe {

namespace {

using namespace dense;

constexpr int kDenseCtasPerSm = 2;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Copy of `bytes` (a multiple of 4) from global to shared memory by the whole CTA.
__device__ __forceinline__ void copy_words(void* dst, const void* src, uint32_t bytes) {
    const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    for (uint32_t i = threadIdx.x; i < bytes / 4; i += blockDim.x) d[i] = __ldg(s + i);
}

// Shared-memory tables of the pass a CTA is working on.
struct PassSmem {
    Pass P;
    uint32_t hi[kHi];
    uint16_t omap[kHi];
};

// The pass's groups, blocks and default matrices, in shared memory when they fit (else global).
struct PassView {
    const Group* groups;
    const Block* blocks;
    const float2* mats;
};

// Loads pass `pass` of a plan into shared memory (whole CTA; ends with a barrier).
__device__ PassView load_pass(PassSmem& S, unsigned char* stage, const Pass* passes, uint32_t pass, const Group* g_groups,
                              const Block* g_blocks, const uint32_t* g_hi, const uint16_t* g_omap, const float2* g_mats) {
    if (threadIdx.x == 0) S.P = passes[pass];
    __syncthreads();
    const Pass& P = S.P;
    for (uint32_t i = threadIdx.x; i < (uint32_t)kHi; i += kThreads) {
        S.hi[i] = __ldg(g_hi + P.hi_off + i);
        S.omap[i] = __ldg(g_omap + P.omap_off + i);
    }
    // every pass's tables fit the stage (the planner guarantees it)
    static_assert(sizeof(Group) % 4 == 0 && sizeof(Block) % 4 == 0, "staged tables move 4-byte words");
    copy_words(stage, g_groups + P.group_begin, (P.group_end - P.group_begin) * (uint32_t)sizeof(Group));
    const uint32_t bo = dense_stage_blocks_off(P), mo = dense_stage_mats_off(P);
    copy_words(stage + bo, g_blocks + P.blk_begin, (P.blk_end - P.blk_begin) * (uint32_t)sizeof(Block));
    copy_words(stage + mo, g_mats + P.mat_begin, (P.mat_end - P.mat_begin) * (uint32_t)sizeof(float2));
    PassView v{reinterpret_cast<const Group*>(stage), reinterpret_cast<const Block*>(stage + bo),
               reinterpret_cast<const float2*>(stage + mo)};
    __syncthreads();
    return v;
}

constexpr int kVec = (1 << (kT - 1)) / kThreads;   // float4 (two amplitudes) per thread per tile
static_assert(kVec % 8 == 0, "tile loads go in rounds of eight");

// One tile of one state for one pass: load (or |0...0> / zero tile), every register group, store;
// with `part`, the tile's FP64 squared norm goes to *part. Starts and ends with a barrier. Tiles
// are read through L2 (ld.global.cg): in the queue kernel they were written by other CTAs of the
// same launch.
__device__ void dense_tile(const PassSmem& S, const PassView& V, float2* tile, double* red, const Node& nd, uint64_t tau,
                           double* part, const Override* __restrict__ ovr, const float2* __restrict__ opool) {
    const uint32_t tid = threadIdx.x;
    const Pass& P = S.P;
    const uint64_t outer = outer_offset(P, tau);
    __syncthreads();   // the previous item's store has read the tile
    if (nd.src == nullptr && tau != 0) {
        // a state starting from |0...0>: every other tile is zero and stays zero in this pass
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < kVec; ++i) {
            const uint32_t L = 2u * (i * kThreads + tid);
            __stcs(reinterpret_cast<float4*>(nd.dst + outer + (L & 15u) + S.hi[L >> kC]), z);
        }
        if (part && tid == 0) *part = 0.0;
        __syncthreads();
        return;
    }
    if (nd.src == nullptr) {
#pragma unroll
        for (int i = 0; i < (1 << kT) / kThreads; ++i) tile[i * kThreads + tid] = make_float2(0.f, 0.f);
        __syncthreads();
        if (tid == 0) tile[0] = make_float2(1.f, 0.f);
    } else {
        // eight 16-byte loads in flight per thread, twice
#pragma unroll
        for (int h = 0; h < kVec; h += 8) {
            float4 x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint32_t t = 2u * ((h + i) * kThreads + tid);
                x[i] = __ldcg(reinterpret_cast<const float4*>(nd.src + outer + (t & 15u) + S.hi[t >> kC]));
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint32_t t = 2u * ((h + i) * kThreads + tid);
                const uint32_t s = swz(t);
                const float4 y = (s & 1u) ? make_float4(x[i].z, x[i].w, x[i].x, x[i].y) : x[i];
                *reinterpret_cast<float4*>(tile + (s & ~1u)) = y;
            }
        }
    }
    __syncthreads();
    // the set's override blocks in this pass, in execution order
    uint32_t ov = nd.ov_begin;
    while (ov < nd.ov_end && ovr[ov].block < P.blk_begin) ++ov;
    uint32_t next_ov = ov < nd.ov_end ? ovr[ov].block : 0xFFFFFFFFu;
    const uint32_t ngroups = P.group_end - P.group_begin;
    for (uint32_t g = 0; g < ngroups; ++g) {
        const Group& G = V.groups[g];
        const uint32_t base = group_base(G, tid);
        float2 v[kAmps];
#pragma unroll
        for (int j = 0; j < kAmps; ++j) v[j] = tile[base ^ G.roff[j]];
        const uint32_t b1 = G.blk_end - P.blk_begin;
        for (uint32_t b = G.blk_begin - P.blk_begin; b < b1; ++b) {
            const Block B = V.blocks[b];
            const float2* m = V.mats + (B.mat - P.mat_begin);
            int code = B.code;
            if (B.id == next_ov) {
                m = opool + ovr[ov].mat;
                code = (int)ovr[ov].code;
                ++ov;
                next_ov = ov < nd.ov_end ? ovr[ov].block : 0xFFFFFFFFu;
            }
            apply_block(v, code, m);
        }
#pragma unroll
        for (int j = 0; j < kAmps; ++j) tile[base ^ G.roff[j]] = v[j];
        __syncthreads();
    }
    double nrm = 0.0;
    const uint32_t o1 = P.olow[1];
#pragma unroll
    for (int i = 0; i < kVec; ++i) {
        const uint32_t L = 2u * (i * kThreads + tid);
        const uint32_t t0 = S.omap[L >> kC] ^ P.olow[L & 15u];
        const float2 p0 = tile[swz(t0)], p1 = tile[swz(t0 ^ o1)];
        __stcs(reinterpret_cast<float4*>(nd.dst + outer + (L & 15u) + S.hi[L >> kC]), make_float4(p0.x, p0.y, p1.x, p1.y));
        if (part) nrm += (double)(p0.x * p0.x + p0.y * p0.y) + (double)(p1.x * p1.x + p1.y * p1.y);
    }
    if (part) {
        nrm = warp_sum(nrm);
        if ((tid & 31) == 0) red[tid >> 5] = nrm;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int i = 0; i < kThreads / 32; ++i) s += red[i];
            *part = s;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads, kDenseCtasPerSm) k_dense_pass(DenseArgs a) {
    __shared__ __align__(16) float2 tile[1 << kT];
    __shared__ PassSmem S;
    __shared__ double red[kThreads / 32];
    extern __shared__ __align__(16) unsigned char stage[];
    const PassView V = load_pass(S, stage, a.passes, (uint32_t)a.pass, a.groups, a.blocks, a.hi, a.omap, a.mats);
    const int ob = a.n - kT;
    const uint64_t items = (uint64_t)a.n_nodes << ob;
    const uint64_t tmask = (1ull << ob) - 1;
    for (uint64_t w = blockIdx.x; w < items; w += gridDim.x) {
        const uint32_t ni = (uint32_t)(w >> ob);
        const uint64_t tau = w & tmask;
        const Node nd = a.nodes[ni];
        dense_tile(S, V, tile, red, nd, tau, a.last ? a.part + ((size_t)nd.part << ob) + tau : nullptr, a.ovr, a.opool);
    }
}

// ---- one persistent launch over many circuits (a device work queue) -----------------------------
// Work items are handed out in order by one global counter. Item w belongs to the task t with
// item0[t] <= w < item0[t + 1]; tasks are (set, level) of a job: levels 0 .. J-1 are the dense
// passes (one item per tile), J the set's finalisation (one item: weight, flag, scale from the
// tile norms) and J + 1 the scaling of its state (one item per 2^kT amplitudes). A task waits until
// every item of its predecessor (the same set's previous level) is done; tasks are ordered level by
// level, so a predecessor's items were handed out earlier to CTAs that are running (a cooperative
// launch keeps every CTA resident) and the earliest unfinished item never waits: the queue cannot
// deadlock. A wait gives up after spin_cycles (clock64) and records the task in *err; every CTA
// then leaves, and the host reports PTSBE_ERR_TIMEOUT.

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(kThreads, kDenseCtasPerSm) k_dense_queue(QueueArgs a) {
    __shared__ __align__(16) float2 tile[1 << kT];
    __shared__ PassSmem S;
    __shared__ double red[kThreads / 32];
    __shared__ double qred[33];
    __shared__ uint64_t s_item;
    __shared__ uint32_t s_task, s_stop;
    extern __shared__ __align__(16) unsigned char stage[];
    const uint32_t tid = threadIdx.x;
    uint32_t cur_job = 0xFFFFFFFFu, cur_pass = 0xFFFFFFFFu;
    PassView V{nullptr, nullptr, nullptr};
    for (;;) {
        if (tid == 0) {
            s_stop = 0;
            if (*(volatile uint32_t*)a.err) {
                s_stop = 1;
            } else {
                const unsigned long long w = atomicAdd(a.next, 1ull);
                if (w >= a.n_items) {
                    s_stop = 1;
                } else {
                    uint32_t lo = 0, hi = a.n_tasks - 1;   // last task with item0 <= w
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if (a.tasks[mid].item0 <= w) lo = mid; else hi = mid - 1;
                    }
                    s_task = lo;
                    s_item = w - a.tasks[lo].item0;
                    const QTask& T = a.tasks[lo];
                    if (T.pred != 0xFFFFFFFFu) {
                        const uint32_t need = T.pred_items + (lo == a.stall_task ? 1u : 0u);
                        const long long t0 = clock64();
                        while (ld_acquire(a.done + T.pred) < need) {
                            if (clock64() - t0 > a.spin_cycles) {
                                atomicCAS(a.err, 0u, lo + 1);
                                s_stop = 1;
                                break;
                            }
                            if (*(volatile uint32_t*)a.err) { s_stop = 1; break; }
                            __nanosleep(128);
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (s_stop) break;
        const uint32_t t = s_task;
        const uint64_t item = s_item;
        const QTask T = a.tasks[t];
        const QJob& J = a.jobs[T.job];
        const int ob = (int)J.n - kT;
        float2* state = J.states + ((size_t)T.set << J.n);
        if (T.level < J.J) {
            if (T.job != cur_job || T.level != cur_pass) {
                __syncthreads();
                V = load_pass(S, stage, J.passes, T.level, J.groups, J.blocks, J.hi, J.omap, J.mats);
                cur_job = T.job;
                cur_pass = T.level;
            }
            Node nd{};
            nd.src = T.level == 0 ? nullptr : state;
            nd.dst = state;
            nd.ov_begin = J.ov_begin[T.set];
            nd.ov_end = J.ov_end[T.set];
            dense_tile(S, V, tile, red, nd, item,
                       T.level + 1 == J.J ? J.part + ((size_t)T.set << ob) + item : nullptr, J.ovr, J.opool);
        } else if (T.level == J.J) {
            // finalisation: squared norm from the tile norms (fixed order), weight, flag, scale
            // (the order of the stand-alone reduction kernel, so the results are the same bit for bit)
            const double* p = J.part + ((size_t)T.set << ob);
            double acc = 0.0;
            for (uint32_t i = tid; i < (1u << ob); i += kThreads) acc += __ldcg(p + i);
            const double tot = tile::cta_sum(acc, qred);
            if (tid == 0) {
                const double w = J.wmix[T.set] * tot;
                const bool null = !(tot > 0.0) || w < 1e-6 * J.qalpha[T.set];
                J.scale[T.set] = null ? 0.0f : (float)(1.0 / sqrt(tot));
                if (J.weights) J.weights[T.set] = w;
                if (J.status) J.status[T.set] = null ? 1 : 0;
            }
        } else {
            // scaling of amplitudes [item 2^kT, (item + 1) 2^kT)
            const float sc = __ldcg(J.scale + T.set);
            float4* v = reinterpret_cast<float4*>(state + (item << kT));
#pragma unroll
            for (int i = 0; i < kVec; ++i) {
                float4 x = __ldcg(v + i * kThreads + tid);
                x.x *= sc; x.y *= sc; x.z *= sc; x.w *= sc;
                __stcg(v + i * kThreads + tid, x);
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(a.done + t, 1u);
        }
    }
}

}  // namespace

int dense_ctas_per_sm() { return kDenseCtasPerSm; }

// Zero-padded dense states back to their own size: thread-strided copy of float4 pairs.
__global__ void __launch_bounds__(256) k_dense_unpad(const float4* __restrict__ src, int n_in, float4* __restrict__ dst,
                                                     int n_out, uint64_t total) {
    const int shift = n_out - 1;                       // float4 per output state: 2^(n_out - 1)
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t st = i >> shift, k = i & ((1ull << shift) - 1ull);
        dst[i] = __ldcs(src + (st << (n_in - 1)) + k);
    }
}

void launch_dense_unpad(const float2* src, int n_in, float2* dst, int n_out, uint32_t count, int n_sm, cudaStream_t s) {
    if (count == 0) return;
    if (n_out < 1 || n_out > n_in) fail(PTSBE_ERR_INVALID, "dense unpad: bad sizes");
    if ((uintptr_t)dst % 16) fail(PTSBE_ERR_INVALID, "d_states must be 16-byte aligned");
    const uint64_t total = (uint64_t)count << (n_out - 1);
    const uint64_t grid = std::min<uint64_t>((total + 255) / 256, (uint64_t)std::max(n_sm, 1) * 8);
    k_dense_unpad<<<(uint32_t)grid, 256, 0, s>>>(reinterpret_cast<const float4*>(src), n_in, reinterpret_cast<float4*>(dst),
                                                  n_out, total);
    PTSBE_CUDA(cudaGetLastError());
    count_launch();
}

void launch_dense_pass(const DenseArgs& a, int n_sm, cudaStream_t s) {
    if (a.n_nodes == 0) return;
    if (a.n < kT || a.n > kMaxQ) fail(PTSBE_ERR_UNSUPPORTED, "dense passes need 12 <= n <= 32");
    const uint64_t items = (uint64_t)a.n_nodes << (a.n - kT);
    const uint64_t cap = (uint64_t)std::max(1, n_sm) * kDenseCtasPerSm;
    const uint32_t grid = (uint32_t)std::min<uint64_t>(items, cap);
    // thread-safe once: two contexts may be driven from two host threads
    static const bool configured = [&] {
        PTSBE_CUDA(cudaFuncSetAttribute(k_dense_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageMax));
        return true;
    }();
    (void)configured;
    k_dense_pass<<<grid, kThreads, a.stage_bytes, s>>>(a);
    PTSBE_CUDA(cudaGetLastError());
    count_launch();
}

int dense_queue_grid(int n_sm) {
    static const int per_sm = [] {    // thread-safe once
        int v = 0;
        PTSBE_CUDA(cudaFuncSetAttribute(k_dense_queue, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageMax));
        PTSBE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_dense_queue, kThreads, kStageMax));
        return v;
    }();
    return std::max(1, per_sm) * std::max(1, n_sm);
}

void launch_dense_queue(const QueueArgs& a, int n_sm, cudaStream_t s) {
    if (a.n_items == 0) return;
    const int grid = (int)std::min<uint64_t>(a.n_items, (uint64_t)dense_queue_grid(n_sm));
    // a cooperative launch: every CTA resident at once (CTAs wait on one another's items)
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kStageMax;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PTSBE_CUDA(cudaLaunchKernelEx(&cfg, k_dense_queue, a));
    count_launch();
}

}  // namespace ptsbe
