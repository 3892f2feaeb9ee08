// Batched state preparation for PTSBE (Sec. 3: each Kraus set alpha is prepared once).
//
// One CTA owns one tile (2^tb complex64 amplitudes, shared memory) of one state for one stage of
// the plan. It gathers the tile from HBM (segments of 2^lb contiguous amplitudes), applies every
// op of the stage in shared memory -- gates, and at each noise site the Kraus operator that the
// state's set alpha selects (operator 0 where alpha lists nothing) -- and scatters the tile back.
// When the whole state fits one tile (n <= tb) the entire circuit runs in a single launch and the
// final renormalisation and branch weight are fused into the same CTA.
//
// Renormalisation (Sec. 2.2) is deferred to the end: the branch weight is the squared norm of
// the unnormalised state times the unitary-mixture probabilities, and dividing once at the end
// gives the same normalised state as dividing after every general Kraus operator.
//
// Prefix reuse: when set beta extends set alpha of the same batch (alpha's entries are a prefix of
// beta's), beta skips the stages before the one holding its first extra site. In that stage it
// reads alpha's input of the stage and runs the whole stage with its own operators (identical to
// alpha's up to the extra site). Stages alternate between two state buffers, so every input of a
// stage is still intact while the stage writes its outputs; one launch per stage covers all sets.
#include <cstdio>

#include "fixed_point.cuh"
#include "frame.cuh"
#include "internal.h"
#include "philox.h"
#include "tile_ops.cuh"

namespace ptsbe {

namespace {
using namespace tile;

// Shared memory of the per-operator kernel: tile (2^tb complex64), hi table (2^(tb-lb) words),
// then, 16-byte aligned, the staged matrices.
__host__ __device__ inline size_t evolve_stage_mats_offset(int tb, int lb) {
    return (((size_t)8 << tb) + ((size_t)4 << (tb - lb)) + 15) & ~(size_t)15;
}

__global__ void __launch_bounds__(1024) k_evolve_stage(EvolveArgs a, int stage_idx, int last, const uint32_t* __restrict__ nodes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ DevStage st;
    __shared__ double red[33];
    const int tb = a.tb, lb = a.lb, n = a.n, ob = n - tb;
    float2* tile = reinterpret_cast<float2*>(smem);
    uint32_t* hi = reinterpret_cast<uint32_t*>(tile + (1u << tb));
    // The circuit's matrices, when the launch stages them: every operator reads its matrix from
    // shared memory instead of a global load on the CTA's serial chain of operators.
    float2* smats = reinterpret_cast<float2*>(smem + evolve_stage_mats_offset(tb, lb));
    const float2* mats = a.stage_mats ? smats : a.mats;
    for (uint32_t i = threadIdx.x; i < a.stage_mats; i += blockDim.x) smats[i] = __ldg(a.mats + i);
    if (threadIdx.x == 0) st = a.stages[stage_idx];
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < (1u << (tb - lb)); i += blockDim.x) hi[i] = a.hi[st.hi_off + i];
    const uint32_t node = nodes[blockIdx.y];
    const uint32_t tau = blockIdx.x;
    uint64_t outer = 0;
    for (int b = 0; b < ob; ++b)
        if ((tau >> b) & 1u) outer |= 1ull << st.outer_q[b];
    float2* g = a.states + ((size_t)node << n);
    const uint32_t src = stage_idx == (int)a.node_sstage[node] ? a.node_src[node] : node;
    const float2* gin = a.states_in + ((size_t)src << n);
    const uint32_t start = st.op_begin;
    __syncthreads();
    if (a.node_fresh[node] && stage_idx == 0) {
        for (uint32_t l = threadIdx.x; l < (1u << tb); l += blockDim.x)
            tile[l] = make_float2((l == 0 && tau == 0) ? 1.0f : 0.0f, 0.0f);
    } else {
        tile_load(tile, gin, tb, lb, hi, outer);
    }
    uint32_t e = a.node_ebeg[node];
    const uint32_t ee = a.node_eend[node];
    while (e < ee && a.site_op[a.ent_site[e]] < start) ++e;
    __syncthreads();

    __shared__ DevOp sops[kOpChunk];
    OpWindow win{sops};
    for (uint32_t op = start; op < st.op_end; ++op) {
        const DevOp o = win.at(a.ops, op, st.op_end);
        if (o.kind == DOP_NOISE) {
            uint32_t k = 0;
            if (e < ee && a.ent_site[e] == o.site) { k = a.ent_k[e]; ++e; }
            const uint32_t u0 = a.chans[o.ch].micro_off[k], u1 = a.chans[o.ch].micro_off[k + 1];
            for (uint32_t u = u0; u < u1; ++u) {
                const DevMicro mi = a.micro[u];
                const int pa = st.pos[mi.operand == 1 ? o.q1 : o.q0];
                const int pb = st.pos[o.q1];
                apply_micro(tile, tb, mi.kind, pa, pb, mats + mi.mat);
                __syncthreads();
            }
        } else {
            if (o.fend != 0 && (e >= ee || a.ent_site[e] >= o.fsite1)) {
                // no error inside the fused block: gate and no-error operators at once
                if (o.fkind != DOP_NOP) {
                    apply_micro(tile, tb, o.fkind, st.pos[o.q0], st.pos[o.q1], mats + o.fmat, o.fperm);
                    __syncthreads();
                }
                op = o.fend - 1;
                continue;
            }
            if (o.kind != DOP_NOP) {
                apply_micro(tile, tb, o.kind, st.pos[o.q0], st.pos[o.q1], mats + o.mat);
                __syncthreads();
            }
        }
    }

    if (!last) {
        tile_store(tile, g, tb, lb, hi, outer, 1.0f);
        return;
    }
    const double part = cta_sum(tile_norm_partial(tile, tb), red);
    if (ob == 0) {
        const double w = a.wmix[node] * part;
        const bool null = !(part > 0.0) || w < 1e-6 * a.qalpha[node];
        const float scale = null ? 0.0f : (float)(1.0 / sqrt(part));
        tile_store(tile, g, tb, lb, hi, outer, scale);
        if (threadIdx.x == 0) {
            if (a.weights) a.weights[node] = w;
            if (a.status) a.status[node] = null ? 1 : 0;
        }
    } else {
        tile_store(tile, g, tb, lb, hi, outer, 1.0f);
        if (threadIdx.x == 0) a.part[((size_t)node << ob) + tau] = part;
    }
}

// Frame kernel: same work as k_evolve_stage, with permutations and diagonals deferred (frame.cuh).
// Thread 0 builds the program of the stage while the other warps bring the tile in.
// Dynamic shared memory of the frame kernel: tile (tamps complex64), hi table, factor tables.
__host__ __device__ inline size_t frame_tab_offset_amps(uint32_t tamps, int tb, int lb) {
    return ((size_t)8 * tamps + ((size_t)4 << (tb - lb)) + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t frame_tab_offset(int tb, int lb) { return frame_tab_offset_amps(1u << tb, tb, lb); }

// One thread per node of a launch builds the node's program for the stage (the first segment, and
// the builder state a tile CTA needs to continue when the program is longer). A CTA serves 16
// nodes (builder states in shared memory); SPW of them share a warp, one per group of 32 / SPW
// lanes. The builders' branches depend on each set's entries, so lanes of one warp diverge: fewer
// sets per warp run shorter instruction streams, and more warps share each scheduler.
constexpr int kProgSets = 16;
template <int SPW>
__global__ void __launch_bounds__(32 * (kProgSets / SPW), SPW == 4 ? 5 : 1)
k_frame_program(EvolveArgs a, int stage_idx, const uint32_t* __restrict__ nodes, uint32_t n_nodes, frame::Program* progs) {
    using namespace frame;
    __shared__ Builder Bs[kProgSets];
    __shared__ DevStage st;
    if (threadIdx.x == 0) st = a.stages[stage_idx];
    __syncthreads();
    constexpr uint32_t stride = 32 / SPW;
    const uint32_t lane = threadIdx.x & 31u;
    if (lane % stride) return;
    const uint32_t slot = (threadIdx.x >> 5) * SPW + lane / stride;
    const uint32_t i = blockIdx.x * kProgSets + slot;
    if (i >= n_nodes) return;
    const uint32_t node = nodes[i];
    Builder& B = Bs[slot];
    Program& P = progs[i];
    builder_init(B, a, st, a.fstages[stage_idx], node, a.node_fresh[node] && stage_idx == 0);
    build_segment(B, P.S, P.pool, a, st, kProgSteps, kProgPool);
    P.B = B;
}

// Zero fill apart from the evolve launch (the small sparse final stage writes only each state's
// support, so every other amplitude of its output is a zero that can be stored before the programs
// exist): the first `prefix` bytes of each of the states at base + i * state_bytes, by bulk copies
// (TMA) of a zeroed shared buffer. Lane l of CTA c copies chunks 32 c + l, 32 (c + G) + l, ... of
// the count * prefix / kFillChunk chunks (G CTAs); prefix is a multiple of kFillChunk.
constexpr uint32_t kFillChunk = 4096;
__global__ void __launch_bounds__(32) k_zero_states(unsigned char* __restrict__ base, uint64_t state_bytes,
                                                    uint64_t prefix, uint64_t chunks) {
    __shared__ __align__(128) float4 z[kFillChunk / 16];
    for (uint32_t v = threadIdx.x; v < kFillChunk / 16; v += 32) z[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    const uint32_t src = (uint32_t)__cvta_generic_to_shared(z);
    const uint64_t per_state = prefix / kFillChunk;
    const uint64_t lanes = (uint64_t)gridDim.x * 32u;
    for (uint64_t c = (uint64_t)blockIdx.x * 32u + threadIdx.x; c < chunks; c += lanes) {
        const uint64_t st = c / per_state, off = st * state_bytes + (c - st * per_state) * kFillChunk;
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                     :: "l"(base + off), "r"(src), "n"(kFillChunk) : "memory");
    }
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Copies from global memory (read-only path: the source must not be in shared memory).
__device__ __forceinline__ void copy_words(void* dst, const void* src, uint32_t bytes, uint32_t t, uint32_t nt) {
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
    for (uint32_t i = t; i < bytes / 4; i += nt) d[i] = __ldg(s + i);
}

// Sparse final store fused with drawing the state's shots (Sec. 3: all m_alpha shots of a
// prepared state at once). The CTA holds the state's support on chip, so the outcome CDF is built
// from it instead of from a read of the stored 2^n amplitudes: every other amplitude is an exact
// zero and adds nothing to an inclusive prefix, so the smallest index whose prefix exceeds a
// target is a support entry, and the shots equal those the stand-alone samplers draw from the
// stored state (same fixed-point probabilities of the same stored values, same Philox counters).
// Support entries are placed in increasing logical order by their bits at the order mask's
// positions (frame::sparse_order_mask); cdf and lidx (2^ncomp entries each) live in scratch.
// A heavy state (exp != null) leaves the CDF in its export slot instead (SupportCdfHeader layout)
// for k_sample_support, which spreads its shots over many CTAs.
__device__ void scatter_and_sample(const EvolveArgs& a, const frame::Step& fin, const DevFrameStage& fs,
                                   const float2* tile, const float2* tabs, const uint32_t* delta, const uint32_t* hi,
                                   float2* g, float scale, bool null, uint32_t node, uint32_t m, unsigned char* exp,
                                   void* scratch, double* red, uint32_t tid, uint32_t nthr) {
    using namespace frame;
    __shared__ uint32_t order, ok;
    const int n = a.n;
    uint32_t* out = exp ? nullptr : a.shot_bits + a.node_shot_out[node];
    if (tid == 0) {
        order = sparse_order_mask(fin, fs, n, a.lb, hi);
        ok = (!null && fin.ncomp != 0xFF && (uint32_t)__popc(order) == fin.ncomp) ? 1u : 0u;
        if (!null && !ok) atomicOr(a.fault, 1u);
    }
    __syncthreads();
    const uint32_t last = (uint32_t)((1ull << n) - 1ull);
    if (!ok) {
        // A null state has no outcome: the all-ones marker when the status is recorded (as the
        // samplers write), else what they draw from its zeroed amplitudes (T = 0: the last index).
        // The other case cannot occur for a plan's support (flagged above) and leaves the marker.
        if (!null) run_sparse_final(fin, fs, tile, tabs, delta, n, a.lb, hi, g, scale, 1, tid, nthr);
        const uint32_t mark = (null && !a.status) ? last : 0xFFFFFFFFu;
        if (exp) {
            if (tid == 0) {
                SupportCdfHeader* h = reinterpret_cast<SupportCdfHeader*>(exp);
                h->T = 0; h->n = 0; h->mark_all = 1; h->mark = mark; h->nq = (uint32_t)n;
            }
            return;
        }
        for (uint32_t k = tid; k < m; k += nthr) out[k] = mark;
        return;
    }
    const uint32_t H = order, N = 1u << fin.ncomp;
    fx* cdf = reinterpret_cast<fx*>(scratch);
    uint32_t* lidx = reinterpret_cast<uint32_t*>(cdf + N);
    for (uint32_t i = tid; i < N; i += nthr) {
        const uint32_t p = enum_base(fin, i, nullptr, 0);
        const float2 v = mul2r(sparse_value(fin, tile, tabs, delta, p), scale);
        const uint32_t l = sparse_logical(fin, fs, n, a.lb, hi, p);
        g[l] = v;
        const uint32_t r = extract_bits(l, H);
        cdf[r] = fx_prob(v);
        lidx[r] = l;
    }
    __syncthreads();
    // inclusive prefix in rank order: thread t owns K consecutive entries
    const uint32_t K = N > nthr ? N / nthr : 1u, c0 = tid * K;
    fx mine = 0;
    if (c0 < N)
        for (uint32_t i = 0; i < K; ++i) mine += cdf[c0 + i];
    fx v = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const fx y = __shfl_up_sync(0xffffffffu, v, o);
        if ((tid & 31) >= (uint32_t)o) v += y;
    }
    fx* fred = reinterpret_cast<fx*>(red);
    const uint32_t w = tid >> 5, nw = nthr >> 5;
    if ((tid & 31) == 31) fred[w] = v;
    __syncthreads();
    if (tid == 0) {
        fx acc = 0;
        for (uint32_t i = 0; i < nw; ++i) { const fx t = fred[i]; fred[i] = acc; acc += t; }
    }
    __syncthreads();
    fx run = fred[w] + (v - mine);
    if (c0 < N)
        for (uint32_t i = 0; i < K; ++i) { run += cdf[c0 + i]; cdf[c0 + i] = run; }
    __syncthreads();
    const fx T = cdf[N - 1];
    if (exp) {
        SupportCdfHeader* h = reinterpret_cast<SupportCdfHeader*>(exp);
        fx* ec = reinterpret_cast<fx*>(exp + sizeof(SupportCdfHeader));
        uint32_t* el = reinterpret_cast<uint32_t*>(ec + N);
        for (uint32_t i = tid; i < N; i += nthr) { ec[i] = cdf[i]; el[i] = lidx[i]; }
        if (tid == 0) { h->T = T; h->n = N; h->mark_all = 0; h->mark = 0; h->nq = (uint32_t)n; }
        return;
    }
    const uint32_t alpha = a.shot_alpha0 + node;
    for (uint32_t k = tid; k < m; k += nthr) {
        const Philox4 x = philox4x32_10(k, 0u, alpha, kDomShot, (uint32_t)a.shot_seed, (uint32_t)(a.shot_seed >> 32));
        const fx t = fx_target(u53_bits(x.x[0], x.x[1]), T);
        uint32_t idx = last;                            // T = 0
        if (t < T) {
            uint32_t lo = 0, hi2 = N - 1;               // smallest rank r with t < cdf[r]
            while (lo < hi2) {
                const uint32_t mid = (lo + hi2) >> 1;
                if (t < cdf[mid]) hi2 = mid; else lo = mid + 1;
            }
            idx = lidx[lo];
        }
        out[k] = idx;
    }
}

constexpr int kFrameThreads = 512;   // 128 registers per thread: grouped mixes stay in registers
// SMALL: a sparse final stage whose support lies below tile address 2^fs.sbits (the plan entered
// the stage in a layout that maps the mixing directions to the low bits); the tile buffer holds
// only that prefix, so several CTAs share an SM and one CTA's stores overlap another's passes.
constexpr int kFrameSmallThreads = 128;
constexpr int kZeroChunk = 4096;      // bytes per bulk zero copy (the state size is a multiple)
constexpr int kFrameSmallCtas = 4;
template <bool SMALL>
__global__ void __launch_bounds__(SMALL ? kFrameSmallThreads : kFrameThreads, SMALL ? kFrameSmallCtas : 1)
k_evolve_frame(EvolveArgs a, int stage_idx, int last, const uint32_t* __restrict__ nodes,
               const frame::Program* __restrict__ progs) {
    using namespace frame;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ DevStage st;
    __shared__ DevFrameStage fs;
    __shared__ double red[33];
    __shared__ Builder B;
    __shared__ Step S[kMaxSteps];
    __shared__ Factor pool[kMaxPool];
    __shared__ uint32_t delta[kMaxTabs * kDeltaSlots];
    __shared__ __align__(128) float4 zbuf[SMALL ? kZeroChunk / 16 : 1];
    const int tb = a.tb, lb = a.lb, n = a.n, ob = n - tb;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    float2* tile = reinterpret_cast<float2*>(smem);
    copy_words(&st, a.stages + stage_idx, sizeof(DevStage), tid, nthr);
    copy_words(&fs, a.fstages + stage_idx, sizeof(DevFrameStage), tid, nthr);
    __syncthreads();
    const uint32_t tamps = SMALL ? (1u << fs.sbits) : (1u << tb);
    uint32_t* hi = reinterpret_cast<uint32_t*>(tile + tamps);
    float2* tabs = reinterpret_cast<float2*>(smem + frame_tab_offset_amps(tamps, tb, lb));
    for (uint32_t i = tid; i < (1u << (tb - lb)); i += nthr) hi[i] = a.hi[st.hi_off + i];
    const uint32_t node = nodes[blockIdx.y];
    const uint32_t tau = blockIdx.x;
    const uint64_t outer = outer_offset(st, ob, tau);
    float2* g = a.states + ((size_t)node << n);
    const uint32_t src = stage_idx == (int)a.node_sstage[node] ? a.node_src[node] : node;
    const float2* gin = a.states_in + ((size_t)src << n);
    const bool fresh = a.node_fresh[node] && stage_idx == 0;
    // From |0...0>, every mix of the first stage moves along directions inside the tile (the plan
    // guarantees it), and permutations and diagonals never widen the set of nonzero amplitudes: all
    // of them stay in the tile holding index 0. Every other tile of the state is zero for the whole
    // stage and only writes zeros where the stage's store puts it.
    const bool zero_tile = fresh && tau != 0;
    __syncthreads();
    // The first program segment is read in place (global memory, the same for all tiles of the
    // set); segments built here when the program is longer live in shared memory.
    const Program& P = progs[blockIdx.y];
    const Step* Sp = P.S;
    const Factor* poolp = P.pool;
    if (tid < 32) {
        // warp 0, while the others bring the tile: the builder state, and the factor pool when it
        // fits shared memory (table builds read it over and over)
        copy_words(&B, &P.B, sizeof(Builder), tid, 32);
        __syncwarp();
        if (B.npool <= (uint32_t)kMaxPool) copy_words(pool, P.pool, B.npool * (uint32_t)sizeof(Factor), tid, 32);
        if (B.nsteps <= (uint32_t)kMaxSteps) copy_words(S, P.S, B.nsteps * (uint32_t)sizeof(Step), tid, 32);
    } else {
        const uint32_t t = tid - 32, nt = nthr - 32, nv = tamps >> 1;
        float4* tile4 = reinterpret_cast<float4*>(tile);
        if (zero_tile) {
            // never read
        } else if (fresh || SMALL) {
            for (uint32_t v = t; v < nv; v += nt)
                tile4[v] = make_float4((v == 0 && tau == 0) ? 1.0f : 0.0f, 0.f, 0.f, 0.f);
        } else {
            // eight independent loads in flight per thread before any lands in shared memory
            for (uint32_t v0 = t; v0 < nv; v0 += 8 * nt) {
                float4 x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const uint32_t v = v0 + u * nt;
                    if (v < nv) x[u] = __ldg(reinterpret_cast<const float4*>(gin + gaddr(2u * v, lb, hi, outer)));
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const uint32_t v = v0 + u * nt;
                    if (v < nv) tile4[v] = x[u];
                }
            }
        }
    }
    if constexpr (SMALL) {
        // The state is all zeros outside the support: the copy engine writes those zeros (bulk
        // copies of a zeroed shared buffer) while the CTA runs the program. Warp 0 only issues
        // the copies (issue stalls while the copy queue is full, so it keeps out of the program's
        // barriers); warps 2-3 run the program with a 64-thread named barrier (the executors step
        // through cosets by thread-count bits, so the count is a power of two); everyone meets
        // for the norm and the scatter once warp 0 has waited for the copies.
        __shared__ Step fin;
        const uint64_t zbytes = (uint64_t)8 << n;
        if (a.prefill_bytes < zbytes) {
            for (uint32_t v = tid; v < (uint32_t)kZeroChunk / 16; v += nthr) zbuf[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (B.npool <= (uint32_t)kMaxPool) poolp = pool;
        if (B.nsteps <= (uint32_t)kMaxSteps) Sp = S;
        const uint32_t warp = tid >> 5;
        if (warp == 0) {
            if (tid == 0 && a.prefill_bytes < zbytes) {
                const uint32_t src = (uint32_t)__cvta_generic_to_shared(zbuf);
                for (uint64_t off = a.prefill_bytes; off < zbytes; off += kZeroChunk)
                    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                                 :: "l"(reinterpret_cast<unsigned char*>(g) + off), "r"(src), "n"(kZeroChunk) : "memory");
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
        } else if (warp >= 2) {
            const uint32_t pt = tid - 64, pn = 64;
            auto pbar = [&]() { asm volatile("bar.sync 1, %0;" :: "r"(pn) : "memory"); };
            if (pt == 0) { fin.kind = ST_FINAL; fin.ncomp = 0xFF; fin.ntab = 0; }   // scatters nothing unless set
            pbar();
            bool found = false;
            while (!found) {
                const uint32_t ns = B.nsteps;
                for (uint32_t si = 0; si < ns; ++si) {
                    const Step& sp = Sp[si];
                    if (sp.ntab) {
                        prepare_tables(sp, fs, poolp, tabs, delta, tb, tau, pt, pn);
                        pbar();
                    }
                    if (sp.kind == ST_MIX1) run_mix1(sp, poolp, tile, tabs, delta, tb, tau, pt, pn);
                    else if (sp.kind == ST_MIX2) run_mix2(sp, tile, tabs, delta, tb, tau, pt, pn);
                    else if (sp.kind == ST_DIAG) run_diag(sp, tile, tabs, delta, tb, pt, pn);
                    else if (sp.kind == ST_FINAL) {
                        // plain loads: the step is in shared memory when the program fits there
                        const uint32_t* s32 = reinterpret_cast<const uint32_t*>(&sp);
                        uint32_t* d32 = reinterpret_cast<uint32_t*>(&fin);
                        for (uint32_t i = pt; i < (uint32_t)(sizeof(Step) / 4); i += pn) d32[i] = s32[i];
                        found = true;
                    }
                    pbar();
                    if (found) break;
                }
                if (found || B.done) break;
                if (pt == 0) build_segment(B, S, pool, a, st, kMaxSteps, kMaxPool);
                pbar();
                Sp = S;
                poolp = pool;
            }
        }
        __syncthreads();
        const double part = cta_sum(run_sparse_final(fin, fs, tile, tabs, delta, n, lb, hi, nullptr, 1.0f, 0, tid, nthr), red);
        const double w = a.wmix[node] * part;
        const bool null = !(part > 0.0) || w < 1e-6 * a.qalpha[node];
        const float scale = null ? 0.0f : (float)(1.0 / sqrt(part));
        const uint32_t m = a.shot_bits ? a.node_shots[node] : 0u;
        const uint32_t e = a.node_export ? a.node_export[node] : 0xFFFFFFFFu;
        unsigned char* exp = e != 0xFFFFFFFFu ? a.support_out + (size_t)e * support_slot_bytes(fs.sbits) : nullptr;
        if (m || exp) {
            // the program's steps and factor pool are dead: their shared memory holds the CDF
            static_assert((sizeof(fx) + sizeof(uint32_t)) << kSmallSupportBits <= sizeof(S), "CDF scratch");
            scatter_and_sample(a, fin, fs, tile, tabs, delta, hi, g, scale, null, node, m, exp, S, red, tid, nthr);
        } else if (!null) {
            run_sparse_final(fin, fs, tile, tabs, delta, n, lb, hi, g, scale, 1, tid, nthr);
        }
        if (tid == 0) {
            if (a.weights) a.weights[node] = w;
            if (a.status) a.status[node] = null ? 1 : 0;
        }
        return;
    }
    __syncthreads();
    if (B.npool <= (uint32_t)kMaxPool) poolp = pool;
    if (B.nsteps <= (uint32_t)kMaxSteps) Sp = S;
    while (true) {
        const uint32_t ns = B.nsteps;
        for (uint32_t si = 0; si < ns; ++si) {
            const Step& sp = Sp[si];
            if (zero_tile && sp.kind <= ST_DIAG) continue;    // uniform across the CTA
            if (sp.ntab && !zero_tile) {
                prepare_tables(sp, fs, poolp, tabs, delta, tb, tau, tid, nthr);
                __syncthreads();
            }
            if (sp.kind == ST_MIX1) {
                run_mix1(sp, poolp, tile, tabs, delta, tb, tau, tid, nthr);
            } else if (sp.kind == ST_MIX2) {
                run_mix2(sp, tile, tabs, delta, tb, tau, tid, nthr);
            } else if (sp.kind == ST_DIAG) {
                run_diag(sp, tile, tabs, delta, tb, tid, nthr);
            } else if (sp.kind == ST_FINAL && fs.sparse_final) {
                // norm over the support, zero-fill, then scatter in logical order (one CTA per state)
                const double part = cta_sum(run_sparse_final(sp, fs, tile, tabs, delta, n, lb, hi, nullptr, 1.0f, 0, tid, nthr), red);
                const double w = a.wmix[node] * part;
                const bool null = !(part > 0.0) || w < 1e-6 * a.qalpha[node];
                const float scale = null ? 0.0f : (float)(1.0 / sqrt(part));
                if constexpr (SMALL) {
                    // the bulk zero copies issued at the start: complete, and ordered before the
                    // scatter's stores
                    if (tid == 0) {
                        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
                        asm volatile("fence.proxy.async.global;" ::: "memory");
                    }
                } else {
                    float4* g4 = reinterpret_cast<float4*>(g);
                    for (uint32_t v = tid; v < (1u << (n - 1)); v += nthr) g4[v] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                __syncthreads();
                if (!null) run_sparse_final(sp, fs, tile, tabs, delta, n, lb, hi, g, scale, 1, tid, nthr);
                if (tid == 0) {
                    if (a.weights) a.weights[node] = w;
                    if (a.status) a.status[node] = null ? 1 : 0;
                }
            } else if (sp.kind == ST_STORE) {
                const double part = run_store(sp, st, tile, tabs, delta, tb, lb, ob, hi, tau, g, tid, nthr, zero_tile);
                if (a.store_norm) {
                    const double tot = cta_sum(part, red);
                    if (tid == 0) a.part[((size_t)node << ob) + tau] = tot;
                }
            } else if (!last) {       // logical order before a frame restart
                run_final(sp, fs, tile, tabs, delta, tb, ob, tau, g, 1.0f, false, tid, nthr, zero_tile);
            } else if (a.scale_in) {
                run_final(sp, fs, tile, tabs, delta, tb, ob, tau, g, a.scale_in[node], false, tid, nthr, zero_tile);
            } else if (ob == 0) {
                const double part = cta_sum(run_final(sp, fs, tile, tabs, delta, tb, ob, tau, nullptr, 1.0f, true, tid, nthr), red);
                const double w = a.wmix[node] * part;
                const bool null = !(part > 0.0) || w < 1e-6 * a.qalpha[node];
                const float scale = null ? 0.0f : (float)(1.0 / sqrt(part));
                run_final(sp, fs, tile, tabs, delta, tb, ob, tau, g, scale, false, tid, nthr);
                if (tid == 0) {
                    if (a.weights) a.weights[node] = w;
                    if (a.status) a.status[node] = null ? 1 : 0;
                }
            } else {
                const double part = cta_sum(run_final(sp, fs, tile, tabs, delta, tb, ob, tau, g, 1.0f, true, tid, nthr, zero_tile), red);
                if (tid == 0) a.part[((size_t)node << ob) + tau] = part;
            }
            __syncthreads();
        }
        if (B.done) break;
        if (tid == 0) build_segment(B, S, pool, a, st, kMaxSteps, kMaxPool);
        Sp = S;
        poolp = pool;
        __syncthreads();
    }
    // no bulk copy may still read this CTA's shared memory when it exits
    if constexpr (SMALL)
        if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Per node: total squared norm from the tile partials (fixed order), weight, null flag, scale.
__global__ void k_evolve_reduce(EvolveArgs a, float* scale_out) {
    __shared__ double red[33];
    const uint32_t node = blockIdx.x;
    const int ob = a.n - a.tb;
    const double* p = a.part + ((size_t)node << ob);
    double acc = 0.0;
    for (uint32_t i = threadIdx.x; i < (1u << ob); i += blockDim.x) acc += p[i];
    const double T = cta_sum(acc, red);
    if (threadIdx.x == 0) {
        const double w = a.wmix[node] * T;
        const bool null = !(T > 0.0) || w < 1e-6 * a.qalpha[node];
        scale_out[node] = null ? 0.0f : (float)(1.0 / sqrt(T));
        if (a.weights) a.weights[node] = w;
        if (a.status) a.status[node] = null ? 1 : 0;
    }
}

__global__ void k_evolve_scale(float2* states, int n, const float* __restrict__ scale) {
    const uint32_t node = blockIdx.y;
    const float s = scale[node];
    float4* v = reinterpret_cast<float4*>(states + ((size_t)node << n));
    const uint64_t nv = 1ull << (n - 1);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (uint64_t)gridDim.x * blockDim.x) {
        float4 x = v[i];
        x.x *= s; x.y *= s; x.z *= s; x.w *= s;
        v[i] = x;
    }
}


// --- register-blocked execution --------------------------------------------------------------------
// Each thread keeps NR = 2^kRegBits amplitudes in registers; register bit b of the index j is the
// tile position reg_pos[b] of the current group. Every op of the group acts on register bits only,
// so it runs as an unrolled loop over j with compile-time partner indices (a Pauli X or CX is a
// register permutation).
constexpr int NR = 1 << kRegBits;
typedef float2 RegArr[NR];

template <int B>
__device__ __forceinline__ void rg1(RegArr& v, const float2* __restrict__ m) {
    const float2 m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
    if (m00.y == 0.f && m01.y == 0.f && m10.y == 0.f && m11.y == 0.f) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j & (1 << B)) continue;
            const float2 x = v[j], y = v[j | (1 << B)];
            v[j] = make_float2(fmaf(m00.x, x.x, m01.x * y.x), fmaf(m00.x, x.y, m01.x * y.y));
            v[j | (1 << B)] = make_float2(fmaf(m10.x, x.x, m11.x * y.x), fmaf(m10.x, x.y, m11.x * y.y));
        }
    } else {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j & (1 << B)) continue;
            const float2 x = v[j], y = v[j | (1 << B)];
            v[j] = cmul2(m00, x, m01, y);
            v[j | (1 << B)] = cmul2(m10, x, m11, y);
        }
    }
}

template <int B>
__device__ __forceinline__ void rd1(RegArr& v, const float2* __restrict__ m) {
    const float2 d0 = m[0], d1 = m[1];
    if (d0.x == 1.f && d0.y == 0.f) {
        if (d1.y == 0.f) {
#pragma unroll
            for (int j = 0; j < NR; ++j)
                if (j & (1 << B)) { v[j].x *= d1.x; v[j].y *= d1.x; }
        } else {
#pragma unroll
            for (int j = 0; j < NR; ++j)
                if (j & (1 << B)) v[j] = cmul(d1, v[j]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NR; ++j) v[j] = cmul((j & (1 << B)) ? d1 : d0, v[j]);
    }
}

template <int B>
__device__ __forceinline__ void rx1(RegArr& v, const float2* __restrict__ m) {
    const float2 a = m[0], b = m[1];
    if (a.x == 1.f && a.y == 0.f && b.x == 1.f && b.y == 0.f) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j & (1 << B)) continue;
            const float2 t = v[j]; v[j] = v[j | (1 << B)]; v[j | (1 << B)] = t;
        }
    } else {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j & (1 << B)) continue;
            const float2 x = v[j], y = v[j | (1 << B)];
            v[j] = cmul(a, y);
            v[j | (1 << B)] = cmul(b, x);
        }
    }
}

struct RCX {   // control bit A, target bit B
    template <int A, int B>
    __device__ __forceinline__ static void run(RegArr& v, const float2*) {
#pragma unroll
        for (int j = 0; j < NR; ++j)
            if ((j & (1 << A)) && !(j & (1 << B))) { const float2 t = v[j]; v[j] = v[j | (1 << B)]; v[j | (1 << B)] = t; }
    }
};
struct RCZ {
    template <int A, int B>
    __device__ __forceinline__ static void run(RegArr& v, const float2*) {
#pragma unroll
        for (int j = 0; j < NR; ++j)
            if ((j & (1 << A)) && (j & (1 << B))) { v[j].x = -v[j].x; v[j].y = -v[j].y; }
    }
};
struct RSWAP {
    template <int A, int B>
    __device__ __forceinline__ static void run(RegArr& v, const float2*) {
#pragma unroll
        for (int j = 0; j < NR; ++j)
            if ((j & (1 << A)) && !(j & (1 << B))) {
                const int k = (j ^ (1 << A)) | (1 << B);
                const float2 t = v[j]; v[j] = v[k]; v[k] = t;
            }
    }
};
struct RM2 {   // monomial on local index 2*bit(A) + bit(B); perm passed in `perm`
    template <int A, int B>
    __device__ __forceinline__ static void run(RegArr& v, const float2* __restrict__ m, uint32_t perm) {
        const float2 d[4] = {m[0], m[1], m[2], m[3]};
        const int p0 = perm & 3, p1 = (perm >> 2) & 3, p2 = (perm >> 4) & 3, p3 = (perm >> 6) & 3;
        const bool real = d[0].y == 0.f && d[1].y == 0.f && d[2].y == 0.f && d[3].y == 0.f;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if ((j & (1 << A)) || (j & (1 << B))) continue;
            const int idx[4] = {j, j | (1 << B), j | (1 << A), j | (1 << A) | (1 << B)};
            const float2 x[4] = {v[idx[0]], v[idx[1]], v[idx[2]], v[idx[3]]};
            const float2 y0 = pick4(x, p0), y1 = pick4(x, p1), y2 = pick4(x, p2), y3 = pick4(x, p3);
            if (real) {
                v[idx[0]] = make_float2(d[0].x * y0.x, d[0].x * y0.y);
                v[idx[1]] = make_float2(d[1].x * y1.x, d[1].x * y1.y);
                v[idx[2]] = make_float2(d[2].x * y2.x, d[2].x * y2.y);
                v[idx[3]] = make_float2(d[3].x * y3.x, d[3].x * y3.y);
            } else {
                v[idx[0]] = cmul(d[0], y0); v[idx[1]] = cmul(d[1], y1);
                v[idx[2]] = cmul(d[2], y2); v[idx[3]] = cmul(d[3], y3);
            }
        }
    }
};

#define PTSBE_C1(F, B) case B: F<B>(v, m); break;
#define PTSBE_C2(K, A, B) case (A) * 8 + (B): K::template run<A, B>(v, m); break;

#define PTSBE_C2P(K, A, B) case (A) * 8 + (B): K::template run<A, B>(v, m, perm); break;
template <class K>
__device__ __forceinline__ void dispatch2p(RegArr& v, int a, int b, const float2* m, uint32_t perm) {
    switch (a * 8 + b) {
        PTSBE_C2P(K, 0, 1) PTSBE_C2P(K, 0, 2) PTSBE_C2P(K, 0, 3)
        PTSBE_C2P(K, 1, 0) PTSBE_C2P(K, 1, 2) PTSBE_C2P(K, 1, 3)
        PTSBE_C2P(K, 2, 0) PTSBE_C2P(K, 2, 1) PTSBE_C2P(K, 2, 3)
        PTSBE_C2P(K, 3, 0) PTSBE_C2P(K, 3, 1) PTSBE_C2P(K, 3, 2)
        default: break;
    }
}

template <class K>
__device__ __forceinline__ void dispatch2(RegArr& v, int a, int b, const float2* m) {
    switch (a * 8 + b) {
        PTSBE_C2(K, 0, 1) PTSBE_C2(K, 0, 2) PTSBE_C2(K, 0, 3)
        PTSBE_C2(K, 1, 0) PTSBE_C2(K, 1, 2) PTSBE_C2(K, 1, 3)
        PTSBE_C2(K, 2, 0) PTSBE_C2(K, 2, 1) PTSBE_C2(K, 2, 3)
        PTSBE_C2(K, 3, 0) PTSBE_C2(K, 3, 1) PTSBE_C2(K, 3, 2)
        default: break;
    }
}
static_assert(kRegBits == 4, "dispatch tables are written for 4 register bits");

__device__ __forceinline__ void apply_reg(RegArr& v, uint8_t kind, int b0, int b1, const float2* m, uint32_t perm = 0) {
    switch (kind) {
    case DOP_M2: dispatch2p<RM2>(v, b0, b1, m, perm); break;
    case DOP_G1: switch (b0) { PTSBE_C1(rg1, 0) PTSBE_C1(rg1, 1) PTSBE_C1(rg1, 2) PTSBE_C1(rg1, 3) default: break; } break;
    case DOP_D1: switch (b0) { PTSBE_C1(rd1, 0) PTSBE_C1(rd1, 1) PTSBE_C1(rd1, 2) PTSBE_C1(rd1, 3) default: break; } break;
    case DOP_X1: switch (b0) { PTSBE_C1(rx1, 0) PTSBE_C1(rx1, 1) PTSBE_C1(rx1, 2) PTSBE_C1(rx1, 3) default: break; } break;
    case DOP_CX: dispatch2<RCX>(v, b0, b1, m); break;
    case DOP_CZ: dispatch2<RCZ>(v, b0, b1, m); break;
    case DOP_SWAP: dispatch2<RSWAP>(v, b0, b1, m); break;
    default: break;
    }
}

// Shared-memory layout of the register-blocked kernel: tile index l lives at sw(l), an XOR swizzle
// that folds bits 5..9 and 10..14 into the bank bits 0..4. It is linear over GF(2), so the slot
// address of a thread is sw(lane base) ^ sw(register offset). The planner orders each group's
// lane positions so that the 32 lanes of a warp land on 32 distinct banks (distinct residues of
// their positions mod 5).
__device__ __forceinline__ uint32_t sw(uint32_t l) { return l ^ (((l >> 5) ^ (l >> 10)) & 31u); }

__device__ __forceinline__ uint32_t slot_addr(uint32_t sbase, const uint32_t (&sbit)[kRegBits], int j) {
    uint32_t o = sbase;
#pragma unroll
    for (int b = 0; b < kRegBits; ++b)
        if (j & (1 << b)) o ^= sbit[b];
    return o;
}

// Per-CTA instruction stream of one stage (built by thread 0 while the other threads load the
// tile): x = opcode | rb0 << 8 | rb1 << 12 | perm << 16, y = matrix offset / group.
enum : uint32_t { OPC_GROUP = 16, OPC_END = 18 };
constexpr int kMaxStream = 1024;

__device__ __forceinline__ uint2 instr(uint32_t opc, uint32_t rb0, uint32_t rb1, uint32_t perm, uint32_t y) {
    return make_uint2(opc | (rb0 << 8) | (rb1 << 12) | (perm << 16), y);
}

// General 4x4 on register bits (ba, bb): every quad lies in one thread's own slots, so the caller
// parks its registers in those slots, this updates the quads there, and the caller reloads.
__device__ __noinline__ void own_slots_g2(float2* tile, uint32_t sbase, const uint32_t* sbits, int ba, int bb,
                                          const float2* __restrict__ m) {
    uint32_t sb[kRegBits];
    for (int b = 0; b < kRegBits; ++b) sb[b] = sbits[b];
    for (int j = 0; j < NR; ++j) {
        if ((j >> ba) & 1 || (j >> bb) & 1) continue;
        const int idx[4] = {j, j | (1 << bb), j | (1 << ba), j | (1 << ba) | (1 << bb)};
        float2 x[4];
        uint32_t ad[4];
        for (int l = 0; l < 4; ++l) {
            uint32_t o = sbase;
            for (int b = 0; b < kRegBits; ++b) if (idx[l] & (1 << b)) o ^= sb[b];
            ad[l] = o;
            x[l] = tile[o];
        }
        for (int r = 0; r < 4; ++r) {
            float2 acc = cmul(m[4 * r], x[0]);
            for (int l = 1; l < 4; ++l) {
                const float2 t = cmul(m[4 * r + l], x[l]);
                acc.x += t.x; acc.y += t.y;
            }
            tile[ad[r]] = acc;
        }
    }
}

__device__ void tile_load_sw(float2* tile, const float2* __restrict__ g, int tb, int lb, const uint32_t* hi, uint64_t outer) {
    const uint32_t nv = 1u << (tb - 1);
    for (uint32_t v = threadIdx.x; v < nv; v += blockDim.x) {
        const uint32_t l = 2 * v;
        const float4 x = __ldg(reinterpret_cast<const float4*>(g + gidx(l, lb, hi, outer)));
        tile[sw(l)] = make_float2(x.x, x.y);
        tile[sw(l + 1)] = make_float2(x.z, x.w);
    }
}

__device__ void tile_store_sw(const float2* tile, float2* g, int tb, int lb, const uint32_t* hi, uint64_t outer, float scale) {
    const uint32_t nv = 1u << (tb - 1);
    for (uint32_t v = threadIdx.x; v < nv; v += blockDim.x) {
        const uint32_t l = 2 * v;
        const float2 p = tile[sw(l)], q = tile[sw(l + 1)];
        float4 x = make_float4(p.x, p.y, q.x, q.y);
        if (scale != 1.0f) { x.x *= scale; x.y *= scale; x.z *= scale; x.w *= scale; }
        *reinterpret_cast<float4*>(g + gidx(l, lb, hi, outer)) = x;
    }
}

// Resumable builder of the stage's instruction stream for one state (thread 0 only). Emits at most
// kMaxStream - 1 instructions, then OPC_MORE when ops remain.
enum : uint32_t { OPC_MORE = 19 };
struct StreamState {
    uint32_t op, e, ee, g;
    int started;
};

__device__ __noinline__ void build_stream(const EvolveArgs& a, const DevStage& st, const DevGroup* sg, StreamState& S, uint2* out) {
    int ip = 0;
    const uint32_t ng = st.group_end - st.group_begin;
    if (!S.started) {
        S.started = 1;
        while (S.g < ng && sg[S.g].op_end <= S.op) ++S.g;
        if (S.g >= ng || S.op >= st.op_end) { out[ip++] = instr(OPC_END, 0, 0, 0, 0); return; }
        out[ip++] = instr(OPC_GROUP, 0, 0, 0, S.g);
    }
    for (; S.op < st.op_end; ++S.op) {
        if (ip > kMaxStream - 24) { out[ip++] = instr(OPC_MORE, 0, 0, 0, 0); return; }
        const uint32_t op = S.op;
        if (op >= sg[S.g].op_end) {
            while (op >= sg[S.g].op_end) ++S.g;
            out[ip++] = instr(OPC_GROUP, 0, 0, 0, S.g);
        }
        const DevOp o = a.ops[op];
        const uint8_t* rbit = sg[S.g].rbit;
        if (o.kind == DOP_NOISE) {
            uint32_t k = 0;
            if (S.e < S.ee && a.ent_site[S.e] == o.site) { k = a.ent_k[S.e]; ++S.e; }
            const uint32_t u0 = a.chans[o.ch].micro_off[k], u1 = a.chans[o.ch].micro_off[k + 1];
            for (uint32_t u = u0; u < u1; ++u) {
                const DevMicro mi = a.micro[u];
                if (mi.kind == DOP_NOP) continue;
                const uint32_t r0 = rbit[st.pos[mi.operand == 1 ? o.q1 : o.q0]], r1 = rbit[st.pos[o.q1]];
                out[ip++] = instr(mi.kind, r0, r1, 0, mi.mat);
            }
        } else {
            const uint32_t r0 = rbit[st.pos[o.q0]], r1 = rbit[st.pos[o.q1]];
            if (o.fend != 0 && (S.e >= S.ee || a.ent_site[S.e] >= o.fsite1)) {
                if (o.fkind != DOP_NOP) out[ip++] = instr(o.fkind, r0, r1, o.fperm, o.fmat);
                S.op = o.fend - 1;
            } else if (o.kind != DOP_NOP) {
                out[ip++] = instr(o.kind, r0, r1, 0, o.mat);
            }
        }
    }
    out[ip++] = instr(OPC_END, 0, 0, 0, 0);
}

__global__ void __launch_bounds__(1024, 1) k_evolve_rb(EvolveArgs a, int stage_idx, int last, const uint32_t* __restrict__ nodes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ DevStage st;
    __shared__ uint32_t sbits_sh[kRegBits];
    __shared__ StreamState S;
    __shared__ double red[33];
    const int tb = a.tb, lb = a.lb, n = a.n, ob = n - tb;
    float2* tile = reinterpret_cast<float2*>(smem);
    uint32_t* hi = reinterpret_cast<uint32_t*>(tile + (1u << tb));
    // instruction stream after the hi table, 16-byte aligned (the hi table is 4 bytes when tb == lb)
    uint2* stream = reinterpret_cast<uint2*>(smem + ((((size_t)8 << tb) + ((size_t)4 << (tb - lb)) + 15) & ~(size_t)15));
    if (threadIdx.x == 0) st = a.stages[stage_idx];
    __syncthreads();
    const DevGroup* sg = a.groups + st.group_begin;   // this stage's register groups (global, broadcast reads)
    for (uint32_t i = threadIdx.x; i < (1u << (tb - lb)); i += blockDim.x) hi[i] = a.hi[st.hi_off + i];
    const uint32_t node = nodes[blockIdx.y];
    const uint32_t tau = blockIdx.x;
    uint64_t outer = 0;
    for (int b = 0; b < ob; ++b)
        if ((tau >> b) & 1u) outer |= 1ull << st.outer_q[b];
    float2* g = a.states + ((size_t)node << n);
    const uint32_t src = stage_idx == (int)a.node_sstage[node] ? a.node_src[node] : node;
    const float2* gin = a.states_in + ((size_t)src << n);
    const uint32_t start = st.op_begin;
    __syncthreads();
    if (threadIdx.x == 0) {
        S.op = start; S.g = 0; S.started = 0;
        S.e = a.node_ebeg[node]; S.ee = a.node_eend[node];
        while (S.e < S.ee && a.site_op[a.ent_site[S.e]] < start) ++S.e;
        build_stream(a, st, sg, S, stream);
    }
    if (a.node_fresh[node] && stage_idx == 0) {
        for (uint32_t l = threadIdx.x; l < (1u << tb); l += blockDim.x)
            tile[l] = make_float2((l == 0 && tau == 0) ? 1.0f : 0.0f, 0.0f);   // sw(0) == 0
    } else {
        tile_load_sw(tile, gin, tb, lb, hi, outer);
    }
    __syncthreads();

    RegArr v;
    uint32_t sbase = 0;
    uint32_t sbit[kRegBits];
#pragma unroll
    for (int b = 0; b < kRegBits; ++b) sbit[b] = 0;
    bool loaded = false;
    for (int ip = 0;; ++ip) {
        const uint2 ins = stream[ip];
        const uint32_t opc = ins.x & 0xFFu;
        if (opc == OPC_MORE) {                  // refill the stream; registers stay loaded
            __syncthreads();
            if (threadIdx.x == 0) build_stream(a, st, sg, S, stream);
            __syncthreads();
            ip = -1;
            continue;
        }
        if (opc == OPC_GROUP || opc == OPC_END) {
            if (loaded) {
                asm volatile("" : "+r"(sbase));
#pragma unroll
                for (int j = 0; j < NR; ++j) tile[slot_addr(sbase, sbit, j)] = v[j];
                loaded = false;
            }
            __syncthreads();
            if (opc == OPC_END) break;
            {
                const DevGroup& G = sg[ins.y];
                uint32_t base = 0;
                for (int i = 0; i < tb - kRegBits; ++i) base |= ((threadIdx.x >> i) & 1u) << G.lane_pos[i];
                sbase = sw(base);
#pragma unroll
                for (int b = 0; b < kRegBits; ++b) sbit[b] = sw(1u << G.reg_pos[b]);
                if (threadIdx.x == 0) {
#pragma unroll
                    for (int b = 0; b < kRegBits; ++b) sbits_sh[b] = sbit[b];
                }
                __syncthreads();
            }
#pragma unroll
            for (int j = 0; j < NR; ++j) v[j] = tile[slot_addr(sbase, sbit, j)];
            loaded = true;
            continue;
        }
        const int rb0 = (ins.x >> 8) & 0xF, rb1 = (ins.x >> 12) & 0xF;
        if (opc == DOP_G2) {
#pragma unroll
            for (int j = 0; j < NR; ++j) tile[slot_addr(sbase, sbit, j)] = v[j];
            own_slots_g2(tile, sbase, sbits_sh, rb0, rb1, a.mats + ins.y);
#pragma unroll
            for (int j = 0; j < NR; ++j) v[j] = tile[slot_addr(sbase, sbit, j)];
        } else {
            apply_reg(v, (uint8_t)opc, rb0, rb1, a.mats + ins.y, (ins.x >> 16) & 0xFF);
        }
    }

    if (!last) {
        tile_store_sw(tile, g, tb, lb, hi, outer, 1.0f);
        return;
    }
    const double part = cta_sum(tile_norm_partial(tile, tb), red);
    if (ob == 0) {
        const double w = a.wmix[node] * part;
        const bool null = !(part > 0.0) || w < 1e-6 * a.qalpha[node];
        const float scale = null ? 0.0f : (float)(1.0 / sqrt(part));
        tile_store_sw(tile, g, tb, lb, hi, outer, scale);
        if (threadIdx.x == 0) {
            if (a.weights) a.weights[node] = w;
            if (a.status) a.status[node] = null ? 1 : 0;
        }
    } else {
        tile_store_sw(tile, g, tb, lb, hi, outer, 1.0f);
        if (threadIdx.x == 0) a.part[((size_t)node << ob) + tau] = part;
    }
}

// Default kernel choice for tile passes (measured on GB300, see the design notes).

int evolve_threads(int tb) {
    const int amps = 1 << tb;
    int t = amps / 16;
    if (t < 64) t = 64;
    if (t > 1024) t = 1024;
    return t;
}

}  // namespace

size_t evolve_smem_bytes(int tb, int lb) { return ((size_t)8 << tb) + ((size_t)4 << (tb - lb)); }
size_t evolve_frame_program_bytes() { return sizeof(frame::Program); }
size_t evolve_frame_smem_bytes(int tb, int lb) {
    return frame_tab_offset(tb, lb) + (size_t)frame::kMaxTabs * frame::kTabSize * sizeof(float2);
}
size_t evolve_frame_small_smem_bytes(int sbits, int tb, int lb) {
    // tables of a small stage index at most sbits tile bits (rows outside the support are dropped)
    return frame_tab_offset_amps(1u << sbits, tb, lb) + ((size_t)frame::kMaxTabs << sbits) * sizeof(float2);
}
size_t evolve_rb_smem_bytes(int tb, int lb) { return ((evolve_smem_bytes(tb, lb) + 15) & ~(size_t)15) + 8 * (size_t)kMaxStream; }

void launch_evolve_stage(const EvolveArgs& a, int stage, bool last, const uint32_t* d_nodes, uint32_t n_nodes,
                         cudaStream_t s, int kernel) {
    if (n_nodes == 0) return;
    static_assert(sizeof(frame::Builder) % 4 == 0 && sizeof(frame::Step) % 4 == 0 && sizeof(frame::Factor) % 4 == 0,
                  "program copies move 4-byte words");
    // thread-safe once: two contexts may be driven from two host threads
    static const bool configured = [&] {
        PTSBE_CUDA(cudaFuncSetAttribute(k_evolve_stage, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)evolve_smem_bytes(kTileMax, 1)));
        PTSBE_CUDA(cudaFuncSetAttribute(k_evolve_rb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)evolve_rb_smem_bytes(kTileMax, 1)));
        PTSBE_CUDA(cudaFuncSetAttribute(k_evolve_frame<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)evolve_frame_smem_bytes(kTileMax, 1)));
        PTSBE_CUDA(cudaFuncSetAttribute(k_evolve_frame<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)evolve_frame_small_smem_bytes(kSmallSupportBits, kTileMax, 1)));
        return true;
    }();
    (void)configured;
    const bool regs = a.tb >= kRegBits && kernel == 2;
    const bool frm = kernel == 0 || kernel == 3;
    const bool small = frm && stage == a.sparse_final_stage && a.small_bits > 0;
    if (small && a.small_bits > kSmallSupportBits) fail(PTSBE_ERR_INVALID, "small frame kernel: support too large");
    const int threads = regs ? (1 << (a.tb - kRegBits)) : small ? kFrameSmallThreads
                      : frm ? std::min(evolve_threads(a.tb), kFrameThreads) : evolve_threads(a.tb);
    const size_t smem = regs ? evolve_rb_smem_bytes(a.tb, a.lb) : small ? evolve_frame_small_smem_bytes(a.small_bits, a.tb, a.lb)
                      : frm ? evolve_frame_smem_bytes(a.tb, a.lb) : evolve_smem_bytes(a.tb, a.lb);
    const uint32_t tiles = (frm && stage == a.sparse_final_stage) ? 1u : 1u << (a.n - a.tb);
    frame::Program* progs = reinterpret_cast<frame::Program*>(a.frame_progs);
    // The per-operator kernel stages the circuit's matrices when they fit beside its tile within
    // the shared memory it was configured for (at most 32 KB of them).
    EvolveArgs ks = a;
    ks.stage_mats = 0;
    if (!regs && !frm && a.n_mats <= 4096u &&
        evolve_stage_mats_offset(a.tb, a.lb) + (size_t)a.n_mats * sizeof(float2) <= evolve_smem_bytes(kTileMax, 1))
        ks.stage_mats = a.n_mats;
    if (frm && !progs) fail(PTSBE_ERR_INVALID, "frame kernel launched without program workspace");
    for (uint32_t b = 0; b < n_nodes; b += 65535) {
        const uint32_t cnt = (n_nodes - b) < 65535u ? (n_nodes - b) : 65535u;
        if (regs)
            k_evolve_rb<<<dim3(tiles, cnt), threads, smem, s>>>(a, stage, last ? 1 : 0, d_nodes + b);
        else if (small)
            k_evolve_frame<true><<<dim3(tiles, cnt), threads, smem, s>>>(a, stage, last ? 1 : 0, d_nodes + b, progs + b);
        else if (frm)
            k_evolve_frame<false><<<dim3(tiles, cnt), threads, smem, s>>>(a, stage, last ? 1 : 0, d_nodes + b, progs + b);
        else
            k_evolve_stage<<<dim3(tiles, cnt), threads,
                             ks.stage_mats ? evolve_stage_mats_offset(a.tb, a.lb) + (size_t)ks.stage_mats * sizeof(float2) : smem,
                             s>>>(ks, stage, last ? 1 : 0, d_nodes + b);
        PTSBE_CUDA(cudaGetLastError());
        count_launch();
    }
}

void launch_zero_states(void* base, uint64_t state_bytes, uint64_t prefix, uint32_t count, int n_sm, cudaStream_t s) {
    if (prefix == 0 || count == 0) return;
    if ((uintptr_t)base % 16 || state_bytes % 16 || prefix % kFillChunk || prefix > state_bytes)
        fail(PTSBE_ERR_INVALID, "zero fill: unaligned base, or a prefix that is not whole 4 KB chunks of the state");
    const uint64_t chunks = (uint64_t)count * (prefix / kFillChunk);
    const uint64_t grid = std::min<uint64_t>((chunks + 31) / 32, (uint64_t)std::max(n_sm, 1));
    k_zero_states<<<(uint32_t)grid, 32, 0, s>>>(reinterpret_cast<unsigned char*>(base), state_bytes, prefix, chunks);
    PTSBE_CUDA(cudaGetLastError());
    count_launch();
}

void launch_frame_program(const EvolveArgs& a, int stage, const uint32_t* d_nodes, uint32_t n_nodes, cudaStream_t s,
                          int sets_per_warp) {
    if (n_nodes == 0) return;
    frame::Program* progs = reinterpret_cast<frame::Program*>(a.frame_progs);
    if (!progs) fail(PTSBE_ERR_INVALID, "frame program prepass launched without workspace");
    const uint32_t ctas = (n_nodes + kProgSets - 1) / kProgSets;
    if (sets_per_warp == 4)
        k_frame_program<4><<<ctas, 32 * (kProgSets / 4), 0, s>>>(a, stage, d_nodes, n_nodes, progs);
    else if (sets_per_warp == 8)
        k_frame_program<8><<<ctas, 32 * (kProgSets / 8), 0, s>>>(a, stage, d_nodes, n_nodes, progs);
    else
        k_frame_program<16><<<ctas, 32 * (kProgSets / 16), 0, s>>>(a, stage, d_nodes, n_nodes, progs);
    PTSBE_CUDA(cudaGetLastError());
    count_launch();
}

void launch_evolve_reduce(const EvolveArgs& a, uint32_t count, float* d_scale, cudaStream_t s) {
    if (count == 0) return;
    k_evolve_reduce<<<count, 256, 0, s>>>(a, d_scale);
    PTSBE_CUDA(cudaGetLastError());
    count_launch();
}

void launch_evolve_finalize(const EvolveArgs& a, uint32_t count, float* d_scale, cudaStream_t s, bool one_tile_too) {
    // a one-tile state's norm is fused into the tile kernels of the other evolve kernels
    if ((a.n == a.tb && !one_tile_too) || count == 0) return;
    k_evolve_reduce<<<count, 256, 0, s>>>(a, d_scale);
    PTSBE_CUDA(cudaGetLastError());
        count_launch();
    const uint64_t nv = 1ull << (a.n - 1);
    uint32_t blocks = (uint32_t)((nv + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    for (uint32_t b = 0; b < count; b += 65535) {
        const uint32_t cnt = (count - b) < 65535u ? (count - b) : 65535u;
        k_evolve_scale<<<dim3(blocks, cnt), 256, 0, s>>>(a.states + ((size_t)b << a.n), a.n, d_scale + b);
        PTSBE_CUDA(cudaGetLastError());
        count_launch();
    }
}

}  // namespace ptsbe
