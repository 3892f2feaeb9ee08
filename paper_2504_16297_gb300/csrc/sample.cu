// Batched shot sampling (Sec. 3: all m_alpha shots of a prepared state are drawn at once).
//
// For a state with P_i = |psi_i|^2 and inclusive prefix C, T = C[last], shot j draws
// u = U53(Philox(seed; j_lo, j_hi, alpha, 2)) and returns the smallest i with u*T < C[i]. The
// prefix is kept in 2^-62 fixed point (64-bit integers): exact sums on the integer pipe, and
// u*T = floor(m T / 2^53) exactly for u = m / 2^53.
//
// n <= 17: the whole CDF is held on chip. A thread-block cluster of CL = 2^(n-14) CTAs (one CTA
// when n <= 14) owns one state: CTA r builds the prefix of amplitudes [r*2^sb, (r+1)*2^sb) in its
// shared memory, the cluster exchanges slice totals over distributed shared memory (DSMEM), and
// every CTA holds a guide table of the whole CDF (the first index past each of 4,096 cuts
// floor(b T / 4096)). A shot's target lies between the cuts named by the top 12 bits of its
// uniform, so the guide narrows each search to the entries between two cuts (through DSMEM when
// remote); each thread runs four searches interleaved. Shots are written in order, so the output
// stream is coalesced. Heavy states are split into several work items (shot ranges), each
// rebuilding the CDF.
//
// n > 17: the CDF is built in global workspace (block prefixes, block offsets) and searched there.
#include <algorithm>
#include <cooperative_groups.h>
#include <mutex>

#include "fixed_point.cuh"
#include "internal.h"
#include "philox.h"

namespace cg = cooperative_groups;

namespace ptsbe {

namespace {

constexpr int kSliceBits = 14;   // per-CTA CDF slice: 2^14 doubles = 128 KiB
constexpr int kSampleThreads = 1024;

// Padded shared-memory address of CDF entry l when every thread owns K = 2^kb consecutive
// entries: one pad slot per K entries keeps a warp's accesses on distinct banks.
__device__ __forceinline__ uint32_t paddr(uint32_t l, int kb) { return l + (l >> kb); }

// log2 of the CDF entries each thread owns for a slice of 2^cb entries (0 when the slice is
// smaller than the CTA).
__device__ __forceinline__ int entries_log2(int cb) {
    const int tl = 31 - __clz(blockDim.x);
    return cb > tl ? cb - tl : 0;
}

// Stage 1 of a slice prefix: P_i in fixed point into cdf (padded layout); thread t owns entries
// [t*K, (t+1)*K) and sums them; the thread sums are scanned across the CTA. Returns the thread's
// exclusive offset.
__device__ fx slice_stage1(const float2* __restrict__ amps, int cb, fx* cdf, fx* red) {
    const uint32_t count = 1u << cb;
    const int kb = entries_log2(cb);
    const uint32_t K = 1u << kb;
    const uint32_t l0 = threadIdx.x * K;
    const bool mine = l0 < count;
    fx tot = 0;
    if (mine) {
        if (K == 1) {
            const fx p = fx_prob(amps[l0]);
            cdf[paddr(l0, kb)] = p;
            tot = p;
        } else {
            for (uint32_t i = 0; i < K; i += 2) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(amps + l0 + i));
                const fx p0 = fx_prob(make_float2(v.x, v.y));
                const fx p1 = fx_prob(make_float2(v.z, v.w));
                cdf[paddr(l0 + i, kb)] = p0;
                cdf[paddr(l0 + i + 1, kb)] = p1;
                tot += p0 + p1;
            }
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    fx x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const fx y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const fx prev = __shfl_up_sync(0xffffffffu, x, 1);   // inclusive sum of the lanes before
    if (lane == 31) red[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        fx acc = 0;
        for (int i = 0; i < nw; ++i) { const fx t = red[i]; red[i] = acc; acc += t; }
    }
    __syncthreads();
    return red[w] + (lane == 0 ? 0ull : prev);
}

// Inclusive fixed-point prefix of |psi|^2 over 2^cb amplitudes into cdf. Returns the last entry.
__device__ fx build_prefix(const float2* __restrict__ amps, int cb, fx* cdf, fx* red) {
    const int kb = entries_log2(cb);
    const uint32_t K = 1u << kb, l0 = threadIdx.x * K;
    fx run = slice_stage1(amps, cb, cdf, red);
    if (l0 < (1u << cb))
        for (uint32_t i = 0; i < K; ++i) {
            run += cdf[paddr(l0 + i, kb)];
            cdf[paddr(l0 + i, kb)] = run;
        }
    __syncthreads();
    return cdf[paddr((1u << cb) - 1, kb)];
}

// smallest l in [0, 2^cb) with t < cdf[l] (the last index if none)
constexpr int kGuideBits = 12;
constexpr int kGuide = 1 << kGuideBits;
constexpr int kShotIlp = 4;

// Guide cut b < kGuide of a CDF with total T: floor(b T / kGuide). A shot whose 53-bit uniform has
// top bits b has floor(u T) in [cut b, cut b+1], so its answer lies in [guide[b], guide[b+1]].
__device__ __forceinline__ fx fx_cut(uint32_t b, fx T) { return __umul64hi((fx)b << (64 - kGuideBits), T); }

template <int CL>
__global__ void __launch_bounds__(kSampleThreads, 1) k_sample_cluster(SampleArgs a, const SampleItem* __restrict__ items, int sb) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ fx red[33];
    __shared__ fx endv[CL];
    __shared__ uint32_t guide[kGuide + 1];   // first state index with C > cut b
    fx* cdf = reinterpret_cast<fx*>(smem);
    int rank = 0;
    if constexpr (CL > 1) rank = (int)cg::this_cluster().block_rank();
    const SampleItem it = items[blockIdx.x / CL];
    const uint32_t nth = blockDim.x;
    const int kb = entries_log2(sb);
    const uint64_t nshots = it.j1 - it.j0;
    if (a.status && a.status[it.state]) {      // null branch: sentinel outcomes
        for (uint64_t k = (uint64_t)rank * nth + threadIdx.x; k < nshots; k += (uint64_t)CL * nth)
            a.bits[it.out0 + k] = 0xFFFFFFFFu;
        return;
    }
    const float2* amps = a.states + ((size_t)it.state << a.n) + ((size_t)rank << sb);
    const fx local_total = build_prefix(amps, sb, cdf, red);
    fx T;
    if constexpr (CL > 1) {
        cg::cluster_group cluster = cg::this_cluster();
        cluster.sync();
        if (threadIdx.x == 0) {
            fx off = 0, my_off = 0;
            for (int r = 0; r < CL; ++r) {
                const fx* rc = cluster.map_shared_rank(cdf, r);
                const fx tot_r = rc[paddr((1u << sb) - 1, kb)];
                if (r == rank) my_off = off;
                endv[r] = off + tot_r;     // == the remote last entry after its own offset add
                off = endv[r];
            }
            red[32] = my_off;
        }
        cluster.sync();                    // everyone has read the raw slice totals
        const fx my_off = red[32];
        if (my_off != 0)
            for (uint32_t l = threadIdx.x; l < (1u << sb); l += nth) cdf[paddr(l, kb)] += my_off;
        __syncthreads();
        T = endv[CL - 1];
    } else {
        T = local_total;
        if (threadIdx.x == 0) endv[0] = local_total;
        __syncthreads();
    }
    // Guide over the whole CDF: each CTA resolves the cuts that fall in its slice (local search),
    // then copies the others' entries over DSMEM, so every CTA holds the full table. Every cut
    // lies in [0, T), so when T > 0 each is resolved by exactly one slice.
    const uint32_t last = (1u << a.n) - 1;
    const uint32_t slast = (1u << sb) - 1;
    {
        const fx st_b = rank == 0 ? 0ull : endv[rank - 1], en_b = endv[rank];
        for (uint32_t b = threadIdx.x; b < (uint32_t)kGuide; b += nth) {
            const fx thr = fx_cut(b, T);
            if (!(thr >= st_b && thr < en_b)) continue;
            uint32_t lo = 0, hi = slast;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (thr < cdf[paddr(mid, kb)]) hi = mid; else lo = mid + 1;
            }
            guide[b] = ((uint32_t)rank << sb) | lo;
        }
        if (threadIdx.x == 0) guide[kGuide] = last;
    }
    if constexpr (CL > 1) {
        cg::cluster_group cluster = cg::this_cluster();
        cluster.sync();
        for (uint32_t b = threadIdx.x; b < (uint32_t)kGuide; b += nth) {
            const fx thr = fx_cut(b, T);
            int r = 0;
            while (r < CL - 1 && !(thr < endv[r])) ++r;
            if (r != rank) guide[b] = cluster.map_shared_rank(guide, r)[b];
        }
    }
    __syncthreads();
    // Shots k, k + stride, ... : kShotIlp of them per thread at a time. A shot's target floor(u T)
    // lies between the cuts of the bucket named by the top bits of its uniform, so its answer is in
    // [guide[b], guide[b+1]]: resolved from the local guide when that range is one index, else by a
    // search of those entries (through DSMEM for remote slices).
    const uint64_t stride = (uint64_t)CL * nth;
    for (uint64_t k0 = (uint64_t)rank * nth + threadIdx.x; k0 < nshots; k0 += kShotIlp * stride) {
        uint32_t lo[kShotIlp], hi[kShotIlp];
        fx tq[kShotIlp];
#pragma unroll
        for (int q = 0; q < kShotIlp; ++q) {
            const uint64_t k = k0 + q * stride;
            lo[q] = hi[q] = last;
            tq[q] = 0;
            if (k >= nshots) continue;
            const uint64_t j = it.j0 + k;
            const Philox4 x = philox4x32_10((uint32_t)j, (uint32_t)(j >> 32), it.alpha, it.dom,
                                            (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
            const uint64_t m = u53_bits(x.x[0], x.x[1]);
            tq[q] = fx_target(m, T);
            if (!(tq[q] < T)) continue;                  // only for T = 0
            const uint32_t b = (uint32_t)(m >> (53 - kGuideBits));
            lo[q] = guide[b];
            hi[q] = guide[b + 1];
        }
        while (true) {
            bool any = false;
#pragma unroll
            for (int q = 0; q < kShotIlp; ++q) {
                if (lo[q] < hi[q]) {
                    any = true;
                    const uint32_t mid = (lo[q] + hi[q]) >> 1;
                    const int r = (int)(mid >> sb);
                    const fx* rc = cdf;
                    if constexpr (CL > 1) rc = cg::this_cluster().map_shared_rank(cdf, r);
                    if (tq[q] < rc[paddr(mid & slast, kb)]) hi[q] = mid; else lo[q] = mid + 1;
                }
            }
            if (!any) break;
        }
#pragma unroll
        for (int q = 0; q < kShotIlp; ++q) {
            const uint64_t k = k0 + q * stride;
            if (k < nshots) a.bits[it.out0 + k] = lo[q];
        }
    }
    if constexpr (CL > 1) cg::this_cluster().sync();  // keep this CTA's slice alive for remote readers
}

// ---- light states: one CTA per state, chunk prefixes ----------------------------------------------------
// For a state with few shots the full CDF is never stored. Pass 1 sums each run of cs = 2^n / 8192
// consecutive P_i (chunk totals, fixed point); a scan turns them into the prefix at every chunk
// start, P[c] (P[8192] = T). A shot finds its chunk by binary search on P and then accumulates the
// chunk's P_i from P[c] in order; the sums are exact, so the chunk's last entry equals P[c+1]. Each
// shot re-reads one chunk (cs amplitudes, mostly from L2).
constexpr int kLightChunkBits = 13;
constexpr int kLightChunks = 1 << kLightChunkBits;
constexpr int kLightThreads = 512;
constexpr int kLightGuideBits = 8;
constexpr int kLightGuide = 1 << kLightGuideBits;
constexpr int kLightPerThread = kLightChunks / kLightThreads;   // chunks scanned by one thread (16)

__device__ __forceinline__ uint32_t lpad(uint32_t c) { return c + (c >> 4); }   // bank-distinct rows of 16

__global__ void __launch_bounds__(kLightThreads, 2) k_sample_light(SampleArgs a, const SampleItem* __restrict__ items) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ fx red[33];
    __shared__ uint16_t lguide[kLightGuide + 1];
    fx* P = reinterpret_cast<fx*>(smem);               // padded: P[lpad(c)], c = 0 .. kLightChunks
    const SampleItem it = items[blockIdx.x];
    const uint64_t nshots = it.j1 - it.j0;
    if (a.status && a.status[it.state]) {
        for (uint64_t k = threadIdx.x; k < nshots; k += blockDim.x) a.bits[it.out0 + k] = 0xFFFFFFFFu;
        return;
    }
    const int n = a.n;
    const int csb = n - kLightChunkBits;                // log2 of the chunk size (2 .. 7)
    const uint32_t cs = 1u << csb;
    const float2* amps = a.states + ((size_t)it.state << n);
    // pass 1: chunk totals (two amplitudes per 16-byte load, the chunk's loads issued together)
    for (uint32_t c = threadIdx.x; c < (uint32_t)kLightChunks; c += blockDim.x) {
        const float4* v = reinterpret_cast<const float4*>(amps + ((size_t)c << csb));
        fx acc = 0;
        for (uint32_t i0 = 0; i0 < cs / 2; i0 += 8) {
            float4 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + u < cs / 2) x[u] = __ldg(v + i0 + u);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + u < cs / 2) acc += fx_prob(make_float2(x[u].x, x[u].y)) + fx_prob(make_float2(x[u].z, x[u].w));
        }
        P[lpad(c)] = acc;
    }
    __syncthreads();
    // scan: thread t owns chunks [16 t, 16 t + 16): its sum, a CTA exclusive scan of the thread
    // sums, then the chunk-start prefixes
    const uint32_t c0 = threadIdx.x * kLightPerThread;
    fx tot[kLightPerThread];
    fx mine = 0;
#pragma unroll
    for (int i = 0; i < kLightPerThread; ++i) { tot[i] = P[lpad(c0 + i)]; mine += tot[i]; }
    fx v = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const fx y = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= (uint32_t)o) v += y;
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 31) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        fx acc = 0;
        for (int i = 0; i < nw; ++i) { const fx t = red[i]; red[i] = acc; acc += t; }
        red[32] = acc;                                  // T
    }
    __syncthreads();
    fx run = red[w] + (v - mine);                       // exclusive prefix of this thread's chunks
#pragma unroll
    for (int i = 0; i < kLightPerThread; ++i) { P[lpad(c0 + i)] = run; run += tot[i]; }
    const fx T = red[32];
    if (threadIdx.x == 0) P[lpad(kLightChunks)] = T;
    __syncthreads();
    // guide: the first chunk c with cut b < P[c + 1], cut b = floor(b T / 256); a shot whose
    // uniform has top bits b has floor(u T) between cuts b and b + 1, so its chunk lies between
    // the two guide entries
    for (uint32_t b = threadIdx.x; b < (uint32_t)kLightGuide; b += blockDim.x) {
        const fx cut = __umul64hi((fx)b << (64 - kLightGuideBits), T);
        uint32_t lo = 0, hi = kLightChunks - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (cut < P[lpad(mid + 1)]) hi = mid; else lo = mid + 1;
        }
        lguide[b] = (uint16_t)lo;
    }
    if (threadIdx.x == 0) lguide[kLightGuide] = kLightChunks - 1;
    __syncthreads();
    for (uint64_t k = threadIdx.x; k < nshots; k += blockDim.x) {
        const uint64_t j = it.j0 + k;
        const Philox4 x = philox4x32_10((uint32_t)j, (uint32_t)(j >> 32), it.alpha, it.dom, (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
        const uint64_t m = u53_bits(x.x[0], x.x[1]);
        const fx t = fx_target(m, T);
        uint32_t idx = (1u << n) - 1;                   // T = 0
        if (t < T) {
            const uint32_t gb = (uint32_t)(m >> (53 - kLightGuideBits));
            uint32_t lo = lguide[gb], hi = lguide[gb + 1];   // first chunk c with t < P[c + 1]
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (t < P[lpad(mid + 1)]) hi = mid; else lo = mid + 1;
            }
            // the chunk's amplitudes, eight 16-byte loads in flight at a time, then scanned in order
            fx acc = P[lpad(lo)];
            const float4* cv = reinterpret_cast<const float4*>(amps + ((size_t)lo << csb));
            idx = (lo << csb) + cs - 1;
            bool hit = false;
            for (uint32_t i0 = 0; i0 < cs / 2 && !hit; i0 += 8) {
                float4 x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + u < cs / 2) x[u] = __ldg(cv + i0 + u);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (hit || i0 + u >= cs / 2) continue;
                    const uint32_t l0 = 2 * (i0 + u);
                    acc += fx_prob(make_float2(x[u].x, x[u].y));
                    if (t < acc) { idx = (lo << csb) + l0; hit = true; continue; }
                    if (l0 + 1 == cs - 1) continue;      // the chunk's last entry is P[lo + 1] > t
                    acc += fx_prob(make_float2(x[u].z, x[u].w));
                    if (t < acc) { idx = (lo << csb) + l0 + 1; hit = true; }
                }
            }
        }
        a.bits[it.out0 + k] = idx;
    }
}

// ---- support CDF: heavy states exported by the small sparse final evolve stage -------------------
// One CTA per shot range of an exported state. The CDF (at most 2^10 entries in increasing outcome
// order) and its outcome indices go to shared memory with a 256-entry guide over them; each shot
// is a Philox draw, the guide bucket of its top bits and a short binary search. Same shots as the
// samplers that read the stored state: only support entries can be the smallest index whose
// prefix exceeds the target, and their prefix values are the same.
constexpr int kSupportThreads = 256;
constexpr int kSupportGuideBits = 8;
constexpr int kSupportGuide = 1 << kSupportGuideBits;

__global__ void __launch_bounds__(kSupportThreads) k_sample_support(const unsigned char* __restrict__ slots, size_t slot_bytes,
                                                                    const SupportItem* __restrict__ items, uint64_t seed,
                                                                    uint32_t* bits) {
    __shared__ fx cdf[1 << kSmallSupportBits];
    __shared__ uint32_t lidx[1 << kSmallSupportBits];
    __shared__ uint16_t guide[kSupportGuide + 1];
    const SupportItem it = items[blockIdx.x];
    const unsigned char* slot = slots + (size_t)it.slot * slot_bytes;
    const SupportCdfHeader h = *reinterpret_cast<const SupportCdfHeader*>(slot);
    uint32_t* out = bits + it.out0;
    const uint64_t m = it.j1 - it.j0;
    if (h.mark_all || h.n == 0 || h.n > (1u << kSmallSupportBits)) {
        const uint32_t mark = h.mark_all ? h.mark : 0xFFFFFFFFu;
        for (uint64_t k = threadIdx.x; k < m; k += blockDim.x) out[k] = mark;
        return;
    }
    const uint32_t N = h.n;
    const fx* gc = reinterpret_cast<const fx*>(slot + sizeof(SupportCdfHeader));
    const uint32_t* gl = reinterpret_cast<const uint32_t*>(gc + N);
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) { cdf[i] = gc[i]; lidx[i] = gl[i]; }
    __syncthreads();
    const fx T = h.T;
    // guide b: the first entry r with cut b < cdf[r], cut b = floor(b T / 256); a shot whose uniform
    // has top bits b has floor(u T) between cuts b and b + 1, so its entry lies between guide b and b + 1
    for (uint32_t b = threadIdx.x; b < (uint32_t)kSupportGuide; b += blockDim.x) {
        const fx cut = __umul64hi((fx)b << (64 - kSupportGuideBits), T);
        uint32_t lo = 0, hi = N - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (cut < cdf[mid]) hi = mid; else lo = mid + 1;
        }
        guide[b] = (uint16_t)lo;
    }
    if (threadIdx.x == 0) guide[kSupportGuide] = (uint16_t)(N - 1);
    __syncthreads();
    const uint32_t last = (uint32_t)((1ull << h.nq) - 1ull);   // T = 0
    for (uint64_t k = threadIdx.x; k < m; k += blockDim.x) {
        const uint64_t j = it.j0 + k;
        const Philox4 x = philox4x32_10((uint32_t)j, (uint32_t)(j >> 32), it.alpha, kDomShot, (uint32_t)seed, (uint32_t)(seed >> 32));
        const uint64_t m53 = u53_bits(x.x[0], x.x[1]);
        const fx t = fx_target(m53, T);
        uint32_t idx = last;
        if (t < T) {
            const uint32_t gb = (uint32_t)(m53 >> (53 - kSupportGuideBits));
            uint32_t lo = guide[gb], hi = guide[gb + 1];     // smallest r with t < cdf[r]
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (t < cdf[mid]) hi = mid; else lo = mid + 1;
            }
            idx = lidx[lo];
        }
        out[k] = idx;
    }
}

// ---- n > 17: global-memory CDF -----------------------------------------------------------------------

// One CTA per block of 2^14 amplitudes: local inclusive prefix (unpadded) and block total.
__global__ void __launch_bounds__(kSampleThreads) k_block_prefix(const float2* __restrict__ amps, fx* cdf, fx* btot) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ fx red[33];
    fx* s = reinterpret_cast<fx*>(smem);
    const uint32_t b = blockIdx.x;
    const int kb = entries_log2(kSliceBits);
    const fx tot = build_prefix(amps + ((size_t)b << kSliceBits), kSliceBits, s, red);
    for (uint32_t l = threadIdx.x; l < (1u << kSliceBits); l += blockDim.x)
        cdf[((size_t)b << kSliceBits) + l] = s[paddr(l, kb)];
    if (threadIdx.x == 0) btot[b] = tot;
}

// One CTA: exclusive block offsets (per thread chunk, then across threads); writes the block end
// values bend[b] = offset[b] + btot[b].
__global__ void k_block_scan(const fx* __restrict__ btot, fx* boff, fx* bend, uint32_t nb) {
    __shared__ fx red[1024];
    const uint32_t nth = blockDim.x;
    const uint32_t per = (nb + nth - 1) / nth;
    const uint32_t b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    fx s = 0;
    for (uint32_t b = b0; b < b1; ++b) s += btot[b];
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        fx acc = 0;
        for (uint32_t i = 0; i < nth; ++i) { const fx t = red[i]; red[i] = acc; acc += t; }
    }
    __syncthreads();
    fx run = red[threadIdx.x];
    for (uint32_t b = b0; b < b1; ++b) {
        boff[b] = run;
        run += btot[b];
        bend[b] = run;
    }
}

__global__ void k_block_add(fx* cdf, const fx* __restrict__ boff) {
    const uint32_t b = blockIdx.x;
    const fx off = boff[b];
    if (off == 0) return;
    fx* c = cdf + ((size_t)b << kSliceBits);
    for (uint32_t l = threadIdx.x; l < (1u << kSliceBits); l += blockDim.x) c[l] += off;
}

__global__ void k_search_global(SampleArgs a, const fx* __restrict__ cdf, const fx* __restrict__ bend,
                                uint32_t nb, uint32_t state, uint32_t alpha, uint64_t j0, uint64_t j1, uint64_t out0,
                                uint32_t dom) {
    const fx T = bend[nb - 1];
    const bool null = a.status && a.status[state];
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < j1 - j0; k += (uint64_t)gridDim.x * blockDim.x) {
        if (null) { a.bits[out0 + k] = 0xFFFFFFFFu; continue; }
        const uint64_t j = j0 + k;
        const Philox4 x = philox4x32_10((uint32_t)j, (uint32_t)(j >> 32), alpha, dom,
                                        (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
        const fx t = fx_target(u53_bits(x.x[0], x.x[1]), T);
        uint32_t lo = 0, hi = nb - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (t < bend[mid]) hi = mid; else lo = mid + 1;
        }
        uint64_t idx;
        if (!(t < bend[lo])) {
            idx = (1ull << a.n) - 1;
        } else {
            const fx* c = cdf + ((size_t)lo << kSliceBits);
            uint32_t l = 0, h = (1u << kSliceBits) - 1;
            while (l < h) {
                const uint32_t mid = (l + h) >> 1;
                if (t < c[mid]) h = mid; else l = mid + 1;
            }
            idx = ((uint64_t)lo << kSliceBits) | l;
        }
        a.bits[out0 + k] = (uint32_t)idx;
    }
}

// Distinct outcomes among the shots of each set (the unique-shot statistic of Sec. 4). Each CTA
// takes one piece of one set's shots (sets are cut into pieces so heavy sets spread over the GPU),
// marks a bitmap of the 2^n outcomes in shared memory, and ORs its nonzero words into the set's
// bitmap in global memory; a second kernel counts each set's bits. Shots that are not outcomes
// (the null-branch sentinel) are skipped.
__global__ void k_unique_mark(const uint32_t* __restrict__ bits, const uint64_t* __restrict__ pieces, int n,
                              uint32_t* gbm) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* bm = reinterpret_cast<uint32_t*>(smem);
    const uint32_t words = (1u << n) >= 32 ? (1u << n) / 32 : 1u;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) bm[i] = 0u;
    __syncthreads();
    const uint64_t set = pieces[3 * blockIdx.x], b0 = pieces[3 * blockIdx.x + 1], b1 = pieces[3 * blockIdx.x + 2];
    const uint64_t lim = 1ull << n;
    for (uint64_t k = b0 + threadIdx.x; k < b1; k += blockDim.x) {
        const uint32_t x = bits[k];
        if ((uint64_t)x < lim) atomicOr(&bm[x >> 5], 1u << (x & 31));
    }
    __syncthreads();
    uint32_t* g = gbm + set * words;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x)
        if (bm[i]) atomicOr(&g[i], bm[i]);
}

__global__ void k_unique_count(const uint32_t* __restrict__ gbm, int n, unsigned long long* out) {
    __shared__ unsigned long long red[32];
    const uint32_t words = (1u << n) >= 32 ? (1u << n) / 32 : 1u;
    const uint32_t* g = gbm + (size_t)blockIdx.x * words;
    unsigned long long c = 0;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) c += (unsigned long long)__popc(g[i]);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (uint32_t w = 0; w < (blockDim.x + 31) / 32; ++w) t += red[w];
        out[blockIdx.x] = t;
    }
}

__global__ void k_fill(uint32_t* bits, uint64_t count, uint32_t v) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (uint64_t)gridDim.x * blockDim.x)
        bits[k] = v;
}

// Padded CDF slice of 2^sb 8-byte entries for a CTA of `threads` threads.
size_t cdf_smem_bytes(int sb, uint32_t threads) {
    const size_t count = (size_t)1 << sb;
    size_t K = count / threads;
    if (K == 0) K = 1;
    return 8 * (count + count / K + 1);
}

template <int CL>
void launch_cluster(const SampleArgs& a, const SampleItem* items, uint32_t n_items, int sb, cudaStream_t s) {
    uint32_t threads = (1u << sb) / 2;
    if (threads < 32) threads = 32;
    if (threads > kSampleThreads) threads = kSampleThreads;
    const size_t smem = cdf_smem_bytes(sb, threads);
    // thread-safe once: two contexts may be driven from two host threads
    static const bool configured = [&] {
        PTSBE_CUDA(cudaFuncSetAttribute(k_sample_cluster<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)cdf_smem_bytes(kSliceBits, kSampleThreads)));
        return true;
    }();
    (void)configured;
    for (uint32_t b = 0; b < n_items; b += (1u << 20)) {
        const uint32_t cnt = (n_items - b) < (1u << 20) ? (n_items - b) : (1u << 20);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cnt * CL);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        PTSBE_CUDA(cudaLaunchKernelEx(&cfg, k_sample_cluster<CL>, a, items + b, sb));
        count_launch();
    }
}

// Fixed scratch for ptsbe_sample_shots_noalloc: every GPU that loads the library holds these
// bytes until the process exits. In host code the name is only a stand-in for the symbol; the
// device address comes from cudaGetSymbolAddress, looked up once per device below.
// Sized for its two uses: 2^20 work items of the cluster sampler (n <= 17), or the global-memory
// CDF workspace of one 21-qubit state (n = 18 .. 21).
constexpr size_t kNoAllocMaxItems = (size_t)1 << 20;
constexpr int kNoAllocMaxQubits = 21;
constexpr size_t kNoAllocCdfBytes =
    (((size_t)1 << kNoAllocMaxQubits) + 3 * ((size_t)1 << (kNoAllocMaxQubits - kSliceBits)) + 8) * 8;
constexpr size_t kNoAllocScratchBytes =
    ((kNoAllocMaxItems * sizeof(SampleItem) > kNoAllocCdfBytes ? kNoAllocMaxItems * sizeof(SampleItem) : kNoAllocCdfBytes)
     + 255) & ~(size_t)255;
static_assert(kNoAllocScratchBytes >= kNoAllocMaxItems * sizeof(SampleItem) && kNoAllocScratchBytes >= kNoAllocCdfBytes,
              "the fixed scratch holds 2^20 work items and a 21-qubit CDF");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

}  // namespace

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }
size_t noalloc_max_items() { return kNoAllocMaxItems; }
int noalloc_max_qubits() { return kNoAllocMaxQubits; }

// Device address of the fixed scratch on `device`, which must be the current device. The first
// call on a device resolves the symbol (a driver call that is not a stream operation, so it has to
// happen before any stream capture that uses the entry point); later calls return the cached value.
void* noalloc_scratch(int device) {
    if (device < 0 || device >= kMaxDevices) fail(PTSBE_ERR_UNSUPPORTED, "device index out of range for the fixed scratch");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        PTSBE_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[device] = p;
    }
    return g_noalloc_ptr[device];
}

// Sets the dynamic shared-memory limits of every sampler kernel (the launchers do the same lazily);
// called before a launch sequence that may be captured into a CUDA graph.
void configure_samplers() {
    PTSBE_CUDA(cudaFuncSetAttribute(k_sample_cluster<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)cdf_smem_bytes(kSliceBits, kSampleThreads)));
    PTSBE_CUDA(cudaFuncSetAttribute(k_sample_cluster<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)cdf_smem_bytes(kSliceBits, kSampleThreads)));
    PTSBE_CUDA(cudaFuncSetAttribute(k_sample_cluster<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)cdf_smem_bytes(kSliceBits, kSampleThreads)));
    PTSBE_CUDA(cudaFuncSetAttribute(k_sample_cluster<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)cdf_smem_bytes(kSliceBits, kSampleThreads)));
    const size_t lsmem = ((size_t)kLightChunks + kLightChunks / 16 + 1) * sizeof(fx);
    PTSBE_CUDA(cudaFuncSetAttribute(k_sample_light, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem));
    PTSBE_CUDA(cudaFuncSetAttribute(k_block_prefix, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)cdf_smem_bytes(kSliceBits, kSampleThreads)));
}

int sample_cluster_max_qubits() { return kSliceBits + 3; }
int sample_light_max_qubits() { return kLightChunkBits + 7; }

void launch_sample_light(const SampleArgs& a, const SampleItem* d_items, uint32_t n_items, cudaStream_t s) {
    if (n_items == 0) return;
    const size_t smem = ((size_t)kLightChunks + kLightChunks / 16 + 1) * sizeof(fx);
    // thread-safe once: two contexts may be driven from two host threads
    static const bool configured = [&] {
        PTSBE_CUDA(cudaFuncSetAttribute(k_sample_light, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        return true;
    }();
    (void)configured;
    for (uint32_t b = 0; b < n_items; b += (1u << 30)) {
        const uint32_t cnt = (n_items - b) < (1u << 30) ? (n_items - b) : (1u << 30);
        k_sample_light<<<cnt, kLightThreads, smem, s>>>(a, d_items + b);
        PTSBE_CUDA(cudaGetLastError());
        count_launch();
    }
}

void launch_sample_support(const unsigned char* slots, size_t slot_bytes, const SupportItem* d_items, uint32_t n_items,
                           uint64_t seed, uint32_t* bits, cudaStream_t s) {
    for (uint32_t b = 0; b < n_items; b += (1u << 30)) {
        const uint32_t cnt = (n_items - b) < (1u << 30) ? (n_items - b) : (1u << 30);
        k_sample_support<<<cnt, kSupportThreads, 0, s>>>(slots, slot_bytes, d_items + b, seed, bits);
        PTSBE_CUDA(cudaGetLastError());
        count_launch();
    }
}

void launch_sample_cluster(const SampleArgs& a, const SampleItem* d_items, uint32_t n_items, cudaStream_t s) {
    if (n_items == 0) return;
    const int n = a.n;
    if (n <= kSliceBits) {
        // small states: at least 2 amplitudes per thread
        launch_cluster<1>(a, d_items, n_items, n < 1 ? 1 : n, s);
    } else if (n == kSliceBits + 1) {
        launch_cluster<2>(a, d_items, n_items, kSliceBits, s);
    } else if (n == kSliceBits + 2) {
        launch_cluster<4>(a, d_items, n_items, kSliceBits, s);
    } else if (n == kSliceBits + 3) {
        launch_cluster<8>(a, d_items, n_items, kSliceBits, s);
    } else {
        fail(PTSBE_ERR_UNSUPPORTED, "cluster sampler handles n <= 17");
    }
}

size_t sample_global_scratch_doubles(int n) {
    const size_t nb = (size_t)1 << (n - kSliceBits);
    return ((size_t)1 << n) + 3 * nb + 8;
}

void launch_sample_global(const SampleArgs& a, uint32_t state, uint32_t alpha, uint64_t j0, uint64_t j1,
                          uint64_t out0, cudaStream_t s, uint32_t dom) {
    const int n = a.n;
    if (j1 <= j0) return;
    const uint32_t nb = 1u << (n - kSliceBits);
    fx* cdf = a.scratch;
    fx* btot = cdf + ((size_t)1 << n);
    fx* boff = btot + nb;
    fx* bend = boff + nb;
    // thread-safe once: two contexts may be driven from two host threads
    static const bool configured = [&] {
        PTSBE_CUDA(cudaFuncSetAttribute(k_block_prefix, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)cdf_smem_bytes(kSliceBits, kSampleThreads)));
        return true;
    }();
    (void)configured;
    const float2* amps = a.states + ((size_t)state << n);
    k_block_prefix<<<nb, kSampleThreads, cdf_smem_bytes(kSliceBits, kSampleThreads), s>>>(amps, cdf, btot);
    PTSBE_CUDA(cudaGetLastError());
        count_launch();
    k_block_scan<<<1, 1024, 0, s>>>(btot, boff, bend, nb);
    PTSBE_CUDA(cudaGetLastError());
        count_launch();
    k_block_add<<<nb, 256, 0, s>>>(cdf, boff);
    PTSBE_CUDA(cudaGetLastError());
        count_launch();
    const uint64_t m = j1 - j0;
    uint32_t blocks = (uint32_t)((m + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_search_global<<<blocks, 256, 0, s>>>(a, cdf, bend, nb, state, alpha, j0, j1, out0, dom);
    PTSBE_CUDA(cudaGetLastError());
        count_launch();
}

int unique_max_qubits() { return 20; }

size_t unique_bitmap_bytes(int n) { return 4 * std::max<size_t>(1, ((size_t)1 << n) / 32); }

void launch_unique(const uint32_t* bits, const uint64_t* d_pieces, uint32_t n_pieces, uint32_t count, int n,
                   uint32_t* d_bitmaps, unsigned long long* out, cudaStream_t s) {
    if (count == 0) return;
    const size_t smem = unique_bitmap_bytes(n);
    // thread-safe once: two contexts may be driven from two host threads
    static const bool configured = [&] {
        PTSBE_CUDA(cudaFuncSetAttribute(k_unique_mark, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)unique_bitmap_bytes(20)));
        return true;
    }();
    (void)configured;
    for (uint32_t b = 0; b < n_pieces; b += 65535u) {
        const uint32_t cnt = std::min<uint32_t>(65535u, n_pieces - b);
        k_unique_mark<<<cnt, 1024, smem, s>>>(bits, d_pieces + 3 * (size_t)b, n, d_bitmaps);
        PTSBE_CUDA(cudaGetLastError());
        count_launch();
    }
    for (uint32_t b = 0; b < count; b += 65535u) {
        const uint32_t cnt = std::min<uint32_t>(65535u, count - b);
        k_unique_count<<<cnt, 256, 0, s>>>(d_bitmaps + (size_t)b * (unique_bitmap_bytes(n) / 4), n, out + b);
        PTSBE_CUDA(cudaGetLastError());
        count_launch();
    }
}

void launch_fill(uint32_t* bits, uint64_t count, uint32_t v, cudaStream_t s) {
    if (count == 0) return;
    uint32_t blocks = (uint32_t)((count + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_fill<<<blocks, 256, 0, s>>>(bits, count, v);
    PTSBE_CUDA(cudaGetLastError());
        count_launch();
}

}  // namespace ptsbe
