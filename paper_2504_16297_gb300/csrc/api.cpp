// C ABI of libptsbe: contexts, registries, workspace and the host-side scheduling of the kernels.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <functional>
#include <atomic>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <tuple>
#include <unordered_map>

#include "internal.h"
#include "philox.h"

namespace ptsbe {

void cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    const int st = (e == cudaErrorMemoryAllocation) ? PTSBE_ERR_OOM : PTSBE_ERR_CUDA;
    fail(st, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t sample_global_scratch_doubles(int n);
size_t noalloc_scratch_bytes();
size_t noalloc_max_items();
int noalloc_max_qubits();
void* noalloc_scratch(int device);

// A named range around an entry point for a timeline profiler (NVTX; nothing is recorded unless a
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint64_t> g_h2d{0};
void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void count_h2d(uint64_t bytes) { g_h2d.fetch_add(bytes, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// Optional per-kernel-class timing: CUDA events recorded on the context stream around each
// launch, plus the algorithmic bytes of that launch.
struct ClassTimer {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    std::vector<cudaEvent_t> pool;
    double ms = 0;
    uint64_t launches = 0;
    double bytes = 0;
};

// A planned batch of jobs for one persistent launch (ptsbe_batch_plan).
struct PlannedSample {
    int kind;                        // 0 light, 1 cluster, 2 global
    SampleArgs A;
    size_t item_off;                 // into the batch's item array (kinds 0, 1)
    const SampleItem* items;         // device address of the first item, set after the upload
    uint32_t n_items;
    uint32_t state, alpha;           // kind 2
    uint64_t m, out0;
};

struct Batch {
    void* dtab = nullptr;            // tables (one device allocation, uploaded at plan time)
    void* dws = nullptr;             // counters, tile norms, scales, status, sampler scratch
    QueueArgs qa{};
    std::vector<PlannedSample> samples;
    uint64_t kernels_per_run = 0;
    uint32_t* d_err = nullptr;
    cudaGraphExec_t graph = nullptr;
    size_t counter_bytes = 0;
};

}  // namespace ptsbe

using namespace ptsbe;

struct ptsbe_ctx {
    int device = -1;
    cudaStream_t stream = nullptr;
    std::string err = "no error";
    std::unordered_map<uint32_t, std::unique_ptr<Circuit>> circuits;
    std::unordered_map<uint32_t, std::unique_ptr<KSet>> sets;
    std::unordered_map<uint32_t, std::unique_ptr<Batch>> batches;
    uint32_t next_batch = 1;
    long long queue_spin_cycles = 20000000000ll;   // ~10 s at 2 GHz: a wait of the work queue gives up after this
    int64_t queue_stall_task = -1;                  // test hook (PTSBE_OPT_QUEUE_STALL_TASK)
    uint32_t next_circuit = 1, next_set = 1;
    DevBuf nodes, part, scale, items, scratch, pershot, progs, pingpong, fault, support, sitems;
    DevBuf dense_tabs, stream_status, dense_pad;          // dense passes: per-call node/override tables; status when the caller passes none
    std::vector<DevBuf> state_pool;            // dense passes without caller states: branch state buffers
    uint64_t reuse_gates_run = 0, reuse_gates_full = 0;   // last evolve call: gates applied / without prefix reuse
    uint64_t dense_launches = 0;               // last evolve call with dense passes: pass launches (set x pass)
    double dense_fma = 0;                      // ... and the FP32 multiply-adds their blocks perform
    std::vector<unsigned char> host_blob;
    std::vector<SampleItem> noalloc_items;
    bool timing = false;
    int evolve_kernel = 0;
    uint64_t light_shots = kLightShotLimit;   // states with at most this many shots: one-CTA sampler
    int prog_sets_per_warp = 8;                // frame program prepass: Kraus sets per warp (measured)
    int pershot_tile_bits = 0;                 // Algorithm 1 path: tile bits of its plan (0: kPershotTileBits)
    int split_fill = 0;                        // small sparse final stage: percent of each state zeroed beside the program prepass
    int prepass_ahead = 1;                     // one-stage frame plans: program prepass on the auxiliary stream, ahead of the context stream
    cudaStream_t aux = nullptr;                // second stream of the context (prepass ahead, zero fill), joined by events
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // Prepass ahead: uploads and the prepass of a call go to the auxiliary stream, which does not
    // wait for the context stream, so they overlap the previous call's launches. The node tables
    // and programs alternate between two lanes; a lane is rewritten only after the context stream
    // has run the evolve launch that read it (ev_used).
    cudaStream_t up = nullptr;                 // stream of uploads and table allocations (nullptr: the context stream)
    DevBuf ahead_nodes[2], ahead_progs[2];
    cudaEvent_t ev_used[2] = {nullptr, nullptr};
    bool used_recorded[2] = {false, false};
    uint32_t lane = 0;
    cudaStream_t ustream() const { return up ? up : stream; }
    int n_sm = 0;                      // streaming multiprocessors of the device
    ClassTimer timers[PTSBE_TIMER_CLASSES];

    cudaEvent_t take_event(ClassTimer& t) {
        if (!t.pool.empty()) { cudaEvent_t e = t.pool.back(); t.pool.pop_back(); return e; }
        cudaEvent_t e;
        PTSBE_CUDA(cudaEventCreate(&e));
        return e;
    }
    // Brackets a launch of kernel class `cls` on stream `s` (no-op when timing is off).
    template <class F>
    void timed_on(cudaStream_t s, int cls, double bytes, F&& launch) {
        if (!timing) { launch(); return; }
        ClassTimer& t = timers[cls];
        cudaEvent_t a = take_event(t), b = take_event(t);
        PTSBE_CUDA(cudaEventRecord(a, s));
        launch();
        PTSBE_CUDA(cudaEventRecord(b, s));
        t.pending.push_back({a, b});
        t.launches += 1;
        t.bytes += bytes;
    }
    template <class F>
    void timed(int cls, double bytes, F&& launch) { timed_on(stream, cls, bytes, static_cast<F&&>(launch)); }
    // Work on the auxiliary stream starts after everything enqueued on the context stream so far
    // (fork) and the context stream waits for it before its next launch (join).
    void fork_aux() {
        PTSBE_CUDA(cudaEventRecord(ev_fork, stream));
        PTSBE_CUDA(cudaStreamWaitEvent(aux, ev_fork, 0));
    }
    void join_aux() {
        PTSBE_CUDA(cudaEventRecord(ev_join, aux));
        PTSBE_CUDA(cudaStreamWaitEvent(stream, ev_join, 0));
    }
    void collect_timers() {
        for (ClassTimer& t : timers) {
            for (auto& ab : t.pending) {
                PTSBE_CUDA(cudaEventSynchronize(ab.second));
                float ms = 0;
                PTSBE_CUDA(cudaEventElapsedTime(&ms, ab.first, ab.second));
                t.ms += ms;
                t.pool.push_back(ab.first);
                t.pool.push_back(ab.second);
            }
            t.pending.clear();
        }
    }
    void free_timers() {
        for (ClassTimer& t : timers) {
            for (auto& ab : t.pending) { cudaEventDestroy(ab.first); cudaEventDestroy(ab.second); }
            for (cudaEvent_t e : t.pool) cudaEventDestroy(e);
            t = ClassTimer{};
        }
    }

    // Device tables of circuits and Kraus sets live in a library memory pool and are allocated and
    // freed in stream order, so releasing them does not wait for the device. Host-to-device copies
    // go through recycled pinned staging slots: a copy from pageable memory would first wait for
    // every earlier launch on the stream, and the host could not run ahead of the device.
    cudaMemPool_t pool = nullptr;
    struct Slot {
        unsigned char* p = nullptr;
        size_t cap = 0;
        cudaEvent_t ev = nullptr;     // recorded after the slot's last copy
        bool used = false;
    };
    static constexpr size_t kSlots = 32;
    static constexpr size_t kSlotMin = (size_t)2 << 20;   // per-step uploads stay below this
    Slot slots[kSlots];
    size_t next_slot = 0;

    // Test hook (PTSBE_OPT_FAIL_ALLOC): the allocation with index fail_alloc_at, counted from when
    // the option was set, fails as if the device or host were out of memory.
    int64_t fail_alloc_at = -1;
    uint64_t alloc_count = 0;
    void inject(const char* what) {
        if (fail_alloc_at >= 0 && alloc_count++ == (uint64_t)fail_alloc_at)
            fail(PTSBE_ERR_OOM, std::string("injected allocation failure: ") + what);
    }

    void* dalloc(size_t bytes) {
        inject("device table");
        void* p = nullptr;
        const cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, ustream());
        if (e != cudaSuccess) { (void)cudaGetLastError(); fail(PTSBE_ERR_OOM, "device table allocation failed"); }
        return p;
    }
    void dfree(void* p) {
        if (p) PTSBE_CUDA(cudaFreeAsync(p, stream));
    }
    // Stream-ordered copy of `bytes` host bytes to dst through the oldest staging slot (its
    // previous copy was issued kSlots copies ago; waiting for it is normally immediate).
    // Grows staging slot `sl` to hold `bytes` (pinned host memory).
    void grow_slot(Slot& sl, size_t bytes) {
        if (sl.cap >= bytes) return;
        if (sl.used) PTSBE_CUDA(cudaEventSynchronize(sl.ev));
        inject("pinned staging");
        if (sl.p) PTSBE_CUDA(cudaFreeHost(sl.p));   // synchronises the device: rare (large uploads)
        sl.p = nullptr;
        sl.cap = 0;
        size_t cap = kSlotMin;
        while (cap < bytes) cap *= 2;
        const cudaError_t e = cudaHostAlloc((void**)&sl.p, cap, cudaHostAllocDefault);
        if (e != cudaSuccess) { (void)cudaGetLastError(); sl.p = nullptr; sl.cap = 0; fail(PTSBE_ERR_OOM, "pinned staging allocation failed"); }
        sl.cap = cap;
    }
    // The next k copies through h2d find slots of at least `bytes`, so a call that reserves before
    // its first launch allocates nothing after it.
    void reserve_staging(size_t bytes, size_t k) {
        for (size_t i = 0; i < k && i < kSlots; ++i) grow_slot(slots[(next_slot + i) % kSlots], bytes);
    }
    void h2d(void* dst, const void* src, size_t bytes) {
        if (!bytes) return;
        Slot& sl = slots[next_slot];
        next_slot = (next_slot + 1) % kSlots;
        if (sl.used) PTSBE_CUDA(cudaEventSynchronize(sl.ev));
        grow_slot(sl, bytes);
        if (!sl.ev) PTSBE_CUDA(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming));
        std::memcpy(sl.p, src, bytes);
        PTSBE_CUDA(cudaMemcpyAsync(dst, sl.p, bytes, cudaMemcpyHostToDevice, ustream()));
        PTSBE_CUDA(cudaEventRecord(sl.ev, ustream()));
        sl.used = true;
        count_h2d(bytes);
    }
    // h2d through a staging slot that already holds `bytes` (the first such slot from the next one
    // on; no allocation of any kind); false when there is none, and nothing is copied.
    bool h2d_no_growth(void* dst, const void* src, size_t bytes) {
        size_t k = 0;
        while (k < kSlots) {
            const Slot& c = slots[(next_slot + k) % kSlots];
            if (c.p && c.cap >= bytes && c.ev) break;
            ++k;
        }
        if (k == kSlots) return false;
        Slot& sl = slots[(next_slot + k) % kSlots];
        next_slot = (next_slot + k + 1) % kSlots;
        if (sl.used) PTSBE_CUDA(cudaEventSynchronize(sl.ev));
        std::memcpy(sl.p, src, bytes);
        PTSBE_CUDA(cudaMemcpyAsync(dst, sl.p, bytes, cudaMemcpyHostToDevice, ustream()));
        PTSBE_CUDA(cudaEventRecord(sl.ev, ustream()));
        sl.used = true;
        count_h2d(bytes);
        return true;
    }
    void free_staging() {
        for (Slot& sl : slots) {
            if (sl.ev) cudaEventDestroy(sl.ev);
            if (sl.p) cudaFreeHost(sl.p);
            sl = Slot{};
        }
    }

    bool has_device() const { return device >= 0; }
    void need_device() const {
        if (!has_device()) fail(PTSBE_ERR_NO_DEVICE, "device entry point on a host-only context");
    }
    void use_device() const { PTSBE_CUDA(cudaSetDevice(device)); }

    // Grows a workspace buffer; waits for in-flight work that may still use the old one.
    void* ws(DevBuf& b, size_t bytes) {
        if (bytes <= b.cap && b.p) return b.p;
        inject("workspace");
        PTSBE_CUDA(cudaStreamSynchronize(stream));
        if (aux) PTSBE_CUDA(cudaStreamSynchronize(aux));
        if (b.p) { PTSBE_CUDA(cudaFree(b.p)); b.p = nullptr; b.cap = 0; }
        const size_t want = std::max<size_t>(bytes + bytes / 4, 4096);
        void* p = nullptr;
        const cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) { (void)cudaGetLastError(); fail(PTSBE_ERR_OOM, "workspace allocation of " + std::to_string(want) + " bytes failed"); }
        b.p = p; b.cap = want;
        return p;
    }
    void free_buf(DevBuf& b) { if (b.p) cudaFree(b.p); b.p = nullptr; b.cap = 0; }
    // Device word that kernels set when they could not do their work (zero when created).
    uint32_t* fault_word() {
        if (!fault.p) {
            void* p = ws(fault, sizeof(uint32_t));
            PTSBE_CUDA(cudaMemsetAsync(p, 0, sizeof(uint32_t), stream));
        }
        return (uint32_t*)fault.p;
    }

    Circuit& circuit(uint32_t id) {
        auto it = circuits.find(id);
        if (it == circuits.end()) fail(PTSBE_ERR_INVALID, "unknown circuit id " + std::to_string(id));
        return *it->second;
    }
    KSet& set(uint32_t id) {
        auto it = sets.find(id);
        if (it == sets.end()) fail(PTSBE_ERR_INVALID, "unknown set id " + std::to_string(id));
        return *it->second;
    }
};

namespace {

template <class F>
int guarded(ptsbe_ctx* ctx, F&& f) {
    if (!ctx) return PTSBE_ERR_INVALID;
    try {
        f();
        return PTSBE_OK;
    } catch (const Error& e) {
        ctx->err = e.what();
        return e.status;
    } catch (const std::bad_alloc&) {
        ctx->err = "host allocation failed";
        return PTSBE_ERR_OOM;
    } catch (const std::exception& e) {
        ctx->err = e.what();
        return PTSBE_ERR_INVALID;
    }
}

void free_device_circuit(ptsbe_ctx* ctx, DeviceCircuit& d) {
    ctx->dfree(d.base);
    if (d.ready) cudaEventDestroy(d.ready);
    d = DeviceCircuit{};
}

// Marks the end of an upload on the stream that made it (the prepass ahead waits for it).
void mark_ready(ptsbe_ctx* ctx, cudaEvent_t& ev) {
    if (!ev) PTSBE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    PTSBE_CUDA(cudaEventRecord(ev, ctx->ustream()));
}

// All tables of a circuit plan in one allocation and one staged copy.
void upload_circuit(ptsbe_ctx* ctx, const Circuit& c, const Plan& P, DeviceCircuit& d) {
    std::vector<unsigned char> blob;
    auto add = [&](const auto& v) {
        const size_t off = (blob.size() + 255) & ~size_t(255);
        const size_t bytes = v.size() * sizeof(v[0]);
        blob.resize(off + std::max<size_t>(bytes, 1));
        if (bytes) std::memcpy(blob.data() + off, v.data(), bytes);
        return v.empty() ? SIZE_MAX : off;
    };
    const size_t o_ops = add(c.dops), o_micro = add(c.dmicro), o_mats = add(c.dmats), o_chans = add(c.dchans);
    const size_t o_site = add(c.site_op), o_stages = add(P.stages), o_groups = add(P.groups), o_hi = add(P.hi);
    const size_t o_fst = add(P.fstages);
    unsigned char* base = (unsigned char*)ctx->dalloc(blob.size());
    ctx->h2d(base, blob.data(), blob.size());
    mark_ready(ctx, d.ready);
    auto at = [&](size_t off) { return off == SIZE_MAX ? nullptr : (void*)(base + off); };
    d.base = base;
    d.ops = (DevOp*)at(o_ops); d.micro = (DevMicro*)at(o_micro); d.mats = (float2*)at(o_mats);
    d.chans = (DevChannel*)at(o_chans); d.site_op = (uint32_t*)at(o_site); d.stages = (DevStage*)at(o_stages);
    d.groups = (DevGroup*)at(o_groups); d.hi = (uint32_t*)at(o_hi); d.fstages = (DevFrameStage*)at(o_fst);
}

// Builds a blob of aligned arrays on the host and returns the device pointers after one upload.
struct Blob {
    std::vector<unsigned char>& buf;
    explicit Blob(std::vector<unsigned char>& b) : buf(b) { buf.clear(); }
    template <class T>
    size_t add(const std::vector<T>& v) {
        size_t off = (buf.size() + 255) & ~size_t(255);
        buf.resize(off + std::max<size_t>(v.size() * sizeof(T), 1));
        if (!v.empty()) std::memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
};

// The set's (site, k) entries, one allocation and one staged copy (d_k follows d_site).
void ensure_set_on_device(ptsbe_ctx* ctx, KSet& s) {
    if (s.d_site || s.site.empty()) return;
    const size_t sb = s.site.size() * sizeof(uint32_t), kb = s.k.size();
    std::vector<unsigned char> blob(sb + kb);
    std::memcpy(blob.data(), s.site.data(), sb);
    std::memcpy(blob.data() + sb, s.k.data(), kb);
    unsigned char* base = (unsigned char*)ctx->dalloc(blob.size());
    ctx->h2d(base, blob.data(), blob.size());
    mark_ready(ctx, s.ready);
    s.d_site = (uint32_t*)base;
    s.d_k = base + sb;
}

// The backward plan's tables in one allocation and one staged copy.
void upload_backward_plan(ptsbe_ctx* ctx, BwPlan& P) {
    std::vector<unsigned char> buf;
    Blob b(buf);
    const size_t o_st = b.add(P.steps), o_it = b.add(P.items), o_me = b.add(P.members), o_po = b.add(P.pool);
    const size_t o_p64 = b.add(P.pool64), o_si = b.add(P.site_item), o_sm = b.add(P.site_mem);
    const size_t o_ds = b.add(P.dslot_out), o_pf = b.add(P.pos_final);
    unsigned char* base = (unsigned char*)ctx->dalloc(buf.size());
    ctx->h2d(base, buf.data(), buf.size());
    P.dev = base;
    P.d_steps = (const BwStep*)(base + o_st); P.d_items = (const BwItem*)(base + o_it);
    P.d_members = (const BwMember*)(base + o_me); P.d_pool = (const float2*)(base + o_po);
    P.d_pool64 = (const double*)(base + o_p64); P.d_site_item = (const uint32_t*)(base + o_si);
    P.d_site_mem = (const uint32_t*)(base + o_sm); P.d_dslot_out = (const uint32_t*)(base + o_ds);
    P.d_pos_final = (const uint8_t*)(base + o_pf);
}

// Same qubits, operations, targets, channel kinds and Kraus counts (parameters may differ).
void check_same_structure(const Circuit& a, const Circuit& b) {
    bool same = a.n == b.n && a.ops.size() == b.ops.size() && a.ch.size() == b.ch.size();
    for (size_t i = 0; same && i < a.ops.size(); ++i) {
        const ptsbe_op &x = a.ops[i], &y = b.ops[i];
        same = x.kind == y.kind && x.id == y.id && x.n_targets == y.n_targets && x.targets[0] == y.targets[0] &&
               (x.n_targets == 1 || x.targets[1] == y.targets[1]);
        if (same && x.kind == PTSBE_OP_GATE && (x.id == PTSBE_G_U1 || x.id == PTSBE_G_U2)) same = x.params[0] == y.params[0];
    }
    for (size_t c = 0; same && c < a.ch.size(); ++c)
        same = a.ch[c].kind == b.ch[c].kind && a.ch[c].arity == b.ch[c].arity && a.ch[c].nk == b.ch[c].nk;
    if (!same) fail(PTSBE_ERR_INVALID, "circuit does not have the structure of the set's circuit");
}

}  // namespace

namespace {

// Shots the last evolve launch draws from the support it holds on chip.
struct FusedShots {
    uint64_t seed;
    uint32_t* bits;
};

void evolve_dense_range(ptsbe_ctx* ctx, KSet& s, Circuit& c, uint32_t first, uint32_t count, void* d_states,
                        double* d_weights, uint8_t* d_status, uint32_t flags);

// prod over unitary-mixture sites of q_{s,k_s} for set alpha (q0mix: the product of every q_{s,0})
double mix_weight(const Circuit& c, const KSet& s, uint32_t alpha, double q0mix) {
    const uint32_t S = (uint32_t)c.site_op.size();
    double w = q0mix;
    if (q0mix > 0) {
        for (uint32_t e = s.off[alpha]; e < s.off[alpha + 1]; ++e) {
            const HostChannel& ch = c.ch[c.site_ch[s.site[e]]];
            if (ch.mixture) w *= ch.q[s.k[e]] / ch.q[0];
        }
    } else {
        w = 1.0;
        uint32_t e = s.off[alpha];
        for (uint32_t site = 0; site < S; ++site) {
            uint32_t k = 0;
            if (e < s.off[alpha + 1] && s.site[e] == site) k = s.k[e++];
            const HostChannel& ch = c.ch[c.site_ch[site]];
            if (ch.mixture) w *= ch.q[k];
        }
    }
    return w;
}

double mix_q0(const Circuit& c) {
    double q0mix = 1.0;
    for (uint32_t site = 0; site < c.site_op.size(); ++site) {
        const HostChannel& ch = c.ch[c.site_ch[site]];
        if (ch.mixture) q0mix *= ch.q[0];
    }
    return q0mix;
}

// Prepares states [first, first + count) of set s (the work of ptsbe_evolve_batch). With fused,
// the small sparse final stage also draws the shots of the states it can (drawn[a] = 1).
// before_launch runs after the call's own uploads and before its first kernel launch (the one-call
// entry point puts the samplers' work items up there, so the sampler launch follows the evolve
// launches with no copy between them); `drawn` is final when it runs.
void evolve_range(ptsbe_ctx* ctx, KSet& s, Circuit& c, uint32_t first, uint32_t count, void* d_states,
                  double* d_weights, uint8_t* d_status, uint32_t flags, const FusedShots* fused,
                  std::vector<uint8_t>* drawn, const std::function<void()>& before_launch = {}) {
    ctx->use_device();
    if (ctx->evolve_kernel == 4) {
        if (drawn) drawn->assign(count, 0);
        if (before_launch) before_launch();
        evolve_dense_range(ctx, s, c, first, count, d_states, d_weights, d_status, flags);
        return;
    }
    if (flags & PTSBE_EVOLVE_PLAN_ONLY) fail(PTSBE_ERR_UNSUPPORTED, "plan-only calls need the dense kernel");
    const bool frame = ctx->evolve_kernel == 0 || ctx->evolve_kernel == 3;
    if (frame && !c.frame_planned) {
        c.plan_frame = make_frame_plan(c, kTileMax);
        c.frame_planned = true;
    }
    if (!frame && !c.op_planned) {
        c.plan = make_plan(c, kTileMax, false);
        c.op_planned = true;
    }
    const Plan& P = frame ? c.plan_frame : c.plan;
    const DeviceCircuit& D = frame ? c.dev_frame : c.dev;
    const uint32_t S = (uint32_t)c.site_op.size();
    const bool reuse = flags & PTSBE_EVOLVE_PREFIX_REUSE;
    // Prepass ahead (one-stage frame plans): the programs depend only on the circuit and the sets,
    // not on any state, so this call's uploads and prepass go to the auxiliary stream without
    // waiting for the context stream, and run while the context stream still executes earlier
    // calls. The evolve launch waits for them. Not while the context stream is being captured
    // (the auxiliary stream would not join the capture) and not with a split zero fill.
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    PTSBE_CUDA(cudaStreamIsCapturing(ctx->stream, &capturing));
    const bool ahead = frame && ctx->prepass_ahead && ctx->aux && P.stages.size() == 1 && ctx->split_fill == 0 &&
                       capturing == cudaStreamCaptureStatusNone;
    // Uploads go to the auxiliary stream while the scope is open; on every exit the context
    // stream joins the auxiliary stream, and the lane is marked as used by everything the context
    // stream has been given up to then.
    struct AheadScope {
        ptsbe_ctx* ctx;
        bool on, pending;
        uint32_t lane;
        AheadScope(ptsbe_ctx* c, bool a) : ctx(c), on(a), pending(a), lane(c->lane) {
            if (on) { ctx->up = ctx->aux; ctx->lane ^= 1u; }
        }
        void uploads_done() { ctx->up = nullptr; }
        void join() {
            ctx->up = nullptr;
            if (!pending) return;
            pending = false;
            PTSBE_CUDA(cudaEventRecord(ctx->ev_join, ctx->aux));
            PTSBE_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
        }
        ~AheadScope() {
            ctx->up = nullptr;
            if (!on) return;
            if (pending) {
                (void)cudaEventRecord(ctx->ev_join, ctx->aux);
                (void)cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0);
            }
            if (cudaEventRecord(ctx->ev_used[lane], ctx->stream) == cudaSuccess) ctx->used_recorded[lane] = true;
        }
    } AS(ctx, ahead);
    const uint32_t lane = AS.lane;
    ensure_set_on_device(ctx, s);
    if (frame && !c.dev_frame.base) upload_circuit(ctx, c, c.plan_frame, c.dev_frame);
    if (!frame && !c.dev.ops) upload_circuit(ctx, c, c.plan, c.dev);
    if (ahead) {              // tables uploaded by earlier calls, possibly on the context stream
        if (s.ready) PTSBE_CUDA(cudaStreamWaitEvent(ctx->aux, s.ready, 0));
        if (c.dev_frame.ready) PTSBE_CUDA(cudaStreamWaitEvent(ctx->aux, c.dev_frame.ready, 0));
    }

    // --- node tables ---
    // With prefix reuse a set whose entries extend those of an earlier set of the range (its
    // parent: longest such prefix) starts at the stage holding its first extra site, from the
    // parent's input of that stage; a start in stage 0 is a start from |0...0>.
    const uint32_t J = (uint32_t)P.stages.size();
    std::vector<uint32_t> ebeg(count), eend(count), sstage(count), src(count);
    std::vector<uint8_t> fresh(count);
    std::vector<double> wmix(count), qa(count);
    std::unordered_map<std::string, uint32_t> index;
    // A set can only start later than stage 0 in a plan with more than one stage.
    const bool trie = reuse && J > 1;
    // prod over unitary-mixture sites of q_{s,0}; a set's product is this times the ratios at its
    // entries (the full product when some q_{s,0} is 0)
    double q0mix = 1.0;
    for (uint32_t site = 0; site < S; ++site) {
        const HostChannel& ch = c.ch[c.site_ch[site]];
        if (ch.mixture) q0mix *= ch.q[0];
    }
    auto key_of = [&](uint32_t alpha, uint32_t len) {
        std::string k;
        k.resize(len * 5);
        for (uint32_t i = 0; i < len; ++i) {
            std::memcpy(&k[5 * i], &s.site[s.off[alpha] + i], 4);
            k[5 * i + 4] = (char)s.k[s.off[alpha] + i];
        }
        return k;
    };
    for (uint32_t a = 0; a < count; ++a) {
        const uint32_t alpha = first + a;
        const uint32_t len = s.off[alpha + 1] - s.off[alpha];
        ebeg[a] = s.off[alpha]; eend[a] = s.off[alpha + 1];
        qa[a] = s.q[alpha];
        uint32_t parent = UINT32_MAX;
        if (trie) {
            for (int64_t p = (int64_t)len - 1; p >= 0; --p) {
                auto it = index.find(key_of(alpha, (uint32_t)p));
                if (it != index.end()) { parent = it->second; break; }
            }
            index.emplace(key_of(alpha, len), a);
        }
        sstage[a] = 0; src[a] = a; fresh[a] = 1;
        if (parent != UINT32_MAX) {
            const uint32_t plen = s.off[first + parent + 1] - s.off[first + parent];
            const uint32_t j = (uint32_t)P.op_stage[c.site_op[s.site[s.off[alpha] + plen]]];
            // The parent starts no later than the child (its extra sites come first). If it
            // starts in the same stage, both read the same input: the parent's source.
            if (j > 0) { sstage[a] = j; src[a] = sstage[parent] == j ? src[parent] : parent; fresh[a] = 0; }
        }
        // prod over unitary-mixture sites of q_{s,k_s}
        double w = q0mix;
        if (q0mix > 0) {
            for (uint32_t e = s.off[alpha]; e < s.off[alpha + 1]; ++e) {
                const HostChannel& ch = c.ch[c.site_ch[s.site[e]]];
                if (ch.mixture) w *= ch.q[s.k[e]] / ch.q[0];
            }
        } else {
            w = 1.0;
            uint32_t e = s.off[alpha];
            for (uint32_t site = 0; site < S; ++site) {
                uint32_t k = 0;
                if (e < s.off[alpha + 1] && s.site[e] == site) k = s.k[e++];
                const HostChannel& ch = c.ch[c.site_ch[site]];
                if (ch.mixture) w *= ch.q[k];
            }
        }
        wmix[a] = w;
    }
    // one launch per stage: every set whose start stage is at or before it
    std::vector<uint32_t> lists;
    std::vector<std::pair<size_t, uint32_t>> launches;  // (offset, count) per stage
    for (uint32_t j = 0; j < J; ++j) {
        const size_t off = lists.size();
        for (uint32_t a = 0; a < count; ++a)
            if (sstage[a] <= j) lists.push_back(a);
        launches.push_back({off, (uint32_t)(lists.size() - off)});
    }
    {   // gates applied with and without prefix reuse
        std::vector<uint64_t> stage_gates(J + 1, 0);
        for (uint32_t j = J; j-- > 0;) {
            uint64_t g = 0;
            for (uint32_t op = P.stages[j].op_begin; op < P.stages[j].op_end; ++op) g += c.ops[op].kind == PTSBE_OP_GATE;
            stage_gates[j] = stage_gates[j + 1] + g;
        }
        ctx->reuse_gates_run = 0;
        for (uint32_t a = 0; a < count; ++a) ctx->reuse_gates_run += stage_gates[sstage[a]];
        ctx->reuse_gates_full = (uint64_t)count * stage_gates[0];
    }
    Blob blob(ctx->host_blob);
    const size_t o_ebeg = blob.add(ebeg), o_eend = blob.add(eend), o_sstage = blob.add(sstage);
    const size_t o_src = blob.add(src), o_fresh = blob.add(fresh);
    const size_t o_wmix = blob.add(wmix), o_q = blob.add(qa), o_lists = blob.add(lists);
    // Shots drawn by the last launch: the small sparse final stage holds each state's support
    // on chip and draws the shots of states with at most light_shots of them (the others are
    // left to the sampler kernels).
    int sparse_last = -1, small_last = 0;
    if (frame)
        for (uint32_t j = 0; j < J; ++j)
            if (P.fstages[j].sparse_final) { sparse_last = (int)j; small_last = (int)P.fstages[j].sbits; }
    const bool fuse = fused && sparse_last == (int)J - 1 && small_last > 0;
    // Heavier states leave their support CDF for k_sample_support (drawn[a] = 2).
    std::vector<uint32_t> nshots, nexport;
    std::vector<uint64_t> nout;
    size_t o_nshots = 0, o_nout = 0, o_nexport = 0;
    uint64_t fused_shots = 0;
    std::vector<SupportItem> support_items;
    uint32_t n_export = 0;
    if (drawn) drawn->assign(count, 0);
    if (fuse) {
        nshots.assign(count, 0);
        nout.assign(count, 0);
        nexport.assign(count, 0xFFFFFFFFu);
        const uint64_t base = s.shot_off[first];
        for (uint32_t a = 0; a < count; ++a) {
            const uint64_t m = s.shots[first + a];
            nout[a] = s.shot_off[first + a] - base;
            if (m == 0) continue;
            if (m <= ctx->light_shots && m <= UINT32_MAX) {
                nshots[a] = (uint32_t)m;
                fused_shots += m;
                if (drawn) (*drawn)[a] = 1;
            } else {
                nexport[a] = n_export;
                for (uint64_t j0 = 0; j0 < m; j0 += kSupportChunk)
                    support_items.push_back({n_export, first + a, j0, std::min(m, j0 + kSupportChunk), nout[a] + j0});
                ++n_export;
                if (drawn) (*drawn)[a] = 2;
            }
        }
        o_nshots = blob.add(nshots);
        o_nout = blob.add(nout);
        if (n_export) o_nexport = blob.add(nexport);
    }
    unsigned char* dblob = (unsigned char*)ctx->ws(ahead ? ctx->ahead_nodes[lane] : ctx->nodes, ctx->host_blob.size());
    if (ahead && ctx->used_recorded[lane]) PTSBE_CUDA(cudaStreamWaitEvent(ctx->aux, ctx->ev_used[lane], 0));
    ctx->h2d(dblob, ctx->host_blob.data(), ctx->host_blob.size());
    AS.uploads_done();        // what follows goes up on the context stream

    EvolveArgs A{};
    A.ops = D.ops; A.micro = D.micro; A.mats = D.mats; A.chans = D.chans;
    A.n_mats = (uint32_t)c.dmats.size();
    A.site_op = D.site_op; A.stages = D.stages; A.groups = D.groups; A.hi = D.hi; A.fstages = D.fstages;
    A.n = (int)c.n; A.tb = P.tb; A.lb = P.lb;
    A.ent_site = s.d_site; A.ent_k = s.d_k;
    A.node_ebeg = (const uint32_t*)(dblob + o_ebeg); A.node_eend = (const uint32_t*)(dblob + o_eend);
    A.node_sstage = (const uint32_t*)(dblob + o_sstage); A.node_src = (const uint32_t*)(dblob + o_src);
    A.node_fresh = (const uint8_t*)(dblob + o_fresh);
    A.wmix = (const double*)(dblob + o_wmix); A.qalpha = (const double*)(dblob + o_q);
    A.weights = d_weights; A.status = d_status;
    if (fuse && fused_shots) {
        A.shot_bits = fused->bits;
        A.shot_seed = fused->seed;
        A.shot_alpha0 = first;
        A.node_shots = (const uint32_t*)(dblob + o_nshots);
        A.node_shot_out = (const uint64_t*)(dblob + o_nout);
    }
    const size_t slot_bytes = support_slot_bytes(small_last);
    if (n_export) {
        A.node_export = (const uint32_t*)(dblob + o_nexport);
        A.support_out = (unsigned char*)ctx->ws(ctx->support, (size_t)n_export * slot_bytes);
    }
    if (fuse && (fused_shots || n_export)) A.fault = ctx->fault_word();
    // the support sampler's work items go up before the first launch (every allocation of the
    // call precedes its kernels)
    SupportItem* d_sitems = nullptr;
    if (!support_items.empty()) {
        d_sitems = (SupportItem*)ctx->ws(ctx->sitems, support_items.size() * sizeof(SupportItem));
        ctx->h2d(d_sitems, support_items.data(), support_items.size() * sizeof(SupportItem));
    }
    const double sbytes = 8.0 * (double)(1ull << c.n);
    // stage j writes out(j); out(J-1) is the caller's buffer. The per-operator kernels without
    // reuse read and write the caller's buffer in place (a tile is read whole before it is
    // written); frame stores move amplitudes between tiles, so they always alternate.
    float2* const user = (float2*)d_states;
    float2* const other = (reuse || frame) && J > 1 ? (float2*)ctx->ws(ctx->pingpong, (size_t)count * (size_t)sbytes) : user;
    auto out_buf = [&](uint32_t j) { return ((J - 1 - j) & 1u) ? other : user; };
    const int ob = (int)c.n - P.tb;
    float* d_scale = nullptr;
    if (ob > 0) {
        A.part = (double*)ctx->ws(ctx->part, ((size_t)count << ob) * sizeof(double));
        d_scale = (float*)ctx->ws(ctx->scale, (size_t)count * sizeof(float));
    }
    if (frame) {
        uint32_t widest = 0;
        for (const auto& L : launches) widest = std::max(widest, L.second);
        A.frame_progs = ctx->ws(ahead ? ctx->ahead_progs[lane] : ctx->progs, (size_t)widest * evolve_frame_program_bytes());
    }
    const uint32_t* d_lists = (const uint32_t*)(dblob + o_lists);
    // When the last frame stage only reorders (no ops), the norm is known after the stage
    // before it: that stage's stores leave tile norms, a reduce turns them into scales, and
    // the last stage writes the normalised state (no separate renormalisation pass).
    const bool early_norm = frame && ob > 0 && J >= 2 && P.stages[J - 1].op_begin == P.stages[J - 1].op_end &&
                            launches[J - 2].second == count;
    A.sparse_final_stage = -1;
    A.small_bits = 0;
    if (frame)
        for (uint32_t j = 0; j < J; ++j)
            if (P.fstages[j].sparse_final) { A.sparse_final_stage = (int)j; A.small_bits = (int)P.fstages[j].sbits; }
    // A one-stage plan ending in the small sparse final store writes only each state's support
    // (at most 2^small_bits amplitudes); every other amplitude is zero. That zero fill needs no
    // program, so it runs as its own HBM-bound kernel on the auxiliary stream while the
    // latency-bound program prepass runs, and the evolve launch waits for it.
    // prefix of each state zeroed beside the prepass: whole 4 KB chunks (the in-launch fill's unit)
    const uint64_t prefill = (uint64_t)((double)sbytes * ctx->split_fill / 100.0) / 4096u * 4096u;
    const bool split_fill = frame && prefill && ctx->aux && J == 1 && A.sparse_final_stage == 0 &&
                            A.small_bits > 0 && launches[0].second == count && (uint64_t)sbytes % 4096u == 0;
    if (before_launch) before_launch();
    for (uint32_t j = 0; j < J; ++j) {
        const auto& L = launches[j];
        if (L.second == 0) continue;
        A.states = out_buf(j);
        A.states_in = j > 0 ? out_buf(j - 1) : out_buf(j);
        A.store_norm = early_norm && j + 2 == J;
        A.scale_in = early_norm && j + 1 == J ? d_scale : nullptr;
        // algorithmic bytes: read (unless started from |0>) and write of each set's state
        double bytes = 0;
        for (size_t t = L.first; t < L.first + L.second; ++t)
            bytes += (fresh[lists[t]] && j == 0) ? sbytes : 2 * sbytes;
        if (split_fill) bytes -= (double)L.second * (double)prefill;   // zeros stored by the prepass-side fill
        if (A.shot_bits && j + 1 == J) bytes += 4.0 * (double)fused_shots;
        if (split_fill) ctx->fork_aux();
        if (frame) {
            cudaStream_t ps = ahead ? ctx->aux : ctx->stream;
            ctx->timed_on(ps, PTSBE_TIMER_EVOLVE_PROGRAM, 0.0, [&] {
                launch_frame_program(A, (int)j, d_lists + L.first, L.second, ps, ctx->prog_sets_per_warp);
            });
            AS.join();
        }
        A.prefill_bytes = 0;
        if (split_fill) {
            ctx->timed_on(ctx->aux, PTSBE_TIMER_ZERO_FILL, (double)count * (double)prefill,
                          [&] { launch_zero_states(user, (uint64_t)sbytes, prefill, count, ctx->n_sm, ctx->aux); });
            ctx->join_aux();
            A.prefill_bytes = prefill;
        }
        ctx->timed(PTSBE_TIMER_EVOLVE_STAGE, bytes, [&] {
            launch_evolve_stage(A, (int)j, j + 1 == J, d_lists + L.first, L.second, ctx->stream, ctx->evolve_kernel);
        });

        if (A.store_norm)
            ctx->timed(PTSBE_TIMER_EVOLVE_FINALIZE, 0.0, [&] { launch_evolve_reduce(A, count, d_scale, ctx->stream); });
    }
    A.states = user;
    A.store_norm = 0;
    A.scale_in = nullptr;
    if (ob > 0 && !early_norm && A.sparse_final_stage < 0)
        ctx->timed(PTSBE_TIMER_EVOLVE_FINALIZE, 2 * sbytes * count, [&] { launch_evolve_finalize(A, count, d_scale, ctx->stream); });
    if (!support_items.empty()) {
        SupportItem* d_items = d_sitems;
        uint64_t heavy = 0;
        for (const SupportItem& it : support_items) heavy += it.j1 - it.j0;
        // algorithmic: each exported CDF read once per item + 4 B per shot
        const double bytes = (double)slot_bytes * (double)support_items.size() + 4.0 * (double)heavy;
        ctx->timed(PTSBE_TIMER_SAMPLE, bytes, [&] {
            launch_sample_support(A.support_out, slot_bytes, d_items, (uint32_t)support_items.size(), fused->seed,
                                  fused->bits, ctx->stream);
        });
    }
}

// Reserves what sample_range will allocate for `count` states (work items: at most one light
// item per state plus chunks; at most 2 count + 4 SMs + 16 of them), so that a call that prepares
// and samples allocates nothing after its first launch.
// Shots per sampler work item. An item rebuilds its state's CDF, so a state is split no finer
// than that work repays: at least 2^16 shots above 14 qubits (a thread-block cluster per item),
// and up to 14 qubits (one CTA per item) as many shots as the CDF has entries, 2^n (at least
// 1,024). Above that floor, about four items per resident cluster over the whole shot budget. The
// split never changes a shot: shot j of a set draws from the Philox counter of j whichever item
// holds it.
uint64_t sample_chunk(int n, uint64_t total, uint64_t clusters) {
    const uint64_t floor_shots = n <= 14 ? std::max<uint64_t>(1024, 1ull << n) : (1ull << 16);
    return std::max<uint64_t>(floor_shots, (total + 4 * clusters - 1) / (4 * clusters));
}

void reserve_sampler(ptsbe_ctx* ctx, const Circuit& c, uint32_t count) {
    const size_t items = 2 * (size_t)count + 4 * (size_t)std::max(ctx->n_sm, 1) + 16;
    ctx->ws(ctx->items, items * sizeof(SampleItem));
    if ((int)c.n > sample_cluster_max_qubits()) ctx->ws(ctx->scratch, sample_global_scratch_doubles((int)c.n) * 8);
    // every staging slot: later copies of the call may land on any of them
    ctx->reserve_staging(std::max(items * sizeof(SampleItem), ptsbe_ctx::kSlotMin), ptsbe_ctx::kSlots);
}

// Draws the shots of states [first, first + count) (the work of ptsbe_sample_shots), except those
// of states marked in drawn.
// The work of sample_range in two halves: the host plan and its upload (work items, scratch), and
// the launches, so that a caller can put the upload before earlier launches of the same call.
struct SampleRun {
    SampleArgs A{};
    SampleItem* d_items = nullptr;
    size_t nl = 0, nh = 0;
    double light_bytes = 0, heavy_bytes = 0;
    std::vector<std::pair<uint32_t, uint64_t>> global;   // (range-local state, shots) for the global CDF
    std::vector<uint32_t> global_alpha;
    std::vector<uint64_t> global_out;
};

SampleRun plan_sample_range(ptsbe_ctx* ctx, KSet& s, Circuit& c, uint32_t first, uint32_t count, const void* d_states,
                            const uint8_t* d_status, uint64_t seed, uint32_t* d_bits, const std::vector<uint8_t>* drawn) {
    ctx->use_device();
    SampleRun R;
    SampleArgs& A = R.A;
    A.n = (int)c.n;
    A.states = (const float2*)d_states;
    A.status = d_status;
    A.seed = seed;
    A.bits = d_bits;
    const int n = (int)c.n;
    const bool light_ok = n > 14 && n <= sample_light_max_qubits();
    std::vector<SampleItem> light, items;
    const uint64_t cl = n <= 14 ? 1 : (1ull << (n - 14));
    const uint64_t clusters = std::max<uint64_t>(1, (uint64_t)ctx->n_sm / cl);
    const uint64_t base = s.shot_off[first];
    uint64_t total = 0;
    for (uint32_t a = 0; a < count; ++a)
        if (!(drawn && (*drawn)[a])) total += s.shots[first + a];
    const uint64_t chunk = sample_chunk(n, total, clusters);
    for (uint32_t a = 0; a < count; ++a) {
        const uint32_t alpha = first + a;
        const uint64_t m = s.shots[alpha], o = s.shot_off[alpha] - base;
        if (m == 0 || (drawn && (*drawn)[a])) continue;
        if (light_ok && m <= ctx->light_shots) { light.push_back({a, alpha, 0, m, o, kDomShot, 0}); continue; }
        if (n <= sample_cluster_max_qubits()) {
            for (uint64_t j0 = 0; j0 < m; j0 += chunk)
                items.push_back({a, alpha, j0, std::min(m, j0 + chunk), o + j0, kDomShot, 0});
        } else {
            R.global.push_back({a, m});
            R.global_alpha.push_back(alpha);
            R.global_out.push_back(o);
        }
    }
    R.nl = light.size();
    R.nh = items.size();
    if (n > sample_cluster_max_qubits())   // reserved before any launch of this call
        A.scratch = (unsigned long long*)ctx->ws(ctx->scratch, sample_global_scratch_doubles(n) * 8);
    if (R.nl + R.nh) {
        // algorithmic: each state read once and 4 bytes per shot written (the light sampler's
        // per-shot chunk re-reads are its design's extra traffic, not counted)
        uint64_t light_shots = 0, heavy_shots = 0;
        for (const SampleItem& it : light) light_shots += it.j1 - it.j0;
        for (const SampleItem& it : items) heavy_shots += it.j1 - it.j0;
        R.light_bytes = 8.0 * (double)(1ull << n) * (double)R.nl + 4.0 * (double)light_shots;
        R.heavy_bytes = 8.0 * (double)(1ull << n) * (double)R.nh + 4.0 * (double)heavy_shots;
        light.insert(light.end(), items.begin(), items.end());
        R.d_items = (SampleItem*)ctx->ws(ctx->items, light.size() * sizeof(SampleItem));
        ctx->h2d(R.d_items, light.data(), light.size() * sizeof(SampleItem));
    }
    return R;
}

void launch_sample_range(ptsbe_ctx* ctx, const SampleRun& R) {
    const SampleArgs& A = R.A;
    if (R.nl)
        ctx->timed(PTSBE_TIMER_SAMPLE_LIGHT, R.light_bytes, [&] { launch_sample_light(A, R.d_items, (uint32_t)R.nl, ctx->stream); });
    if (R.nh)
        ctx->timed(PTSBE_TIMER_SAMPLE, R.heavy_bytes, [&] { launch_sample_cluster(A, R.d_items + R.nl, (uint32_t)R.nh, ctx->stream); });
    const double sb = 8.0 * (double)(1ull << A.n);
    for (size_t i = 0; i < R.global.size(); ++i) {
        const uint64_t m = R.global[i].second;
        ctx->timed(PTSBE_TIMER_SAMPLE, 5 * sb + 4.0 * m, [&] {
            launch_sample_global(A, R.global[i].first, R.global_alpha[i], 0, m, R.global_out[i], ctx->stream);
        });
    }
}

void sample_range(ptsbe_ctx* ctx, KSet& s, Circuit& c, uint32_t first, uint32_t count, const void* d_states,
                  const uint8_t* d_status, uint64_t seed, uint32_t* d_bits, const std::vector<uint8_t>* drawn) {
    launch_sample_range(ctx, plan_sample_range(ctx, s, c, first, count, d_states, d_status, seed, d_bits, drawn));
}

// ---- dense tile passes -------------------------------------------------------------------------

void ensure_dense_plan(ptsbe_ctx* ctx, Circuit& c) {
    DensePlan& P = c.dense;
    if (!P.built) make_dense_plan(c, P);
    if (P.dev) return;
    std::vector<unsigned char> buf;
    Blob b(buf);
    const size_t o_p = b.add(P.passes), o_g = b.add(P.groups), o_b = b.add(P.blocks), o_h = b.add(P.hi);
    const size_t o_o = b.add(P.omap), o_m = b.add(P.mats);
    unsigned char* base = (unsigned char*)ctx->dalloc(buf.size());
    ctx->h2d(base, buf.data(), buf.size());
    P.dev = base;
    P.d_passes = (const dense::Pass*)(base + o_p);
    P.d_groups = (const dense::Group*)(base + o_g);
    P.d_blocks = (const dense::Block*)(base + o_b);
    P.d_hi = (const uint32_t*)(base + o_h);
    P.d_omap = (const uint16_t*)(base + o_o);
    P.d_mats = (const float2*)(base + o_m);
}

// Override blocks of set alpha: every block holding one of its entries, with the set's Kraus
// operators in it, sorted by block id. Appends to ovr / pool; returns [begin, end).
std::pair<uint32_t, uint32_t> dense_overrides(const Circuit& c, const DensePlan& P, const KSet& s, uint32_t alpha,
                                              std::vector<dense::Override>& ovr, std::vector<float2>& pool) {
    const uint32_t e0 = s.off[alpha], e1 = s.off[alpha + 1];
    std::vector<std::pair<uint32_t, uint32_t>> eb;   // (block, entry)
    for (uint32_t e = e0; e < e1; ++e) eb.push_back({P.site_block[s.site[e]], e});
    std::sort(eb.begin(), eb.end());
    const uint32_t begin = (uint32_t)ovr.size();
    std::vector<uint32_t> sites;
    std::vector<uint8_t> ks;
    for (size_t i = 0; i < eb.size();) {
        const uint32_t blk = eb[i].first;
        sites.clear();
        ks.clear();
        for (; i < eb.size() && eb[i].first == blk; ++i) { sites.push_back(s.site[eb[i].second]); ks.push_back(s.k[eb[i].second]); }
        const uint32_t cnt = P.blk_nq[blk] == 1 ? 4 : 16;
        const uint32_t off = (uint32_t)pool.size();
        pool.resize(pool.size() + cnt);
        uint32_t code = 0;
        dense_block_matrix(c, P, blk, sites.data(), ks.data(), (uint32_t)sites.size(), &pool[off], &code);
        ovr.push_back({blk, off, code});
    }
    return {begin, (uint32_t)ovr.size()};
}

DenseArgs dense_args(const DensePlan& P, int n) {
    DenseArgs A{};
    A.passes = P.d_passes; A.groups = P.d_groups; A.blocks = P.d_blocks;
    A.hi = P.d_hi; A.omap = P.d_omap; A.mats = P.d_mats;
    A.n = n;
    return A;
}

// Algorithmic bytes of one dense pass launch over `nodes` states (read unless started from
// |0...0>, then write; 8 bytes per amplitude each way).
double dense_bytes(int n, uint32_t nodes, uint32_t fresh) {
    const double sb = 8.0 * (double)(1ull << n);
    return (2.0 * (nodes - fresh) + (double)fresh) * sb;
}

// ptsbe_evolve_batch with the dense kernel: one launch per pass for every set of the range, each
// set's override blocks inserted. Prefix reuse: a set starts at the first pass that holds a block
// with one of its entries beyond those of an earlier set of the range (its parent: the longest
// such prefix that has computed its state at that pass), reading the parent's input of that pass.
void evolve_dense_range(ptsbe_ctx* ctx, KSet& s, Circuit& c, uint32_t first, uint32_t count, void* d_states,
                        double* d_weights, uint8_t* d_status, uint32_t flags) {
    if (flags & PTSBE_EVOLVE_PLAN_ONLY) {
        if (!c.dense.built) make_dense_plan(c, c.dense);
    } else {
        ensure_dense_plan(ctx, c);
    }
    const DensePlan& P = c.dense;
    const int n = P.n;                   // >= kT: a smaller state runs zero-padded to kT qubits
    const uint32_t J = (uint32_t)P.passes.size();
    const bool reuse = (flags & PTSBE_EVOLVE_PREFIX_REUSE) && J > 1;
    std::vector<dense::Override> ovr;
    std::vector<float2> pool;
    std::vector<uint32_t> ovb(count), ove(count), sstage(count, 0), src(count);
    std::vector<double> wmix(count), qa(count);
    const double q0mix = mix_q0(c);
    std::unordered_map<std::string, uint32_t> index;
    auto key_of = [&](uint32_t alpha, uint32_t len) {
        std::string k;
        k.resize(len * 5);
        for (uint32_t i = 0; i < len; ++i) {
            std::memcpy(&k[5 * i], &s.site[s.off[alpha] + i], 4);
            k[5 * i + 4] = (char)s.k[s.off[alpha] + i];
        }
        return k;
    };
    for (uint32_t a = 0; a < count; ++a) {
        const uint32_t alpha = first + a;
        const uint32_t len = s.off[alpha + 1] - s.off[alpha];
        auto r = dense_overrides(c, P, s, alpha, ovr, pool);
        ovb[a] = r.first;
        ove[a] = r.second;
        wmix[a] = mix_weight(c, s, alpha, q0mix);
        qa[a] = s.q[alpha];
        src[a] = a;
        if (reuse) {
            for (int64_t p = (int64_t)len - 1; p >= 0; --p) {
                auto it = index.find(key_of(alpha, (uint32_t)p));
                if (it == index.end()) continue;
                const uint32_t par = it->second;
                uint32_t j = J;
                for (uint32_t e = s.off[alpha] + (uint32_t)p; e < s.off[alpha + 1]; ++e)
                    j = std::min(j, P.blk_pass[P.site_block[s.site[e]]]);
                if (j == 0 || sstage[par] > j) continue;
                sstage[a] = j;
                src[a] = sstage[par] == j ? src[par] : par;
                break;
            }
            index.emplace(key_of(alpha, len), a);
        }
    }
    ctx->reuse_gates_run = 0;
    uint64_t total_gates = 0;
    std::vector<uint64_t> suffix(J + 1, 0);
    for (uint32_t j = J; j-- > 0;) suffix[j] = suffix[j + 1] + P.pass_gates[j];
    total_gates = suffix[0];
    for (uint32_t a = 0; a < count; ++a) ctx->reuse_gates_run += suffix[sstage[a]];
    ctx->reuse_gates_full = (uint64_t)count * total_gates;
    if (flags & PTSBE_EVOLVE_PLAN_ONLY) return;

    const size_t sb = (size_t)8 << n;
    // padded states go through a library buffer; the caller's states are copied out at the end
    const bool padded = n > (int)c.n;
    float2* const user = padded ? (float2*)ctx->ws(ctx->dense_pad, (size_t)count * sb) : (float2*)d_states;
    float2* const other = reuse ? (float2*)ctx->ws(ctx->pingpong, (size_t)count * sb) : user;
    auto out_buf = [&](uint32_t j) { return ((J - 1 - j) & 1u) ? other : user; };
    auto slot = [&](float2* b, uint32_t a) { return b + ((size_t)a << n); };
    std::vector<dense::Node> nodes;
    std::vector<std::pair<size_t, uint32_t>> launches;
    std::vector<uint32_t> fresh_cnt;
    for (uint32_t j = 0; j < J; ++j) {
        const size_t off = nodes.size();
        uint32_t fr = 0;
        for (uint32_t a = 0; a < count; ++a) {
            if (sstage[a] > j) continue;
            dense::Node nd{};
            if (j == sstage[a] && j == 0) { nd.src = nullptr; ++fr; }
            else nd.src = slot(j == 0 ? user : out_buf(j - 1), j == sstage[a] ? src[a] : a);
            nd.dst = slot(out_buf(j), a);
            nd.ov_begin = ovb[a];
            nd.ov_end = ove[a];
            nd.part = a;
            nodes.push_back(nd);
        }
        launches.push_back({off, (uint32_t)(nodes.size() - off)});
        fresh_cnt.push_back(fr);
    }
    std::vector<unsigned char> buf;
    Blob b(buf);
    const size_t o_n = b.add(nodes), o_o = b.add(ovr), o_p = b.add(pool), o_w = b.add(wmix), o_q = b.add(qa);
    unsigned char* d = (unsigned char*)ctx->ws(ctx->dense_tabs, buf.size());
    ctx->h2d(d, buf.data(), buf.size());
    const int ob = n - dense::kT;
    double* part = (double*)ctx->ws(ctx->part, ((size_t)count << ob) * sizeof(double));
    float* d_scale = (float*)ctx->ws(ctx->scale, (size_t)count * sizeof(float));
    DenseArgs A = dense_args(P, n);
    A.ovr = (const dense::Override*)(d + o_o);
    A.opool = (const float2*)(d + o_p);
    A.part = part;
    ctx->dense_launches = 0;
    ctx->dense_fma = 0;
    for (uint32_t j = 0; j < J; ++j) {
        if (launches[j].second == 0) continue;
        ctx->dense_launches += launches[j].second;
        ctx->dense_fma += (double)P.pass_fma[j] * (double)(1ull << n) * launches[j].second;
        A.nodes = (const dense::Node*)(d + o_n) + launches[j].first;
        A.n_nodes = launches[j].second;
        A.pass = (int)j;
        A.last = j + 1 == J ? 1 : 0;
        A.stage_bytes = P.passes[j].stage_bytes;
        ctx->timed(PTSBE_TIMER_DENSE, dense_bytes(n, A.n_nodes, fresh_cnt[j]), [&] { launch_dense_pass(A, ctx->n_sm, ctx->stream); });
    }
    EvolveArgs E{};
    E.n = n;
    E.tb = dense::kT;
    E.part = part;
    E.wmix = (const double*)(d + o_w);
    E.qalpha = (const double*)(d + o_q);
    E.weights = d_weights;
    E.status = d_status;
    E.states = user;
    ctx->timed(PTSBE_TIMER_EVOLVE_FINALIZE, 2.0 * (double)sb * count, [&] { launch_evolve_finalize(E, count, d_scale, ctx->stream, true); });
    if (padded)
        ctx->timed(PTSBE_TIMER_EVOLVE_FINALIZE, 2.0 * (double)((size_t)8 << c.n) * count,
                   [&] { launch_dense_unpad(user, n, (float2*)d_states, (int)c.n, count, ctx->n_sm, ctx->stream); });
}

// ptsbe_evolve_sample without caller states: the states live in library buffers, one branch at
// a time. The sets of the range are split, pass by pass, by their entries in that pass: every
// group with entries there branches into a new buffer (reading the shared input of the pass) and
// runs to the end first; then the sets with none continue in place. A branch that reaches the end
// holds exactly one set's state: it is normalised (weight, status) and sampled, and its buffer is
// released. Live buffers never exceed the nesting depth of the branches plus one.
void stream_evolve_sample(ptsbe_ctx* ctx, KSet& s, Circuit& c, uint32_t first, uint32_t count, double* d_weights,
                          uint8_t* d_status, uint64_t seed, uint32_t* d_bits, bool plan_only) {
    if (plan_only) {
        if (!c.dense.built) make_dense_plan(c, c.dense);
    } else {
        ensure_dense_plan(ctx, c);
    }
    const DensePlan& P = c.dense;
    const int n = (int)c.n;
    const uint32_t J = (uint32_t)P.passes.size();
    std::vector<dense::Override> ovr;
    std::vector<float2> pool;
    std::vector<uint32_t> ovb(count), ove(count);
    std::vector<double> wmix(count), qa(count);
    const double q0mix = mix_q0(c);
    // entries of each set as (pass, site, k), sorted
    std::vector<std::vector<std::tuple<uint32_t, uint32_t, uint8_t>>> byp(count);
    for (uint32_t a = 0; a < count; ++a) {
        const uint32_t alpha = first + a;
        auto r = dense_overrides(c, P, s, alpha, ovr, pool);
        ovb[a] = r.first;
        ove[a] = r.second;
        wmix[a] = mix_weight(c, s, alpha, q0mix);
        qa[a] = s.q[alpha];
        for (uint32_t e = s.off[alpha]; e < s.off[alpha + 1]; ++e)
            byp[a].emplace_back(P.blk_pass[P.site_block[s.site[e]]], s.site[e], s.k[e]);
        std::sort(byp[a].begin(), byp[a].end());
    }
    struct Act {
        uint32_t pass;                 // J: leaf -- normalise and sample set `rep`
        int src, dst;                  // buffer indices (-1: |0...0>)
        uint32_t rep;                  // a set of the group (its overrides serve the whole group)
    };
    std::vector<Act> acts;
    int nbuf = 0;
    std::vector<int> freeb;
    auto alloc = [&]() {
        if (!freeb.empty()) { const int x = freeb.back(); freeb.pop_back(); return x; }
        return nbuf++;
    };
    std::vector<size_t> cur(count, 0);
    uint64_t gates_run = 0;
    std::function<void(uint32_t, int, std::vector<uint32_t>&)> rec = [&](uint32_t j, int X, std::vector<uint32_t>& sets) {
        if (j == J) {
            for (uint32_t a : sets) acts.push_back({J, X, X, a});
            freeb.push_back(X);
            return;
        }
        std::vector<std::vector<uint32_t>> groups;
        std::unordered_map<std::string, size_t> gi;
        std::vector<uint32_t> main;
        for (uint32_t a : sets) {
            std::string key;
            while (cur[a] < byp[a].size() && std::get<0>(byp[a][cur[a]]) == j) {
                const uint32_t site = std::get<1>(byp[a][cur[a]]);
                key.append((const char*)&site, 4);
                key.push_back((char)std::get<2>(byp[a][cur[a]]));
                ++cur[a];
            }
            if (key.empty()) { main.push_back(a); continue; }
            auto it = gi.find(key);
            if (it == gi.end()) { gi.emplace(key, groups.size()); groups.push_back({a}); }
            else groups[it->second].push_back(a);
        }
        for (auto& g : groups) {
            const int Y = alloc();
            acts.push_back({j, X, Y, g[0]});
            gates_run += P.pass_gates[j];
            rec(j + 1, Y, g);
        }
        if (main.empty()) {
            if (X >= 0) freeb.push_back(X);
            return;
        }
        const int D = X >= 0 ? X : alloc();
        acts.push_back({j, X, D, main[0]});
        gates_run += P.pass_gates[j];
        rec(j + 1, D, main);
    };
    {
        std::vector<uint32_t> all(count);
        for (uint32_t a = 0; a < count; ++a) all[a] = a;
        rec(0, -1, all);
    }
    uint64_t total_gates = 0;
    for (uint32_t g : P.pass_gates) total_gates += g;
    ctx->reuse_gates_run = gates_run;
    ctx->reuse_gates_full = (uint64_t)count * total_gates;
    if (plan_only) return;

    const size_t sb = (size_t)8 << n;
    if (ctx->state_pool.size() < (size_t)nbuf) ctx->state_pool.resize(nbuf);
    std::vector<float2*> bufs(nbuf);
    for (int i = 0; i < nbuf; ++i) bufs[i] = (float2*)ctx->ws(ctx->state_pool[i], sb);
    std::vector<dense::Node> nodes;
    std::vector<uint32_t> fresh;
    for (const Act& x : acts) {
        if (x.pass == J) continue;
        dense::Node nd{};
        nd.src = x.src >= 0 ? bufs[x.src] : nullptr;
        nd.dst = bufs[x.dst];
        nd.ov_begin = ovb[x.rep];
        nd.ov_end = ove[x.rep];
        nd.part = 0;
        nodes.push_back(nd);
    }
    std::vector<unsigned char> buf;
    Blob b(buf);
    const size_t o_n = b.add(nodes), o_o = b.add(ovr), o_p = b.add(pool), o_w = b.add(wmix), o_q = b.add(qa);
    unsigned char* d = (unsigned char*)ctx->ws(ctx->dense_tabs, buf.size());
    ctx->h2d(d, buf.data(), buf.size());
    if (!d_status) d_status = (uint8_t*)ctx->ws(ctx->stream_status, count);
    const int ob = n - dense::kT;
    double* part = (double*)ctx->ws(ctx->part, ((size_t)1 << ob) * sizeof(double));
    float* d_scale = (float*)ctx->ws(ctx->scale, sizeof(float));
    reserve_sampler(ctx, c, 1);
    DenseArgs A = dense_args(P, n);
    A.ovr = (const dense::Override*)(d + o_o);
    A.opool = (const float2*)(d + o_p);
    A.part = part;
    A.n_nodes = 1;
    const dense::Node* dn = (const dense::Node*)(d + o_n);
    const uint64_t base = s.shot_off[first];
    size_t ni = 0;
    ctx->dense_launches = 0;
    ctx->dense_fma = 0;
    for (const Act& x : acts) {
        if (x.pass < J) {
            ctx->dense_launches += 1;
            ctx->dense_fma += (double)P.pass_fma[x.pass] * (double)(1ull << n);
            A.nodes = dn + ni++;
            A.pass = (int)x.pass;
            A.last = x.pass + 1 == J ? 1 : 0;
            A.stage_bytes = P.passes[x.pass].stage_bytes;
            ctx->timed(PTSBE_TIMER_DENSE, dense_bytes(n, 1, x.src < 0 ? 1 : 0), [&] { launch_dense_pass(A, ctx->n_sm, ctx->stream); });
            continue;
        }
        const uint32_t a = x.rep;
        EvolveArgs E{};
        E.n = n;
        E.tb = dense::kT;
        E.part = part;
        E.wmix = (const double*)(d + o_w) + a;
        E.qalpha = (const double*)(d + o_q) + a;
        E.weights = d_weights ? d_weights + a : nullptr;
        E.status = d_status + a;
        E.states = bufs[x.src];
        ctx->timed(PTSBE_TIMER_EVOLVE_FINALIZE, 2.0 * (double)sb, [&] { launch_evolve_finalize(E, 1, d_scale, ctx->stream, true); });
        if (s.shots[first + a])
            sample_range(ctx, s, c, first + a, 1, bufs[x.src], d_status + a, seed, d_bits + (s.shot_off[first + a] - base), nullptr);
    }
}

// ---- one persistent launch over many jobs (ptsbe_batch_*) --------------------------------------

// The sampler launches of ptsbe_sample_shots for a range, planned up front (same kernels, items and
// counters as sample_range), so that a run enqueues kernels only.
void plan_samples(const ptsbe_ctx* ctx, const KSet& s, const Circuit& c, uint32_t first, uint32_t count,
                  const float2* states, const uint8_t* status, uint64_t seed, uint32_t* bits,
                  std::vector<SampleItem>& items, std::vector<PlannedSample>& out) {
    const int n = (int)c.n;
    SampleArgs A{};
    A.n = n; A.states = states; A.status = status; A.seed = seed; A.bits = bits;
    const bool light_ok = n > 14 && n <= sample_light_max_qubits();
    const uint64_t cl = n <= 14 ? 1 : (1ull << (n - 14));
    const uint64_t clusters = std::max<uint64_t>(1, (uint64_t)ctx->n_sm / cl);
    const uint64_t base = s.shot_off[first];
    uint64_t total = 0;
    for (uint32_t a = 0; a < count; ++a) total += s.shots[first + a];
    const uint64_t chunk = sample_chunk(n, total, clusters);
    std::vector<SampleItem> light, heavy;
    for (uint32_t a = 0; a < count; ++a) {
        const uint32_t alpha = first + a;
        const uint64_t m = s.shots[alpha], o = s.shot_off[alpha] - base;
        if (m == 0) continue;
        if (light_ok && m <= ctx->light_shots) { light.push_back({a, alpha, 0, m, o, kDomShot, 0}); continue; }
        if (n <= sample_cluster_max_qubits()) {
            for (uint64_t j0 = 0; j0 < m; j0 += chunk) heavy.push_back({a, alpha, j0, std::min(m, j0 + chunk), o + j0, kDomShot, 0});
        } else {
            PlannedSample g{};
            g.kind = 2; g.A = A; g.state = a; g.alpha = alpha; g.m = m; g.out0 = o;
            out.push_back(g);
        }
    }
    if (!light.empty()) {
        PlannedSample p{};
        p.kind = 0; p.A = A; p.item_off = items.size(); p.n_items = (uint32_t)light.size();
        items.insert(items.end(), light.begin(), light.end());
        out.push_back(p);
    }
    if (!heavy.empty()) {
        PlannedSample p{};
        p.kind = 1; p.A = A; p.item_off = items.size(); p.n_items = (uint32_t)heavy.size();
        items.insert(items.end(), heavy.begin(), heavy.end());
        out.push_back(p);
    }
}

// Enqueues one run of a batch: counters cleared, the persistent queue launch, the samplers.
void batch_enqueue(ptsbe_ctx* ctx, Batch& B) {
    QueueArgs qa = B.qa;
    qa.spin_cycles = ctx->queue_spin_cycles;
    qa.stall_task = ctx->queue_stall_task < 0 ? 0xFFFFFFFFu : (uint32_t)ctx->queue_stall_task;
    PTSBE_CUDA(cudaMemsetAsync(B.dws, 0, B.counter_bytes, ctx->stream));
    launch_dense_queue(qa, ctx->n_sm, ctx->stream);
    for (const PlannedSample& p : B.samples) {
        if (p.kind == 0) launch_sample_light(p.A, p.items, p.n_items, ctx->stream);
        else if (p.kind == 1) launch_sample_cluster(p.A, p.items, p.n_items, ctx->stream);
        else launch_sample_global(p.A, p.state, p.alpha, 0, p.m, p.out0, ctx->stream);
    }
}

}  // namespace

extern "C" {

int ptsbe_create(ptsbe_ctx** out, int device, void* cuda_stream) {
    if (!out) return PTSBE_ERR_INVALID;
    *out = nullptr;
    std::unique_ptr<ptsbe_ctx> ctx;
    try {
        ctx.reset(new ptsbe_ctx());
    } catch (...) {
        return PTSBE_ERR_OOM;
    }
    ctx->device = device < 0 ? -1 : device;
    ctx->stream = (cudaStream_t)cuda_stream;
    if (device >= 0) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) {
            (void)cudaGetLastError();
            return PTSBE_ERR_NO_DEVICE;
        }
        if (cudaSetDevice(device) != cudaSuccess) { (void)cudaGetLastError(); return PTSBE_ERR_CUDA; }
        if (cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            (void)cudaGetLastError();
            return PTSBE_ERR_CUDA;
        }
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        const uint64_t keep = UINT64_MAX;   // freed blocks stay in the pool for the next call
        if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess ||
            cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, (void*)&keep) != cudaSuccess) {
            (void)cudaGetLastError();
            return PTSBE_ERR_CUDA;
        }
        // The auxiliary stream runs the prepass ahead of the context stream: at the highest
        // priority its CTAs are dispatched before the remaining CTAs of launches already running,
        // so the prepass starts as soon as SM slots free up.
        int prio_least = 0, prio_greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
            (void)cudaGetLastError();
            prio_greatest = 0;
        }
        if (cudaStreamCreateWithPriority(&ctx->aux, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_used[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_used[1], cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            if (ctx->aux) cudaStreamDestroy(ctx->aux);
            for (cudaEvent_t e : {ctx->ev_fork, ctx->ev_join, ctx->ev_used[0], ctx->ev_used[1]})
                if (e) cudaEventDestroy(e);
            cudaMemPoolDestroy(ctx->pool);
            return PTSBE_ERR_CUDA;
        }
    }
    *out = ctx.release();
    return PTSBE_OK;
}

int ptsbe_destroy(ptsbe_ctx* ctx) {
    if (!ctx) return PTSBE_ERR_INVALID;
    int status = PTSBE_OK;
    // Every free is attempted even after a failed one (a device error left by an earlier kernel
    // makes them all fail); nothing throws out of this call.
    if (ctx->has_device()) try {
        auto qfree = [&](void* p) {
            if (p && cudaFreeAsync(p, ctx->stream) != cudaSuccess) status = PTSBE_ERR_CUDA;
        };
        cudaSetDevice(ctx->device);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) status = PTSBE_ERR_CUDA;
        if (ctx->aux && cudaStreamSynchronize(ctx->aux) != cudaSuccess) status = PTSBE_ERR_CUDA;
        for (auto& kv : ctx->circuits) {
            qfree(kv.second->dev.base); qfree(kv.second->dev_pershot.base); qfree(kv.second->dev_frame.base);
            qfree(kv.second->bw.dev); qfree(kv.second->dense.dev);
            for (DeviceCircuit* d : {&kv.second->dev, &kv.second->dev_pershot, &kv.second->dev_frame})
                if (d->ready) cudaEventDestroy(d->ready);
        }
        for (auto& kv : ctx->sets) {
            qfree(kv.second->d_site);   // d_k shares the allocation
            if (kv.second->ready) cudaEventDestroy(kv.second->ready);
        }
        for (auto& kv : ctx->batches) {
            qfree(kv.second->dtab);
            qfree(kv.second->dws);
            if (kv.second->graph) cudaGraphExecDestroy(kv.second->graph);
        }
        cudaStreamSynchronize(ctx->stream);
        if (ctx->aux) {
            if (cudaStreamSynchronize(ctx->aux) != cudaSuccess) status = PTSBE_ERR_CUDA;
            cudaStreamDestroy(ctx->aux);
        }
        if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
        if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
        for (int l = 0; l < 2; ++l) {
            if (ctx->ev_used[l]) cudaEventDestroy(ctx->ev_used[l]);
            ctx->free_buf(ctx->ahead_nodes[l]);
            ctx->free_buf(ctx->ahead_progs[l]);
        }
        ctx->free_staging();
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        ctx->free_buf(ctx->nodes); ctx->free_buf(ctx->part); ctx->free_buf(ctx->scale);
        ctx->free_buf(ctx->items); ctx->free_buf(ctx->scratch); ctx->free_buf(ctx->pershot);
        ctx->free_buf(ctx->progs); ctx->free_buf(ctx->pingpong); ctx->free_buf(ctx->fault); ctx->free_buf(ctx->support);
        ctx->free_buf(ctx->dense_tabs); ctx->free_buf(ctx->stream_status); ctx->free_buf(ctx->sitems);
        ctx->free_buf(ctx->dense_pad);
        for (DevBuf& b : ctx->state_pool) ctx->free_buf(b);
        ctx->free_timers();
    } catch (const Error& e) {
        status = e.status;
    } catch (...) {
        status = PTSBE_ERR_CUDA;
    }
    delete ctx;
    return status;
}

int ptsbe_set_stream(ptsbe_ctx* ctx, void* cuda_stream) {
    return guarded(ctx, [&] { ctx->stream = (cudaStream_t)cuda_stream; });
}

const char* ptsbe_last_error(const ptsbe_ctx* ctx) {
    return ctx ? ctx->err.c_str() : "null context";
}

int ptsbe_synchronize(ptsbe_ctx* ctx) {
    return guarded(ctx, [&] {
        ctx->need_device();
        ctx->use_device();
        PTSBE_CUDA(cudaStreamSynchronize(ctx->stream));
        PTSBE_CUDA(cudaGetLastError());
        for (auto& kv : ctx->batches) {
            uint32_t e = 0;
            PTSBE_CUDA(cudaMemcpy(&e, kv.second->d_err, sizeof(e), cudaMemcpyDeviceToHost));
            if (e) {
                PTSBE_CUDA(cudaMemset(kv.second->d_err, 0, sizeof(e)));
                fail(PTSBE_ERR_TIMEOUT, "batch " + std::to_string(kv.first) + ": the work queue's wait for task " +
                                            std::to_string(e - 1) + " ran out; the batch's outputs are incomplete");
            }
        }
        if (ctx->fault.p) {
            uint32_t f = 0;
            PTSBE_CUDA(cudaMemcpy(&f, ctx->fault.p, sizeof(f), cudaMemcpyDeviceToHost));
            if (f) {
                PTSBE_CUDA(cudaMemset(ctx->fault.p, 0, sizeof(f)));
                fail(PTSBE_ERR_UNSUPPORTED, "a fused sampling launch found a support it cannot order (shots left at 0xFFFFFFFF)");
            }
        }
    });
}

int ptsbe_register_circuit(ptsbe_ctx* ctx, uint32_t n_qubits, const ptsbe_op* ops, uint64_t n_ops,
                           const ptsbe_channel* channels, uint32_t n_channels, const double* custom_gates,
                           uint32_t n_custom, uint32_t* circuit_id) {
    const NvtxRange nvtx("ptsbe_register_circuit");
    return guarded(ctx, [&] {
        if (!circuit_id) fail(PTSBE_ERR_INVALID, "circuit_id is NULL");
        if (n_qubits < 1 || n_qubits > (uint32_t)kMaxQubits) fail(PTSBE_ERR_INVALID, "n_qubits must be in [1, 32]");
        if (n_ops && !ops) fail(PTSBE_ERR_INVALID, "ops is NULL");
        if (n_channels && !channels) fail(PTSBE_ERR_INVALID, "channels is NULL");
        auto c = std::make_unique<Circuit>();
        c->n = n_qubits;
        c->ch.resize(n_channels);
        for (uint32_t j = 0; j < n_channels; ++j) build_channel(channels[j], c->ch[j]);
        register_ops(*c, ops, n_ops, custom_gates, n_custom);
        build_device_ops(*c);
        // plans and device tables are built by the first call that needs them
        const uint32_t id = ctx->next_circuit++;
        ctx->circuits[id] = std::move(c);
        *circuit_id = id;
    });
}

int ptsbe_circuit_info(ptsbe_ctx* ctx, uint32_t circuit_id, uint32_t* n_qubits, uint64_t* n_sites, uint64_t* n_gates) {
    return guarded(ctx, [&] {
        Circuit& c = ctx->circuit(circuit_id);
        if (n_qubits) *n_qubits = c.n;
        if (n_sites) *n_sites = c.site_op.size();
        if (n_gates) *n_gates = c.n_gates;
    });
}

int ptsbe_release_circuit(ptsbe_ctx* ctx, uint32_t circuit_id) {
    return guarded(ctx, [&] {
        Circuit& c = ctx->circuit(circuit_id);
        if (ctx->has_device()) {
            ctx->use_device();
            free_device_circuit(ctx, c.dev);            // stream-ordered: after the launches that use them
            free_device_circuit(ctx, c.dev_pershot);
            free_device_circuit(ctx, c.dev_frame);
            ctx->dfree(c.bw.dev);
            c.bw.dev = nullptr;
            ctx->dfree(c.dense.dev);
            c.dense.dev = nullptr;
        }
        ctx->circuits.erase(circuit_id);
    });
}

int ptsbe_sample_kraus(ptsbe_ctx* ctx, uint32_t circuit_id, const ptsbe_pts_params* params, uint64_t seed,
                       uint32_t* set_id, uint32_t* count, uint64_t* n_entries, uint64_t* total_shots) {
    const NvtxRange nvtx("ptsbe_sample_kraus");
    return guarded(ctx, [&] {
        if (!params) fail(PTSBE_ERR_INVALID, "params is NULL");
        Circuit& c = ctx->circuit(circuit_id);
        auto s = std::make_unique<KSet>();
        s->circuit = circuit_id;
        pts_run(c, *params, seed, *s);
        if (s->count() > 0xFFFFFFF0u) fail(PTSBE_ERR_UNSUPPORTED, "too many sets");
        const uint32_t id = ctx->next_set++;
        if (count) *count = s->count();
        if (n_entries) *n_entries = s->site.size();
        if (total_shots) *total_shots = s->shot_off.back();
        ctx->sets[id] = std::move(s);
        if (set_id) *set_id = id;
    });
}

int ptsbe_set_export(ptsbe_ctx* ctx, uint32_t set_id, const ptsbe_set_view* out) {
    return guarded(ctx, [&] {
        if (!out) fail(PTSBE_ERR_INVALID, "out is NULL");
        const KSet& s = ctx->set(set_id);
        const uint32_t n = s.count();
        if (out->offsets) std::memcpy(out->offsets, s.off.data(), (n + 1) * sizeof(uint32_t));
        if (out->sites && !s.site.empty()) std::memcpy(out->sites, s.site.data(), s.site.size() * sizeof(uint32_t));
        if (out->kidx && !s.k.empty()) std::memcpy(out->kidx, s.k.data(), s.k.size());
        if (out->mult && n) std::memcpy(out->mult, s.mult.data(), n * sizeof(uint64_t));
        if (out->q && n) std::memcpy(out->q, s.q.data(), n * sizeof(double));
        if (out->shots && n) std::memcpy(out->shots, s.shots.data(), n * sizeof(uint64_t));
        if (out->shot_offsets) std::memcpy(out->shot_offsets, s.shot_off.data(), (n + 1) * sizeof(uint64_t));
    });
}

int ptsbe_release_set(ptsbe_ctx* ctx, uint32_t set_id) {
    return guarded(ctx, [&] {
        KSet& s = ctx->set(set_id);
        if (ctx->has_device() && s.d_site) {
            ctx->use_device();
            ctx->dfree(s.d_site);                        // stream-ordered (d_k shares the allocation)
        }
        if (s.ready) cudaEventDestroy(s.ready);
        ctx->sets.erase(set_id);
    });
}

int ptsbe_evolve_batch(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count, void* d_states,
                       double* d_weights, uint8_t* d_status, uint32_t flags) {
    const NvtxRange nvtx("ptsbe_evolve_batch");
    return guarded(ctx, [&] {
        ctx->need_device();
        KSet& s = ctx->set(set_id);
        Circuit& c = ctx->circuit(s.circuit);
        if ((uint64_t)first + count > s.count()) fail(PTSBE_ERR_INVALID, "set range out of bounds");
        if (count == 0) return;
        if (flags & ~(uint32_t)(PTSBE_EVOLVE_PREFIX_REUSE | PTSBE_EVOLVE_PLAN_ONLY)) fail(PTSBE_ERR_INVALID, "unknown flags");
        const bool plan_only = flags & PTSBE_EVOLVE_PLAN_ONLY;
        if (!d_states && !plan_only) fail(PTSBE_ERR_INVALID, "d_states is NULL");
        if ((uintptr_t)d_states % 16) fail(PTSBE_ERR_INVALID, "d_states must be 16-byte aligned");
        evolve_range(ctx, s, c, first, count, d_states, d_weights, d_status, flags, nullptr, nullptr);
    });
}

int ptsbe_sample_shots(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count, const void* d_states,
                       const uint8_t* d_status, uint64_t seed, uint32_t* d_bits, uint64_t d_bits_capacity) {
    const NvtxRange nvtx("ptsbe_sample_shots");
    return guarded(ctx, [&] {
        ctx->need_device();
        KSet& s = ctx->set(set_id);
        Circuit& c = ctx->circuit(s.circuit);
        if ((uint64_t)first + count > s.count()) fail(PTSBE_ERR_INVALID, "set range out of bounds");
        if (count == 0) return;
        const uint64_t base = s.shot_off[first];
        const uint64_t total = s.shot_off[first + count] - base;
        if (total == 0) return;
        if (!d_states || !d_bits) fail(PTSBE_ERR_INVALID, "null device pointer");
        if ((uintptr_t)d_states % 16) fail(PTSBE_ERR_INVALID, "d_states must be 16-byte aligned");
        if (d_bits_capacity < total) fail(PTSBE_ERR_BUFFER_TOO_SMALL, "d_bits holds " + std::to_string(d_bits_capacity) +
                                                                          " shots, the range needs " + std::to_string(total));
        if (c.n > 32) fail(PTSBE_ERR_UNSUPPORTED, "outcomes are 32-bit");
        ctx->use_device();
        sample_range(ctx, s, c, first, count, d_states, d_status, seed, d_bits, nullptr);
    });
}

int ptsbe_evolve_sample(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count, void* d_states,
                        double* d_weights, uint8_t* d_status, uint32_t flags, uint64_t seed, uint32_t* d_bits,
                        uint64_t d_bits_capacity) {
    const NvtxRange nvtx("ptsbe_evolve_sample");
    return guarded(ctx, [&] {
        ctx->need_device();
        KSet& s = ctx->set(set_id);
        Circuit& c = ctx->circuit(s.circuit);
        if ((uint64_t)first + count > s.count()) fail(PTSBE_ERR_INVALID, "set range out of bounds");
        if (count == 0) return;
        if ((uintptr_t)d_states % 16) fail(PTSBE_ERR_INVALID, "d_states must be 16-byte aligned");
        if (flags & ~(uint32_t)(PTSBE_EVOLVE_PREFIX_REUSE | PTSBE_EVOLVE_PLAN_ONLY)) fail(PTSBE_ERR_INVALID, "unknown flags");
        const bool plan_only = flags & PTSBE_EVOLVE_PLAN_ONLY;
        const uint64_t total = s.shot_off[first + count] - s.shot_off[first];
        if (plan_only) {
            if (!d_states && (int)c.n >= dense::kT) stream_evolve_sample(ctx, s, c, first, count, nullptr, nullptr, seed, nullptr, true);
            else evolve_range(ctx, s, c, first, count, d_states, nullptr, nullptr, flags, nullptr, nullptr);
            return;
        }
        if (total && !d_bits) fail(PTSBE_ERR_INVALID, "null device pointer");
        if (d_bits_capacity < total) fail(PTSBE_ERR_BUFFER_TOO_SMALL, "d_bits holds " + std::to_string(d_bits_capacity) +
                                                                          " shots, the range needs " + std::to_string(total));
        if (total && c.n > 32) fail(PTSBE_ERR_UNSUPPORTED, "outcomes are 32-bit");
        if (!d_states) {
            if ((int)c.n < dense::kT) fail(PTSBE_ERR_UNSUPPORTED, "d_states may be NULL only for n >= 12 (dense passes)");
            ctx->use_device();
            ensure_set_on_device(ctx, s);
            stream_evolve_sample(ctx, s, c, first, count, d_weights, d_status, seed, d_bits, false);
            return;
        }
        std::vector<uint8_t> drawn;
        const FusedShots fs{seed, d_bits};
        ctx->use_device();
        if (total) reserve_sampler(ctx, c, count);
        SampleRun run;
        evolve_range(ctx, s, c, first, count, d_states, d_weights, d_status, flags, total ? &fs : nullptr, &drawn, [&] {
            if (total) run = plan_sample_range(ctx, s, c, first, count, d_states, d_status, seed, d_bits, &drawn);
        });
        if (total) launch_sample_range(ctx, run);
    });
}

int ptsbe_unique_shots(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count, const uint32_t* d_bits,
                       uint64_t* d_unique) {
    const NvtxRange nvtx("ptsbe_unique_shots");
    return guarded(ctx, [&] {
        ctx->need_device();
        KSet& s = ctx->set(set_id);
        Circuit& c = ctx->circuit(s.circuit);
        if ((uint64_t)first + count > s.count()) fail(PTSBE_ERR_INVALID, "set range out of bounds");
        if (count == 0) return;
        if (!d_bits || !d_unique) fail(PTSBE_ERR_INVALID, "null device pointer");
        if ((int)c.n > unique_max_qubits()) fail(PTSBE_ERR_UNSUPPORTED, "unique-shot statistic handles n <= 20");
        ctx->use_device();
        // pieces (set, begin, end) of at most 2^18 shots, so heavy sets spread over many CTAs
        const uint64_t base = s.shot_off[first];
        const uint64_t piece = 1ull << 18;
        std::vector<uint64_t> pieces;
        for (uint32_t a = 0; a < count; ++a) {
            const uint64_t b0 = s.shot_off[first + a] - base, b1 = s.shot_off[first + a + 1] - base;
            for (uint64_t x = b0; x < b1; x += piece) pieces.insert(pieces.end(), {(uint64_t)a, x, std::min(b1, x + piece)});
        }
        const uint32_t np = (uint32_t)(pieces.size() / 3);
        const size_t bm_bytes = unique_bitmap_bytes((int)c.n) * count;
        unsigned char* buf = (unsigned char*)ctx->dalloc(((bm_bytes + 255) & ~(size_t)255) + std::max<size_t>(pieces.size(), 1) * 8);
        uint32_t* d_bm = (uint32_t*)buf;
        uint64_t* d_p = (uint64_t*)(buf + ((bm_bytes + 255) & ~(size_t)255));
        PTSBE_CUDA(cudaMemsetAsync(d_bm, 0, bm_bytes, ctx->stream));
        if (np) ctx->h2d(d_p, pieces.data(), pieces.size() * sizeof(uint64_t));
        launch_unique(d_bits, d_p, np, count, (int)c.n, d_bm, (unsigned long long*)d_unique, ctx->stream);
        ctx->dfree(buf);
    });
}

int ptsbe_set_option(ptsbe_ctx* ctx, int option, int64_t value) {
    return guarded(ctx, [&] {
        if (option == PTSBE_OPT_EVOLVE_KERNEL) {
            if (value < 0 || value > 4) fail(PTSBE_ERR_INVALID, "evolve kernel must be 0 .. 4");
            ctx->evolve_kernel = (int)value;
        } else if (option == PTSBE_OPT_LIGHT_SHOTS) {
            if (value < 0) fail(PTSBE_ERR_INVALID, "light-sampler shot limit must be >= 0");
            ctx->light_shots = (uint64_t)value;
        } else if (option == PTSBE_OPT_QUEUE_SPIN_CYCLES) {
            if (value <= 0) fail(PTSBE_ERR_INVALID, "queue wait budget must be positive");
            ctx->queue_spin_cycles = value;
        } else if (option == PTSBE_OPT_QUEUE_STALL_TASK) {
            if (value < -1) fail(PTSBE_ERR_INVALID, "stall task must be >= -1");
            ctx->queue_stall_task = value;
        } else if (option == PTSBE_OPT_FAIL_ALLOC) {
            if (value < -1) fail(PTSBE_ERR_INVALID, "allocation failure index must be >= -1");
            ctx->fail_alloc_at = value;
            ctx->alloc_count = 0;
        } else if (option == PTSBE_OPT_PERSHOT_TILE_BITS) {
            if (value != 0 && (value < 9 || value > kTileMax)) fail(PTSBE_ERR_INVALID, "per-shot tile bits must be 0 or 9 to 14");
            ctx->pershot_tile_bits = (int)value;
        } else if (option == PTSBE_OPT_SPLIT_FILL) {
            if (value < 0 || value > 100) fail(PTSBE_ERR_INVALID, "split fill must be a percentage, 0 to 100");
            ctx->split_fill = (int)value;
        } else if (option == PTSBE_OPT_PREPASS_AHEAD) {
            if (value != 0 && value != 1) fail(PTSBE_ERR_INVALID, "prepass ahead must be 0 or 1");
            ctx->prepass_ahead = (int)value;
        } else if (option == PTSBE_OPT_PROGRAM_SETS_PER_WARP) {
            if (value != 0 && value != 4 && value != 8 && value != 16) fail(PTSBE_ERR_INVALID, "sets per warp must be 0, 4, 8 or 16");
            ctx->prog_sets_per_warp = value ? (int)value : 8;
        } else {
            fail(PTSBE_ERR_INVALID, "unknown option");
        }
    });
}

int ptsbe_autotune(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count, void* d_states, double* d_weights,
                   uint8_t* d_status, uint32_t flags, uint64_t seed, uint32_t* d_bits, uint64_t d_bits_capacity,
                   uint32_t reps, ptsbe_tuning* out) {
    const NvtxRange nvtx("ptsbe_autotune");
    return guarded(ctx, [&] {
        ctx->need_device();
        if (reps == 0) fail(PTSBE_ERR_INVALID, "reps must be positive");
        ctx->use_device();
        ptsbe_tuning t{};
        cudaEvent_t e0, e1;
        PTSBE_CUDA(cudaEventCreate(&e0));
        PTSBE_CUDA(cudaEventCreate(&e1));
        auto timed_ms = [&](auto&& call) {
            int st = call();                                   // warm-up (plans, tables, workspace)
            if (st != PTSBE_OK) return -1.0;
            PTSBE_CUDA(cudaEventRecord(e0, ctx->stream));
            for (uint32_t r = 0; r < reps && st == PTSBE_OK; ++r) st = call();
            PTSBE_CUDA(cudaEventRecord(e1, ctx->stream));
            PTSBE_CUDA(cudaEventSynchronize(e1));
            if (st != PTSBE_OK) return -1.0;
            float ms = 0;
            PTSBE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            return (double)ms / reps;
        };
        const int keep_kernel = ctx->evolve_kernel;
        const uint64_t keep_light = ctx->light_shots;
        int best_k = -1;
        double best = 0;
        try {
            for (int k : {3, 1, 2, 4}) {
                ctx->evolve_kernel = k;
                const double ms = timed_ms([&] { return ptsbe_evolve_batch(ctx, set_id, first, count, d_states, d_weights, d_status, flags); });
                if (ms < 0) fail(PTSBE_ERR_INVALID, std::string("autotune: evolve kernel ") + std::to_string(k) + ": " + ctx->err);
                t.evolve_ms[k] = ms;
                if (best_k < 0 || ms < best) { best = ms; best_k = k; }
            }
            ctx->evolve_kernel = best_k;
            PTSBE_CUDA(cudaStreamSynchronize(ctx->stream));
            // the shot limit splits states between the sampling fused into the last evolve launch
            // (or the one-CTA sampler) and the cluster sampler: timed on the one-call path
            const uint64_t cand[4] = {512, 4096, 65536, 1ull << 20};
            int best_l = -1;
            double best_s = 0;
            for (int i = 0; i < 4; ++i) {
                ctx->light_shots = cand[i];
                t.light_candidates[i] = cand[i];
                const double ms = timed_ms([&] {
                    return ptsbe_evolve_sample(ctx, set_id, first, count, d_states, d_weights, d_status, flags, seed, d_bits,
                                               d_bits_capacity);
                });
                if (ms < 0) fail(PTSBE_ERR_INVALID, "autotune: sampler: " + ctx->err);
                t.sample_ms[i] = ms;
                if (best_l < 0 || ms < best_s) { best_s = ms; best_l = i; }
            }
            ctx->light_shots = cand[best_l];
        } catch (...) {
            ctx->evolve_kernel = keep_kernel;
            ctx->light_shots = keep_light;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        t.evolve_kernel = ctx->evolve_kernel;
        t.light_shots = ctx->light_shots;
        if (out) *out = t;
    });
}

int ptsbe_set_timing(ptsbe_ctx* ctx, int enable) {
    return guarded(ctx, [&] {
        ctx->need_device();
        ctx->timing = enable != 0;
    });
}

int ptsbe_get_timing(ptsbe_ctx* ctx, int kernel_class, double* ms, uint64_t* launches, double* bytes, int reset) {
    return guarded(ctx, [&] {
        ctx->need_device();
        if (kernel_class < 0 || kernel_class >= PTSBE_TIMER_CLASSES) fail(PTSBE_ERR_INVALID, "unknown kernel class");
        ctx->use_device();
        ctx->collect_timers();
        ClassTimer& t = ctx->timers[kernel_class];
        if (ms) *ms = t.ms;
        if (launches) *launches = t.launches;
        if (bytes) *bytes = t.bytes;
        if (reset) { t.ms = 0; t.launches = 0; t.bytes = 0; }
    });
}

int ptsbe_kernel_launches(uint64_t* count) {
    if (!count) return PTSBE_ERR_INVALID;
    *count = launches_so_far();
    return PTSBE_OK;
}

int ptsbe_h2d_bytes(uint64_t* bytes) {
    if (!bytes) return PTSBE_ERR_INVALID;
    *bytes = g_h2d.load(std::memory_order_relaxed);
    return PTSBE_OK;
}

int ptsbe_reuse_stats(ptsbe_ctx* ctx, uint64_t* gates_applied, uint64_t* gates_without_reuse) {
    return guarded(ctx, [&] {
        if (gates_applied) *gates_applied = ctx->reuse_gates_run;
        if (gates_without_reuse) *gates_without_reuse = ctx->reuse_gates_full;
    });
}

int ptsbe_dense_work(ptsbe_ctx* ctx, uint64_t* pass_launches, double* fma) {
    return guarded(ctx, [&] {
        if (pass_launches) *pass_launches = ctx->dense_launches;
        if (fma) *fma = ctx->dense_fma;
    });
}

int ptsbe_dense_plan_info(ptsbe_ctx* ctx, uint32_t circuit_id, uint32_t* passes, uint32_t* fixup_passes,
                          uint64_t* blocks_1q, uint64_t* blocks_2q, double* fma_per_amplitude) {
    return guarded(ctx, [&] {
        Circuit& c = ctx->circuit(circuit_id);
        if (!c.dense.built) make_dense_plan(c, c.dense);
        const DensePlan& P = c.dense;
        uint64_t b1 = 0, b2 = 0;
        for (uint8_t q : P.blk_nq) (q == 1 ? b1 : b2) += 1;
        double f = 0;
        for (uint32_t x : P.pass_fma) f += x;
        if (passes) *passes = (uint32_t)P.passes.size();
        if (fixup_passes) *fixup_passes = P.fixup_passes;
        if (blocks_1q) *blocks_1q = b1;
        if (blocks_2q) *blocks_2q = b2;
        if (fma_per_amplitude) *fma_per_amplitude = f;
    });
}

int ptsbe_sample_shots_noalloc(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count, const void* d_states,
                               const uint8_t* d_status, uint64_t seed, uint32_t* d_bits, uint64_t d_bits_capacity) {
    const NvtxRange nvtx("ptsbe_sample_shots_noalloc");
    return guarded(ctx, [&] {
        ctx->need_device();
        KSet& s = ctx->set(set_id);
        Circuit& c = ctx->circuit(s.circuit);
        if ((uint64_t)first + count > s.count()) fail(PTSBE_ERR_INVALID, "set range out of bounds");
        if (count == 0) return;
        const uint64_t base = s.shot_off[first];
        const uint64_t total = s.shot_off[first + count] - base;
        if (total == 0) return;
        if (!d_states || !d_bits) fail(PTSBE_ERR_INVALID, "null device pointer");
        if ((uintptr_t)d_states % 16) fail(PTSBE_ERR_INVALID, "d_states must be 16-byte aligned");
        if (d_bits_capacity < total) fail(PTSBE_ERR_BUFFER_TOO_SMALL, "d_bits holds " + std::to_string(d_bits_capacity) +
                                                                          " shots, the range needs " + std::to_string(total));
        const int n = (int)c.n;
        const size_t cap = noalloc_scratch_bytes();
        SampleArgs A{};
        A.n = n;
        A.states = (const float2*)d_states;
        A.status = d_status;
        A.seed = seed;
        A.bits = d_bits;
        if (n <= sample_cluster_max_qubits()) {
            const uint64_t cl = n <= 14 ? 1 : (1ull << (n - 14));
            const uint64_t clusters = std::max<uint64_t>(1, (uint64_t)ctx->n_sm / cl);
            const uint64_t chunk = sample_chunk(n, total, clusters);
            std::vector<SampleItem>& items = ctx->noalloc_items;
            items.clear();
            for (uint32_t a = 0; a < count; ++a) {
                const uint32_t alpha = first + a;
                const uint64_t m = s.shots[alpha], o = s.shot_off[alpha] - base;
                for (uint64_t j0 = 0; j0 < m; j0 += chunk)
                    items.push_back({a, alpha, j0, std::min(m, j0 + chunk), o + j0, kDomShot, 0});
            }
            if (items.size() > noalloc_max_items() || items.size() * sizeof(SampleItem) > cap)
                fail(PTSBE_ERR_UNSUPPORTED, "range needs " + std::to_string(items.size()) + " work items; the fixed scratch holds " +
                                                std::to_string(noalloc_max_items()));
            ctx->use_device();
            SampleItem* d_items = (SampleItem*)noalloc_scratch(ctx->device);
            // Through a pinned staging slot that already has room (asynchronous); otherwise from
            // pageable host memory, which allocates nothing either but first waits for the work
            // already queued on the stream (documented in the header).
            const size_t ib = items.size() * sizeof(SampleItem);
            if (!ctx->h2d_no_growth(d_items, items.data(), ib))
                PTSBE_CUDA(cudaMemcpyAsync(d_items, items.data(), ib, cudaMemcpyHostToDevice, ctx->stream));
            launch_sample_cluster(A, d_items, (uint32_t)items.size(), ctx->stream);
        } else {
            const size_t need = sample_global_scratch_doubles(n) * 8;
            if (n > noalloc_max_qubits() || need > cap)
                fail(PTSBE_ERR_UNSUPPORTED, std::to_string(n) + "-qubit states need " + std::to_string(need) +
                                                " bytes of CDF workspace; the fixed scratch holds " + std::to_string(cap) +
                                                " (at most 21 qubits)");
            ctx->use_device();
            A.scratch = (unsigned long long*)noalloc_scratch(ctx->device);
            for (uint32_t a = 0; a < count; ++a) {
                const uint32_t alpha = first + a;
                const uint64_t m = s.shots[alpha], o = s.shot_off[alpha] - base;
                if (m) launch_sample_global(A, a, alpha, 0, m, o, ctx->stream);
            }
        }
    });
}

int ptsbe_backward_plan_info(ptsbe_ctx* ctx, uint32_t circuit_id, uint32_t* blocks_1q, uint32_t* blocks_2q,
                             uint32_t* swaps, uint32_t* differentiable_blocks, uint32_t* conditioning_checkpoints) {
    return guarded(ctx, [&] {
        Circuit& c = ctx->circuit(circuit_id);
        if (c.n > (uint32_t)kBwMaxQubits) fail(PTSBE_ERR_UNSUPPORTED, "backward handles at most 16 qubits");
        BwPlan local;
        const BwPlan* P = &c.bw;
        if (!c.bw.built) { make_backward_plan(c, local); P = &local; }
        uint32_t n1 = 0, n2 = 0, ns = 0, nd = 0;
        for (const BwItem& it : P->items) { (it.nq == 2 ? n2 : n1)++; nd += it.diff ? 1u : 0u; }
        for (const BwStep& st : P->steps) ns += st.kind == 1 ? 1u : 0u;
        if (blocks_1q) *blocks_1q = n1;
        if (blocks_2q) *blocks_2q = n2;
        if (swaps) *swaps = ns;
        if (differentiable_blocks) *differentiable_blocks = nd;
        if (conditioning_checkpoints) *conditioning_checkpoints = P->cond_ckpts;
    });
}

int ptsbe_backward(ptsbe_ctx* ctx, uint32_t circuit_id, uint32_t set_id, uint32_t first, uint32_t count,
                   const ptsbe_observable* obs, uint32_t checkpoint_every, double* d_loss, double* d_per_set,
                   double* d_grad_params, double* d_grad_noise) {
    const NvtxRange nvtx("ptsbe_backward");
    return guarded(ctx, [&] {
        ctx->need_device();
        ctx->use_device();
        if (!obs) fail(PTSBE_ERR_INVALID, "null observable");
        if (obs->n_terms && (!obs->masks || !obs->coeffs)) fail(PTSBE_ERR_INVALID, "observable terms without masks or coefficients");
        KSet& S = ctx->set(set_id);
        Circuit& c = ctx->circuit(circuit_id);
        check_same_structure(c, ctx->circuit(S.circuit));
        if ((uint64_t)first + count > S.count()) fail(PTSBE_ERR_INVALID, "set range out of bounds");
        if (c.n > (uint32_t)kBwMaxQubits) fail(PTSBE_ERR_UNSUPPORTED, "backward handles at most 16 qubits");
        const int n = (int)c.n;
        for (uint32_t t = 0; t < obs->n_terms; ++t)
            if (obs->masks[t] >> n) fail(PTSBE_ERR_INVALID, "observable mask names a qubit >= n");
        if (!c.bw.built) {
            make_backward_plan(c, c.bw);
            upload_backward_plan(ctx, c.bw);
        }
        const BwPlan& P = c.bw;
        const uint32_t nch = (uint32_t)c.ch.size();
        // per-set weights: W = mult s^2 / (N q), s^2 = prod over unit-mixture sites of q_{s,k}
        std::vector<uint32_t> ebeg(count + 1);
        std::vector<double> W(count), s2q(count), gmix((size_t)count * std::max<uint32_t>(nch, 1), 0.0);
        std::vector<uint32_t> nsites_ch(nch, 0), nerr_ch(nch, 0);
        for (uint32_t s = 0; s < c.site_ch.size(); ++s) nsites_ch[c.site_ch[s]]++;
        double Nmult = 0;
        for (uint32_t a = 0; a < count; ++a) Nmult += (double)S.mult[first + a];
        if (count && !(Nmult > 0)) fail(PTSBE_ERR_INVALID, "sets with zero total multiplicity");
        uint32_t base_ck = (uint32_t)P.defsing_items.size() + P.cond_ckpts;
        if (checkpoint_every) base_ck += (uint32_t)((P.items.size() + checkpoint_every - 1) / checkpoint_every);
        uint32_t extra_ck = 0;
        std::vector<uint32_t> seen_items;
        for (uint32_t a = 0; a < count; ++a) {
            const uint32_t g = first + a;
            const uint32_t e0 = S.off[g], e1 = S.off[g + 1];
            if (e1 - e0 > (uint32_t)kBwMaxErr) fail(PTSBE_ERR_UNSUPPORTED, "backward handles sets of at most 64 entries");
            if (!(S.q[g] > 0)) fail(PTSBE_ERR_INVALID, "a set with q_alpha = 0");
            ebeg[a] = e0;
            double s2 = 1.0;
            std::fill(nerr_ch.begin(), nerr_ch.end(), 0u);
            for (uint32_t e = e0; e < e1; ++e) {
                const uint32_t ch = c.site_ch[S.site[e]];
                nerr_ch[ch]++;
            }
            // product over every unit-mixture site, factored as (all variant 0) x (ratios at entries)
            bool ratio_ok = P.P0mix > 0;
            for (uint32_t e = e0; e < e1 && ratio_ok; ++e) {
                const HostChannel& H = c.ch[c.site_ch[S.site[e]]];
                if (bw_unit_channel(H)) s2 *= H.q[S.k[e]] / H.q[0];
            }
            if (ratio_ok) s2 *= P.P0mix;
            else {
                s2 = 1.0;
                uint32_t e = e0;
                for (uint32_t s = 0; s < c.site_ch.size(); ++s) {
                    uint32_t k = 0;
                    if (e < e1 && S.site[e] == s) k = S.k[e++];
                    const HostChannel& H = c.ch[c.site_ch[s]];
                    if (bw_unit_channel(H)) s2 *= H.q[k];
                }
            }
            // the kernel's general-channel variants are scaled to norm 1: divide their product out
            double logC = P.logc_default;
            for (uint32_t e = e0; e < e1; ++e) {
                const uint32_t m = P.site_mem[S.site[e]];
                if (m < P.logc_off.size() && P.logc_off[m] != kBwNone)
                    logC += P.logc[P.logc_off[m] + S.k[e]] - P.logc[P.logc_off[m]];
            }
            const double invC = std::exp(-logC);
            W[a] = (double)S.mult[g] * s2 / (Nmult * S.q[g]) * invC;
            s2q[a] = s2 / S.q[g] * invC;
            for (uint32_t ch = 0; ch < nch; ++ch) {
                const HostChannel& H = c.ch[ch];
                const bool pauli_kind = H.kind == PTSBE_CH_DEPOL1 || H.kind == PTSBE_CH_DEPOL2 ||
                                        H.kind == PTSBE_CH_BITFLIP || H.kind == PTSBE_CH_PHASEFLIP;
                if (!pauli_kind) continue;
                const double p = H.param;
                const uint32_t n1 = nerr_ch[ch], n0 = nsites_ch[ch] - n1;
                double gv = 0;   // d log(prod q_k) / dp: q_0 = 1 - p, q_k = p / (d^2 - 1) or p
                if (n0) gv += -(double)n0 / (1.0 - p);
                if (n1) gv += (double)n1 / p;
                gmix[(size_t)a * nch + ch] = gv;
            }
            // items of this set whose chosen variants cannot be inverted (beyond the default ones)
            seen_items.clear();
            uint32_t ex = 0;
            for (uint32_t e = e0; e < e1; ++e) {
                const uint32_t it = P.site_item[S.site[e]];
                if (std::find(seen_items.begin(), seen_items.end(), it) != seen_items.end()) continue;
                seen_items.push_back(it);
                const BwItem& I = P.items[it];
                if (I.defsing) continue;
                bool sing = false;
                for (uint32_t m = I.mbeg; m < I.mend && !sing; ++m) {
                    uint32_t k = 0;
                    for (uint32_t f = e0; f < e1; ++f)
                        if (P.site_mem[S.site[f]] == m) k = S.k[f];
                    sing = (P.members[m].sing >> k) & 1u;
                }
                ex += sing ? 1u : 0u;
            }
            extra_ck = std::max(extra_ck, ex);
        }
        ebeg[count] = count ? S.off[first + count] : 0;
        std::vector<uint32_t> pmask(std::max<uint32_t>(obs->n_terms, 1), 0u);
        std::vector<double> coeff(std::max<uint32_t>(obs->n_terms, 1), 0.0);
        for (uint32_t t = 0; t < obs->n_terms; ++t) {
            uint32_t m = 0;
            for (int q = 0; q < n; ++q)
                if ((obs->masks[t] >> q) & 1u) m |= 1u << P.pos_final[q];
            pmask[t] = m;
            coeff[t] = obs->coeffs[t];
        }
        ensure_set_on_device(ctx, S);
        // per-call tables: one upload
        std::vector<unsigned char>& hb = ctx->host_blob;
        Blob blob(hb);
        const size_t o_eb = blob.add(ebeg), o_w = blob.add(W), o_s2 = blob.add(s2q), o_g = blob.add(gmix);
        const size_t o_pm = blob.add(pmask), o_co = blob.add(coeff);
        unsigned char* tab = (unsigned char*)ctx->dalloc(hb.size());
        ctx->h2d(tab, hb.data(), hb.size());
        // workspace
        const int nl = P.nl, cl = 1 << (n - nl);
        const uint32_t nslots = count ? backward_slots(n, count, ctx->n_sm) : 1u;
        const uint32_t maxck = base_ck + extra_ck;
        const size_t ng = P.ngs, nd = std::max<uint32_t>(P.ndslots, 1);
        const size_t b_ck = (size_t)nslots * maxck * ((size_t)8 << n);
        const size_t b_g = (size_t)nslots * cl * ng * 32 * sizeof(double);
        const size_t b_acc = ((size_t)nslots * (nd + std::max<uint32_t>(nch, 1) + 1) + nd) * sizeof(double);
        auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
        unsigned char* wsp = (unsigned char*)ctx->dalloc(al(b_ck) + 2 * al(b_g) + al(b_acc) + 256);
        unsigned char* zero_begin = wsp + al(b_ck);
        PTSBE_CUDA(cudaMemsetAsync(zero_begin, 0, 2 * al(b_g) + al(b_acc), ctx->stream));
        BwArgs A{};
        A.n = n; A.nl = nl; A.cl = cl; A.nslots = nslots; A.count = count;
        A.steps = P.d_steps; A.nsteps = (uint32_t)P.steps.size(); A.first_diff_step = P.first_diff_step;
        A.items = P.d_items; A.nitems = (uint32_t)P.items.size(); A.members = P.d_members;
        A.pool = P.d_pool; A.pool64 = P.d_pool64; A.site_item = P.d_site_item; A.site_mem = P.d_site_mem;
        A.dslot_out = P.d_dslot_out; A.pos_final = P.d_pos_final;
        A.ent_site = S.d_site; A.ent_k = S.d_k;
        A.ebeg = (const uint32_t*)(tab + o_eb); A.W = (const double*)(tab + o_w); A.s2q = (const double*)(tab + o_s2);
        A.gmix = (const double*)(tab + o_g); A.nch = (int)nch;
        A.nterms = obs->n_terms; A.pmask = (const uint32_t*)(tab + o_pm); A.coeff = (const double*)(tab + o_co);
        A.diag = obs->d_diag;
        A.ckpt_every = checkpoint_every; A.maxck = maxck; A.ngs = (uint32_t)ng; A.ndslots = P.ndslots;
        A.n_ops = (uint32_t)c.ops.size();
        A.ckpt = (float2*)wsp;
        A.Ga = (double*)zero_begin;
        A.Gbar = (double*)(zero_begin + al(b_g));
        double* acc = (double*)(zero_begin + 2 * al(b_g));
        A.acc_err = acc;
        A.acc_mix = acc + (size_t)nslots * nd;
        A.acc_loss = A.acc_mix + (size_t)nslots * std::max<uint32_t>(nch, 1);
        A.dtot = A.acc_loss + nslots;
        A.per_set = d_per_set; A.loss = d_loss; A.grad_params = d_grad_params; A.grad_noise = d_grad_noise;
        ctx->timed(PTSBE_TIMER_BACKWARD, 0.0, [&] { launch_backward(A, ctx->stream); });
        ctx->dfree(wsp);
        ctx->dfree(tab);
    });
}

int ptsbe_pershot_run(ptsbe_ctx* ctx, uint32_t circuit_id, uint64_t seed, uint64_t first_shot, uint64_t n_shots,
                      uint32_t* d_bits, uint8_t* d_kraus) {
    const NvtxRange nvtx("ptsbe_pershot_run");
    return guarded(ctx, [&] {
        ctx->need_device();
        Circuit& c = ctx->circuit(circuit_id);
        if (n_shots == 0) return;
        if (!d_bits) fail(PTSBE_ERR_INVALID, "d_bits is NULL");
        ctx->use_device();
        // Its stages break at every general noise site whatever the tile size, and a stage holds a
        // few operators, so small tiles (many CTAs per SM) stream the states best (measured).
        const int tb = ctx->pershot_tile_bits ? ctx->pershot_tile_bits : kPershotTileBits;
        if (!c.pershot_planned || c.pershot_tb != tb) {
            if (c.pershot_planned) free_device_circuit(ctx, c.dev_pershot);
            c.pershot_planned = false;
            c.plan_pershot = make_plan(c, tb, true);
            upload_circuit(ctx, c, c.plan_pershot, c.dev_pershot);
            c.pershot_planned = true;
            c.pershot_tb = tb;
        }
        const Plan& P = c.plan_pershot;
        const int n = (int)c.n, ob = n - P.tb;
        const size_t sbytes = (size_t)8 << n;
        // states in flight: up to 2 GiB of workspace, at most 65535 per launch
        const uint64_t batch = std::min<uint64_t>({n_shots, std::max<uint64_t>(1, ((size_t)2 << 30) / sbytes), 65535});
        PershotArgs A{};
        A.ops = c.dev_pershot.ops; A.micro = c.dev_pershot.micro; A.mats = c.dev_pershot.mats;
        A.chans = c.dev_pershot.chans; A.stages = c.dev_pershot.stages; A.hi = c.dev_pershot.hi;
        A.n = n; A.tb = P.tb; A.lb = P.lb; A.seed = seed; A.n_sites = c.site_op.size();
        A.states = (float2*)ctx->ws(ctx->pershot, batch * sbytes);
        A.part = (double*)ctx->ws(ctx->part, 2 * (batch << ob) * kMaxKraus * sizeof(double));
        SampleArgs R{};
        R.n = n; R.states = A.states; R.status = nullptr; R.seed = seed;
        const bool cluster = n <= sample_cluster_max_qubits();
        if (!cluster) R.scratch = (unsigned long long*)ctx->ws(ctx->scratch, sample_global_scratch_doubles(n) * 8);
        if (cluster) {   // the readout work items of every batch: allocated before the first launch
            ctx->ws(ctx->items, (size_t)batch * sizeof(SampleItem));
            ctx->reserve_staging((size_t)batch * sizeof(SampleItem), (size_t)((n_shots + batch - 1) / batch));
        }
        std::vector<SampleItem> items;
        for (uint64_t b0 = 0; b0 < n_shots; b0 += batch) {
            const uint32_t cnt = (uint32_t)std::min<uint64_t>(batch, n_shots - b0);
            A.first_shot = first_shot + b0;
            A.kraus = d_kraus ? d_kraus + b0 * A.n_sites : nullptr;
            // algorithmic bytes: each stage reads and writes every state once, the first one only
            // writes (it starts from |0...0>)
            ctx->timed(PTSBE_TIMER_PERSHOT, (double)sbytes * cnt * (2.0 * (double)P.stages.size() - 1.0), [&] {
                for (size_t j = 0; j < P.stages.size(); ++j) launch_pershot_stage(A, (int)j, cnt, ctx->stream);
            });
            // read every state out once with its own uniform (the sampler with the per-shot domain)
            R.bits = d_bits + b0;
            if (cluster) {
                items.clear();
                for (uint32_t i = 0; i < cnt; ++i) {
                    const uint64_t jj = first_shot + b0 + i;
                    items.push_back({i, 0u, jj, jj + 1, (uint64_t)i, kDomPershotRead, 0});   // bits[b0 + i]
                }
                SampleItem* d_items = (SampleItem*)ctx->ws(ctx->items, items.size() * sizeof(SampleItem));
                ctx->h2d(d_items, items.data(), items.size() * sizeof(SampleItem));
                ctx->timed(PTSBE_TIMER_SAMPLE, (double)sbytes * cnt + 4.0 * cnt,
                           [&] { launch_sample_cluster(R, d_items, cnt, ctx->stream); });
            } else {
                for (uint32_t i = 0; i < cnt; ++i) {
                    const uint64_t jj = first_shot + b0 + i;
                    ctx->timed(PTSBE_TIMER_SAMPLE, 5.0 * sbytes,
                               [&] { launch_sample_global(R, i, 0u, jj, jj + 1, (uint64_t)i, ctx->stream, kDomPershotRead); });
                }
            }
        }
    });
}

int ptsbe_batch_plan(ptsbe_ctx* ctx, const ptsbe_job* jobs, uint32_t n_jobs, uint32_t* batch_id) {
    const NvtxRange nvtx("ptsbe_batch_plan");
    return guarded(ctx, [&] {
        ctx->need_device();
        if (!batch_id) fail(PTSBE_ERR_INVALID, "batch_id is NULL");
        if (n_jobs && !jobs) fail(PTSBE_ERR_INVALID, "jobs is NULL");
        ctx->use_device();
        struct JobHost {
            KSet* s;
            Circuit* c;
            int n, J;
            std::vector<dense::Override> ovr;
            std::vector<float2> pool;
            std::vector<uint32_t> ovb, ove;
            std::vector<double> wmix, qa;
        };
        std::vector<JobHost> H(n_jobs);
        int maxJ = 0;
        for (uint32_t j = 0; j < n_jobs; ++j) {
            const ptsbe_job& jb = jobs[j];
            KSet& s = ctx->set(jb.set_id);
            Circuit& c = ctx->circuit(s.circuit);
            if ((uint64_t)jb.first + jb.count > s.count()) fail(PTSBE_ERR_INVALID, "job " + std::to_string(j) + ": set range out of bounds");
            if ((int)c.n < dense::kT) fail(PTSBE_ERR_UNSUPPORTED, "job " + std::to_string(j) + ": batches need n >= 12");
            if (jb.count && !jb.d_states) fail(PTSBE_ERR_INVALID, "job " + std::to_string(j) + ": d_states is NULL");
            if ((uintptr_t)jb.d_states % 16) fail(PTSBE_ERR_INVALID, "job " + std::to_string(j) + ": d_states must be 16-byte aligned");
            const uint64_t total = s.shot_off[jb.first + jb.count] - s.shot_off[jb.first];
            if (jb.d_bits && jb.d_bits_capacity < total)
                fail(PTSBE_ERR_BUFFER_TOO_SMALL, "job " + std::to_string(j) + ": d_bits holds " + std::to_string(jb.d_bits_capacity) +
                                                     " shots, the range needs " + std::to_string(total));
            if (!c.dense.built) make_dense_plan(c, c.dense);
            JobHost& h = H[j];
            h.s = &s; h.c = &c; h.n = (int)c.n; h.J = (int)c.dense.passes.size();
            maxJ = std::max(maxJ, h.J);
            const double q0mix = mix_q0(c);
            h.ovb.resize(jb.count); h.ove.resize(jb.count); h.wmix.resize(jb.count); h.qa.resize(jb.count);
            for (uint32_t a = 0; a < jb.count; ++a) {
                auto r = dense_overrides(c, c.dense, s, jb.first + a, h.ovr, h.pool);
                h.ovb[a] = r.first; h.ove[a] = r.second;
                h.wmix[a] = mix_weight(c, s, jb.first + a, q0mix);
                h.qa[a] = s.q[jb.first + a];
            }
        }
        // tasks, level by level: dense passes 0 .. J-1, finalisation J, scaling J + 1
        std::vector<QTask> tasks;
        std::vector<std::vector<uint32_t>> last(n_jobs);
        for (uint32_t j = 0; j < n_jobs; ++j) last[j].assign(jobs[j].count, 0xFFFFFFFFu);
        uint64_t item = 0;
        for (int lvl = 0; lvl < maxJ + 2; ++lvl)
            for (uint32_t j = 0; j < n_jobs; ++j) {
                const int J = H[j].J, ob = H[j].n - dense::kT;
                if (lvl > J + 1) continue;
                for (uint32_t a = 0; a < jobs[j].count; ++a) {
                    QTask t{};
                    t.item0 = item; t.job = j; t.set = a; t.level = (uint32_t)lvl;
                    t.items = lvl == J ? 1u : (1u << ob);
                    t.pred = last[j][a];
                    t.pred_items = t.pred == 0xFFFFFFFFu ? 0u : tasks[t.pred].items;
                    last[j][a] = (uint32_t)tasks.size();
                    tasks.push_back(t);
                    item += t.items;
                }
            }
        if (tasks.size() >= 0xFFFFFFF0u) fail(PTSBE_ERR_UNSUPPORTED, "too many tasks in one batch");
        // device workspace: [next][err][done per task] then per job tile norms, scales, status; sampler scratch
        auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
        size_t off = 0;
        const size_t o_next = off; off += 8;
        const size_t o_err = off; off += 8;
        const size_t o_done = off; off += 4 * tasks.size();
        const size_t counter_bytes = off;
        off = al(off);
        std::vector<size_t> o_part(n_jobs), o_scale(n_jobs), o_stat(n_jobs, SIZE_MAX);
        int max_global_n = 0;
        for (uint32_t j = 0; j < n_jobs; ++j) {
            const int ob = H[j].n - dense::kT;
            o_part[j] = off; off = al(off + ((size_t)jobs[j].count << ob) * sizeof(double));
            o_scale[j] = off; off = al(off + (size_t)jobs[j].count * sizeof(float));
            if (!jobs[j].d_status) { o_stat[j] = off; off = al(off + jobs[j].count); }
            if (jobs[j].d_bits && H[j].n > sample_cluster_max_qubits()) max_global_n = std::max(max_global_n, H[j].n);
        }
        size_t o_scr = SIZE_MAX;
        if (max_global_n) { o_scr = off; off = al(off + sample_global_scratch_doubles(max_global_n) * 8); }
        auto B = std::make_unique<Batch>();
        unsigned char* dws = (unsigned char*)ctx->dalloc(off);
        B->dws = dws;
        B->counter_bytes = counter_bytes;
        // tables: the plans of every job, the sets' overrides and weights, jobs, tasks, sampler items
        std::vector<unsigned char> buf;
        Blob b(buf);
        struct Offs { size_t p, g, bl, h, o, m, ov, pl, ob, oe, w, q; };
        std::vector<Offs> O(n_jobs);
        for (uint32_t j = 0; j < n_jobs; ++j) {
            const DensePlan& P = H[j].c->dense;
            O[j] = {b.add(P.passes), b.add(P.groups), b.add(P.blocks), b.add(P.hi), b.add(P.omap), b.add(P.mats),
                    b.add(H[j].ovr), b.add(H[j].pool), b.add(H[j].ovb), b.add(H[j].ove), b.add(H[j].wmix), b.add(H[j].qa)};
        }
        std::vector<QJob> qj(n_jobs);
        const size_t o_jobs = b.add(qj), o_tasks = b.add(tasks);
        std::vector<SampleItem> items;
        std::vector<PlannedSample> samples;
        for (uint32_t j = 0; j < n_jobs; ++j) {
            if (!jobs[j].d_bits) continue;
            const uint8_t* st = jobs[j].d_status ? jobs[j].d_status : dws + o_stat[j];
            const size_t before = samples.size();
            plan_samples(ctx, *H[j].s, *H[j].c, jobs[j].first, jobs[j].count, (const float2*)jobs[j].d_states, st,
                         jobs[j].seed, jobs[j].d_bits, items, samples);
            for (size_t i = before; i < samples.size(); ++i)
                if (o_scr != SIZE_MAX) samples[i].A.scratch = (unsigned long long*)(dws + o_scr);
        }
        const size_t o_items = b.add(items);
        unsigned char* dt = (unsigned char*)ctx->dalloc(buf.size());
        B->dtab = dt;
        for (uint32_t j = 0; j < n_jobs; ++j) {
            QJob& q = qj[j];
            q.passes = (const dense::Pass*)(dt + O[j].p); q.groups = (const dense::Group*)(dt + O[j].g);
            q.blocks = (const dense::Block*)(dt + O[j].bl); q.hi = (const uint32_t*)(dt + O[j].h);
            q.omap = (const uint16_t*)(dt + O[j].o); q.mats = (const float2*)(dt + O[j].m);
            q.ovr = (const dense::Override*)(dt + O[j].ov); q.opool = (const float2*)(dt + O[j].pl);
            q.ov_begin = (const uint32_t*)(dt + O[j].ob); q.ov_end = (const uint32_t*)(dt + O[j].oe);
            q.wmix = (const double*)(dt + O[j].w); q.qalpha = (const double*)(dt + O[j].q);
            q.states = (float2*)jobs[j].d_states;
            q.part = (double*)(dws + o_part[j]);
            q.weights = jobs[j].d_weights;
            q.status = jobs[j].d_status ? jobs[j].d_status : dws + o_stat[j];
            q.scale = (float*)(dws + o_scale[j]);
            q.n = (uint32_t)H[j].n; q.J = (uint32_t)H[j].J; q.count = jobs[j].count;
        }
        std::memcpy(buf.data() + o_jobs, qj.data(), qj.size() * sizeof(QJob));
        ctx->h2d(dt, buf.data(), buf.size());
        for (PlannedSample& p : samples) p.items = (const SampleItem*)(dt + o_items) + p.item_off;
        B->qa.jobs = (const QJob*)(dt + o_jobs);
        B->qa.tasks = (const QTask*)(dt + o_tasks);
        B->qa.n_tasks = (uint32_t)tasks.size();
        B->qa.n_items = item;
        B->qa.next = (unsigned long long*)(dws + o_next);
        B->qa.err = (uint32_t*)(dws + o_err);
        B->qa.done = (uint32_t*)(dws + o_done);
        B->d_err = B->qa.err;
        B->samples = std::move(samples);
        B->kernels_per_run = item ? 1 : 0;
        for (const PlannedSample& p : B->samples) B->kernels_per_run += p.kind == 2 ? 4 : 1;
        PTSBE_CUDA(cudaMemsetAsync(B->d_err, 0, 4, ctx->stream));
        dense_queue_grid(ctx->n_sm);      // kernel attributes set now, not during a capture
        configure_samplers();
        const uint32_t id = ctx->next_batch++;
        ctx->batches[id] = std::move(B);
        *batch_id = id;
    });
}

int ptsbe_batch_run(ptsbe_ctx* ctx, uint32_t batch_id, uint32_t flags) {
    const NvtxRange nvtx("ptsbe_batch_run");
    return guarded(ctx, [&] {
        ctx->need_device();
        auto it = ctx->batches.find(batch_id);
        if (it == ctx->batches.end()) fail(PTSBE_ERR_INVALID, "unknown batch id " + std::to_string(batch_id));
        if (flags & ~(uint32_t)PTSBE_BATCH_GRAPH) fail(PTSBE_ERR_INVALID, "unknown flags");
        Batch& B = *it->second;
        ctx->use_device();
        if (!(flags & PTSBE_BATCH_GRAPH)) {
            batch_enqueue(ctx, B);
            return;
        }
        if (!B.graph) {
            if (!ctx->stream) fail(PTSBE_ERR_UNSUPPORTED, "graph capture needs a stream other than the legacy default stream");
            const uint64_t l0 = launches_so_far();
            PTSBE_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            try {
                batch_enqueue(ctx, B);
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(ctx->stream, &g);
                if (g) cudaGraphDestroy(g);
                (void)cudaGetLastError();
                throw;
            }
            cudaGraph_t g = nullptr;
            PTSBE_CUDA(cudaStreamEndCapture(ctx->stream, &g));
            const cudaError_t e = cudaGraphInstantiate(&B.graph, g, 0);
            cudaGraphDestroy(g);
            PTSBE_CUDA(e);
            count_launch((uint64_t)0 - (launches_so_far() - l0));   // nothing ran yet: the launches count at replay
        }
        PTSBE_CUDA(cudaGraphLaunch(B.graph, ctx->stream));
        count_launch(B.kernels_per_run);
    });
}

int ptsbe_batch_info(ptsbe_ctx* ctx, uint32_t batch_id, uint64_t* tasks, uint64_t* items, uint32_t* grid,
                     uint64_t* kernels_per_run) {
    return guarded(ctx, [&] {
        auto it = ctx->batches.find(batch_id);
        if (it == ctx->batches.end()) fail(PTSBE_ERR_INVALID, "unknown batch id " + std::to_string(batch_id));
        const Batch& B = *it->second;
        if (tasks) *tasks = B.qa.n_tasks;
        if (items) *items = B.qa.n_items;
        if (grid) *grid = (uint32_t)std::min<uint64_t>(B.qa.n_items, (uint64_t)dense_queue_grid(ctx->n_sm));
        if (kernels_per_run) *kernels_per_run = B.kernels_per_run;
    });
}

int ptsbe_batch_release(ptsbe_ctx* ctx, uint32_t batch_id) {
    return guarded(ctx, [&] {
        auto it = ctx->batches.find(batch_id);
        if (it == ctx->batches.end()) fail(PTSBE_ERR_INVALID, "unknown batch id " + std::to_string(batch_id));
        Batch& B = *it->second;
        if (ctx->has_device()) {
            ctx->use_device();
            ctx->dfree(B.dtab);
            ctx->dfree(B.dws);
            if (B.graph) PTSBE_CUDA(cudaGraphExecDestroy(B.graph));
        }
        ctx->batches.erase(it);
    });
}

}  // extern "C"
