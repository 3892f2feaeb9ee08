/*
 * ptsbe.h -- C ABI of libptsbe: Pre-Trajectory Sampling with Batched Execution (PTSBE) on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Patti, Nguyen, Lietz, McCaskey, Khailany, "Augmenting Simulated Noisy Quantum Data
 * Collection by Orders of Magnitude Using Pre-Trajectory Sampling with Batched Execution"
 * (SC'25). A noisy circuit is registered (Fig. 1), a PTS algorithm picks Kraus-operator sets
 * alpha and their shot counts m_alpha up front (Sec. 3.1, Algorithm 2), each unique noisy state
 * is prepared once and all m_alpha shots are drawn from it at once (Sec. 3, batched execution).
 * The traditional per-operator trajectory loop (Algorithm 1) is provided as a comparison path.
 *
 * Conventions for every call:
 *   - Every function returns a ptsbe_status; nothing throws or aborts across the ABI. On error
 *     the outputs are unspecified, the context stays usable and ptsbe_last_error() describes
 *     the failure.
 *   - Host buffers are owned by the caller. Device buffers passed in (states, weights, shot
 *     bitstrings) are owned by the caller (e.g. PyTorch tensors); the library never frees them.
 *     The library owns its own device tables and workspace and frees them in ptsbe_destroy.
 *   - Device work is enqueued on the context's CUDA stream and is asynchronous unless stated.
 *   - Qubit q is bit q of a basis-state index. States are complex64, interleaved (re, im), one
 *     state of 2^n amplitudes after another.
 *   - Noise sites are the NOISE operations numbered 0..S-1 in circuit order. A Kraus set alpha
 *     is a list of (site, k) with k != 0, sites strictly increasing; a site not listed uses
 *     Kraus operator 0 ("no error").
 *   - Counter-based randomness is Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed
 *     (key = {seed_lo, seed_hi}); a 53-bit uniform is ((x0 << 21) | (x1 >> 11)) * 2^-53 of the
 *     first two output words. Every draw is a pure function of (seed, counter), so any slice of a
 *     job can be recomputed bit-identically.
 */
#ifndef PTSBE_H
#define PTSBE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PTSBE_API __attribute__((visibility("default")))
#else
#define PTSBE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ptsbe_ctx ptsbe_ctx;

typedef enum {
    PTSBE_OK = 0,
    PTSBE_ERR_INVALID = 1,          /* malformed argument (bad id, qubit >= n, unsorted set ...) */
    PTSBE_ERR_NOT_CPTP = 2,         /* a channel violates sum_k K_k^dag K_k = I (Sec. 2.2)      */
    PTSBE_ERR_OOM = 3,              /* host or device allocation failed (before any kernel of the
                                       call was enqueued: no output was written)                  */
    PTSBE_ERR_CUDA = 4,             /* a CUDA runtime call failed                                */
    PTSBE_ERR_TIMEOUT = 5,          /* a bounded device-side wait gave up                        */
    PTSBE_ERR_BUFFER_TOO_SMALL = 6, /* a caller buffer is smaller than the result                */
    PTSBE_ERR_UNSUPPORTED = 7,      /* well-formed request outside what the library handles      */
    PTSBE_ERR_NO_DEVICE = 8         /* a device entry point was called on a host-only context    */
} ptsbe_status;

/* ---------------------------------------------------------------------------------------- */
/* Context                                                                                   */
/* ---------------------------------------------------------------------------------------- */

/* Creates a context on CUDA device `device` that enqueues work on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream). device = -1 creates a host-only context: registration, PTS
 * and set export work, device entry points return PTSBE_ERR_NO_DEVICE. *out receives the handle. */
PTSBE_API int ptsbe_create(ptsbe_ctx** out, int device, void* cuda_stream);

/* Waits for the context's stream, frees every library-owned host and device resource. */
PTSBE_API int ptsbe_destroy(ptsbe_ctx* ctx);

/* Replaces the stream later calls enqueue on. */
PTSBE_API int ptsbe_set_stream(ptsbe_ctx* ctx, void* cuda_stream);

/* Message of the last failed call on this context (owned by the library, valid until the next
 * call on the context). Never NULL. */
PTSBE_API const char* ptsbe_last_error(const ptsbe_ctx* ctx);

/* Blocks until all work enqueued by the context has finished; returns PTSBE_ERR_CUDA (with the
 * CUDA error text) if an asynchronous kernel failed, PTSBE_ERR_TIMEOUT if a bounded device wait
 * gave up, PTSBE_ERR_UNSUPPORTED if a fused sampling launch flagged the context (see
 * ptsbe_evolve_sample; the flag is cleared). */
PTSBE_API int ptsbe_synchronize(ptsbe_ctx* ctx);

/* ---------------------------------------------------------------------------------------- */
/* Circuit registration (Fig. 1: "an arbitrary noisy circuit is registered"; Sec. 2.2)        */
/* ---------------------------------------------------------------------------------------- */

enum { PTSBE_OP_GATE = 0, PTSBE_OP_NOISE = 1 };

/* Gate codes. Matrices: OpenQASM U3(theta, phi, lambda) = [[cos t/2, -e^{i l} sin t/2],
 * [e^{i p} sin t/2, e^{i(p+l)} cos t/2]]; RX/RY/RZ(theta) = exp(-i theta P/2). Two-qubit gates act
 * on the local index 2*bit(targets[0]) + bit(targets[1]); CX has control targets[0]. U1/U2 take
 * their matrix from the custom-gate table, row params[0]. */
enum {
    PTSBE_G_I = 0, PTSBE_G_X, PTSBE_G_Y, PTSBE_G_Z, PTSBE_G_H, PTSBE_G_S, PTSBE_G_SDG, PTSBE_G_T,
    PTSBE_G_TDG, PTSBE_G_RX, PTSBE_G_RY, PTSBE_G_RZ, PTSBE_G_U3, PTSBE_G_CX, PTSBE_G_CZ,
    PTSBE_G_SWAP, PTSBE_G_U1, PTSBE_G_U2
};

/* Channel kinds (Sec. 2.2: channels given as CPTP Kraus sets). With strength p (or gamma):
 *   DEPOL1    {sqrt(1-p) I, sqrt(p/3) X, Y, Z}
 *   DEPOL2    {sqrt(1-p) I(x)I, sqrt(p/15) P_a (x) P_b}, k = 4a + b, P_a on targets[0]
 *   AMPDAMP   {[[1,0],[0,sqrt(1-g)]], [[0,sqrt(g)],[0,0]]}
 *   BITFLIP   {sqrt(1-p) I, sqrt(p) X};  PHASEFLIP {sqrt(1-p) I, sqrt(p) Z}
 *   CUSTOM    n_kraus <= 16 caller matrices of size 2^arity.
 * Kraus operator 0 is "no error". Nominal probabilities q_k = tr(K_k^dag K_k)/d (closed forms
 * 1-p, p/3 ... for the named kinds). A channel with K_k^dag K_k = q_k I for every k is a unitary
 * mixture (Sec. 2.2 item 2): it is applied as U_k = K_k/sqrt(q_k) and needs no norm. */
enum {
    PTSBE_CH_DEPOL1 = 0, PTSBE_CH_DEPOL2, PTSBE_CH_AMPDAMP, PTSBE_CH_BITFLIP, PTSBE_CH_PHASEFLIP,
    PTSBE_CH_CUSTOM
};

typedef struct {
    uint32_t kind;        /* PTSBE_OP_GATE or PTSBE_OP_NOISE                                 */
    uint32_t id;          /* gate code, or channel index into the channel array              */
    uint32_t n_targets;   /* 1 or 2; must equal the gate's or channel's arity                */
    uint32_t targets[2];  /* distinct qubits < n_qubits                                      */
    double params[3];     /* angles (U3: theta, phi, lambda; RX/RY/RZ: theta)                */
} ptsbe_op;

typedef struct {
    uint32_t kind;        /* PTSBE_CH_*                                                      */
    uint32_t arity;       /* 1 or 2                                                          */
    uint32_t n_kraus;     /* 4 / 16 / 2 / 2 / 2 for the named kinds; <= 16 for CUSTOM         */
    double param;         /* p or gamma in [0, 1] for the named kinds                        */
    const double* kraus;  /* CUSTOM only: n_kraus row-major (2^arity x 2^arity) complex128
                             matrices as (re, im) pairs; copied during the call                */
} ptsbe_channel;

/* Validates and copies a noisy circuit; builds its device tables (gate matrices and Kraus
 * operators rounded once to complex64, unitary-mixture flags, the tiling plan). n_qubits in
 * [1, 32]. custom_gates: n_custom rows of 4x4 complex128 (re, im) (a 1-qubit custom gate uses the
 * top-left 2x2). *circuit_id receives the handle.
 * Errors: PTSBE_ERR_INVALID (bad op or channel), PTSBE_ERR_NOT_CPTP (|sum K^dag K - I| > 1e-10). */
PTSBE_API int ptsbe_register_circuit(ptsbe_ctx* ctx, uint32_t n_qubits, const ptsbe_op* ops, uint64_t n_ops,
                           const ptsbe_channel* channels, uint32_t n_channels,
                           const double* custom_gates, uint32_t n_custom, uint32_t* circuit_id);

/* Number of noise sites S and gates of a registered circuit. */
PTSBE_API int ptsbe_circuit_info(ptsbe_ctx* ctx, uint32_t circuit_id, uint32_t* n_qubits, uint64_t* n_sites,
                       uint64_t* n_gates);

PTSBE_API int ptsbe_release_circuit(ptsbe_ctx* ctx, uint32_t circuit_id);

/* ---------------------------------------------------------------------------------------- */
/* Pre-trajectory sampling (Sec. 3.1, Algorithm 2). Host-synchronous.                        */
/* ---------------------------------------------------------------------------------------- */

typedef enum {
    /* Algorithm 2 with one categorical draw per noise site (reading of "sampled ... in much the
     * same way as they would be at state preparation runtime"): sample i at site s draws
     * u = U53(Philox(seed; s, i_lo, i_hi, 1)) and takes the smallest k with u < q_0 + ... + q_k
     * (FP64, listed order; the last k if rounding leaves u above the sum). */
    PTSBE_PTS_PROPORTIONAL = 0,
    /* The k most likely sets (Sec. 3.1, "most common errors ... above a given cutoff"): key of a
     * set = product of its ratios q_{s,k}/q_{s,0} multiplied in descending order; order = key
     * descending, then canonical order. Needs q_{s,0} > q_{s,k} at every site. */
    PTSBE_PTS_TOPK = 1,
    /* Every set with p_min <= q_alpha <= p_max (probability band; cutoff = band with p_max = 1). */
    PTSBE_PTS_BAND = 2,
    /* Caller-given sets (targeted errors; Sec. 3.1 "selection criteria"). */
    PTSBE_PTS_TARGETED = 3,
    /* Algorithm 2 as printed: each (site, k != 0) draws r = U53(Philox(seed; s, i_lo, i_hi,
     * 4 | k << 8)) and is appended when r <= q_{s,k} and its site is still free (compatible). */
    PTSBE_PTS_LITERAL = 4,
    /* Targeted error sets by rule (Sec. 3.1 "selection criteria"): every set of 1 .. max_errors
     * errors at distinct sites whose every error (s, k) passes the filters -- site in
     * [site_lo, site_hi), all qubits of the site in qubit_mask, Kraus index k in kraus_mask, the
     * gate the site follows (the last gate before it that shares one of its qubits) in gate_mask
     * -- and whose weight passes weight_parity; plus the empty set when include_empty. A zero
     * mask or site_hi = 0 accepts everything. Shots by BY_PROB (default), UNIFORM or BY_COUNT. */
    PTSBE_PTS_PREDICATE = 5
} ptsbe_pts_mode;

typedef enum {
    PTSBE_SHOTS_BY_COUNT = 0, /* largest-remainder apportionment of total_shots by multiplicity  */
    PTSBE_SHOTS_UNIFORM = 1,  /* shots_per_set for every set (Algorithm 2's nshots)             */
    PTSBE_SHOTS_BY_PROB = 2,  /* largest-remainder apportionment of total_shots by q_alpha      */
    PTSBE_SHOTS_GIVEN = 3     /* TARGETED only: t_shots[i] per given set                        */
} ptsbe_shot_alloc;

typedef struct {
    uint32_t mode;              /* ptsbe_pts_mode                                             */
    uint32_t shot_alloc;        /* ptsbe_shot_alloc                                           */
    uint64_t nsamples;          /* PROPORTIONAL, LITERAL                                      */
    uint64_t k;                 /* TOPK                                                       */
    double p_min, p_max;        /* BAND                                                       */
    uint64_t total_shots;       /* BY_COUNT, BY_PROB                                          */
    uint64_t shots_per_set;     /* UNIFORM                                                    */
    uint32_t t_count;           /* TARGETED: number of sets                                   */
    const uint32_t* t_offsets;  /* TARGETED: [t_count + 1] CSR offsets into t_sites/t_kidx    */
    const uint32_t* t_sites;    /* TARGETED: strictly increasing per set                      */
    const uint8_t* t_kidx;      /* TARGETED: 0 < k < n_kraus                                  */
    const uint64_t* t_shots;    /* TARGETED with SHOTS_GIVEN: [t_count]                       */
    uint32_t max_errors;        /* PREDICATE: 1 .. 8 errors per set                           */
    uint32_t include_empty;     /* PREDICATE: 1 adds the error-free set                       */
    uint64_t qubit_mask;        /* PREDICATE: bit q allows sites on qubit q (0: all)          */
    uint32_t kraus_mask;        /* PREDICATE: bit k allows Kraus index k >= 1 (0: all)        */
    uint32_t gate_mask;         /* PREDICATE: bit g allows sites after gate code g (0: all)   */
    uint32_t site_lo, site_hi;  /* PREDICATE: site range (site_hi = 0: all sites)             */
    uint32_t weight_parity;     /* PREDICATE: 0 any, 1 odd, 2 even number of errors           */
    uint64_t max_sets;          /* PREDICATE: PTSBE_ERR_UNSUPPORTED above this (0: 10^7)      */
} ptsbe_pts_params;

/* Runs a PTS algorithm and stores the resulting Kraus sets in the context. Sets are returned in
 * canonical order (lexicographic over the (site, k) list, a prefix before its extensions, so the
 * empty set comes first) with duplicates merged (uniqueKraus); mult = how many samples produced
 * the set; q_alpha = (prod_s q_{s,0}) * key. Largest-remainder apportionment gives the extra
 * shots to the largest remainders, ties to the lower index. The shot layout of the set is the
 * exclusive prefix of m_alpha ("shot offsets"): shot j of set a is global shot offset[a] + j.
 * Outputs (any may be NULL): *set_id, *count (unique sets), *n_entries (total (site, k) entries),
 * *total_shots. Errors: PTSBE_ERR_INVALID, PTSBE_ERR_UNSUPPORTED (TOPK/BAND with a site whose
 * q_0 is not the strict maximum), PTSBE_ERR_OOM. */
PTSBE_API int ptsbe_sample_kraus(ptsbe_ctx* ctx, uint32_t circuit_id, const ptsbe_pts_params* params, uint64_t seed,
                       uint32_t* set_id, uint32_t* count, uint64_t* n_entries, uint64_t* total_shots);

/* Caller buffers for a set export; any pointer may be NULL. Sizes: offsets/shot_offsets
 * [count+1], sites/kidx [n_entries], mult/q/shots [count]. These are the error-provenance labels
 * of Sec. 3 ("lightweight metadata"): shot g belongs to the set a with
 * shot_offsets[a] <= g < shot_offsets[a+1]. */
typedef struct {
    uint32_t* offsets;
    uint32_t* sites;
    uint8_t* kidx;
    uint64_t* mult;
    double* q;
    uint64_t* shots;
    uint64_t* shot_offsets;
} ptsbe_set_view;

PTSBE_API int ptsbe_set_export(ptsbe_ctx* ctx, uint32_t set_id, const ptsbe_set_view* out);
PTSBE_API int ptsbe_release_set(ptsbe_ctx* ctx, uint32_t set_id);

/* ---------------------------------------------------------------------------------------- */
/* Batched execution (Sec. 3)                                                                */
/* ---------------------------------------------------------------------------------------- */

enum {
    /* Prefix reuse: a set whose (site, k) list extends another set of the same call skips the
     * tile stages before the one holding its first extra site, starting there from the other
     * set's input of that stage instead of from |0...0>. Stages alternate between d_states and a
     * library workspace of the same size. */
    PTSBE_EVOLVE_PREFIX_REUSE = 1u,
    /* Plan only (dense passes, n >= 12: evolve kernel 4, or d_states NULL in ptsbe_evolve_sample): build the
     * call's schedule (prefix reuse, branches) and set the counters of ptsbe_reuse_stats, but
     * enqueue no device work and write no output; output pointers may be NULL. For sizing a job
     * before running it. With another evolve kernel: PTSBE_ERR_UNSUPPORTED. */
    PTSBE_EVOLVE_PLAN_ONLY = 2u
};

/* Prepares the states of sets [first, first + count) of set_id (each once, Sec. 3):
 *   psi_alpha = normalise( prod_ops (K_{s,k_s} or U_{s,k_s}) G ... |0...0> ),
 * the Kraus operators of alpha inserted at their sites; unitary-mixture sites apply U_k, other
 * sites apply K_k, and the state is renormalised at the end (Sec. 2.2 renormalisation; deferred
 * renormalisation gives the same normalised state). Outputs (device, caller-owned):
 *   d_states  complex64 [count][2^n], 16-byte aligned; written completely
 *   d_weights float64 [count]: w_alpha = prod_{mixture sites} q_{s,k_s} * ||unnormalised psi||^2,
 *             the Born probability of the Kraus branch (may be NULL)
 *   d_status  uint8 [count]: 0 ok, 1 null (w_alpha < 1e-6 q_alpha: a branch the state cannot take,
 *             e.g. damping a qubit with no |1> population; its state is zeroed) (may be NULL).
 * Asynchronous on the context stream. Errors: PTSBE_ERR_INVALID (range, null pointer, alignment),
 * PTSBE_ERR_OOM (workspace), PTSBE_ERR_CUDA (launch). */
PTSBE_API int ptsbe_evolve_batch(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count, void* d_states,
                       double* d_weights, uint8_t* d_status, uint32_t flags);

/* Draws all m_alpha shots of sets [first, first + count) from their prepared states (Sec. 3,
 * "sampling all m_alpha desired quantum bitstrings at once"). For state alpha with
 * P_i = |psi_i|^2 and C its inclusive prefix, T = C[2^n - 1]: shot j uses
 * u = U53(Philox(seed; j_lo, j_hi, alpha, 2)) (alpha = index of the set within set_id) and returns
 * the smallest i with u*T < C[i] (2^n - 1 if none). Arithmetic: P_i is the FP32 value
 * re^2 + im^2, held as floor(P_i 2^62) in 64-bit integers; C and T are exact integer sums of those
 * and u*T is floor(m T / 2^53) for u = m / 2^53, so the prefix carries no rounding (resolution
 * 2^-62 against 2^-53 for an FP64 running sum near 1). States must have T < 4 (normalised states
 * from ptsbe_evolve_batch have T = 1). Outputs:
 *   d_bits  uint32 [sum of m_alpha over the range], set-major: shot j of set first+a lands at
 *           shot_offsets[first+a] - shot_offsets[first] + j. Null states (d_status 1) yield
 *           0xFFFFFFFF. d_bits_capacity = number of uint32 slots available.
 * d_states as written by ptsbe_evolve_batch for the same range; d_status may be NULL.
 * Asynchronous. Errors: PTSBE_ERR_BUFFER_TOO_SMALL, PTSBE_ERR_INVALID, PTSBE_ERR_OOM. */
PTSBE_API int ptsbe_sample_shots(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count, const void* d_states,
                       const uint8_t* d_status, uint64_t seed, uint32_t* d_bits, uint64_t d_bits_capacity);

/* Batched execution in one call (Sec. 3: each unique state prepared once, then all m_alpha of its
 * shots drawn at once): the outputs of ptsbe_evolve_batch(ctx, set_id, first, count, d_states,
 * d_weights, d_status, flags) followed by ptsbe_sample_shots(ctx, set_id, first, count, d_states,
 * d_status, seed, d_bits, d_bits_capacity), bit for bit (states, weights, status and shots).
 * When the last tile stage prepares each state from its support in one CTA (a sparse final
 * stage), that CTA also draws the shots of states with at most PTSBE_OPT_LIGHT_SHOTS shots from
 * the support it holds on chip, so those states are never read back; the CDF of a state over its
 * support in increasing index order has the same prefix values as over all 2^n entries (the
 * others are exact zeros). Heavier states leave that CDF (at most 2^10 entries) in a library
 * workspace, and a sampler kernel spreads their shots over many CTAs, each holding the CDF in
 * shared memory. Without a sparse final stage the states go to the sampler kernels of
 * ptsbe_sample_shots. Arguments, layouts and
 * ownership as for the two calls. Asynchronous. Errors: those of the two calls; a kernel that
 * finds a support not of the form the plan guarantees flags the context, and the next
 * ptsbe_synchronize returns PTSBE_ERR_UNSUPPORTED (the affected shots hold 0xFFFFFFFF). */
/* d_states may be NULL when n >= 12: the states are then not returned and live only in library
 * buffers (for states too large to keep one per set, e.g. 8 GiB at 30 qubits). The sets of the
 * range are prepared with dense passes, one branch at a time: at each pass the sets are split by
 * their Kraus entries inside that pass; a group with entries there branches into a new buffer from
 * the state all of them share at that pass (prefix reuse) and is finished -- prepared, normalised,
 * sampled -- before the sets without entries there continue in place. Device memory: one 2^n
 * complex64 buffer per level of branch nesting plus one (Kraus sets with e entries nest at most
 * e + 1 deep), plus the sampler's workspace. Weights, status and shots are as above (the same
 * states up to rounding, bit-identical to evolve kernel 4 with d_states given). */
PTSBE_API int ptsbe_evolve_sample(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count, void* d_states,
                                  double* d_weights, uint8_t* d_status, uint32_t flags, uint64_t seed,
                                  uint32_t* d_bits, uint64_t d_bits_capacity);

/* Unique-shot statistic (Sec. 4: the fraction of distinct outcomes among a set's shots): for sets
 * [first, first + count) of set_id, d_unique[a] = number of distinct values among the shots of set
 * first + a in d_bits (laid out as ptsbe_sample_shots writes them; the null-branch sentinel is not
 * an outcome and is skipped). Device outputs, asynchronous. n_qubits <= 20 (else
 * PTSBE_ERR_UNSUPPORTED). Errors: PTSBE_ERR_INVALID (range, null pointers). */
PTSBE_API int ptsbe_unique_shots(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count,
                                 const uint32_t* d_bits, uint64_t* d_unique);

/* Same shots as ptsbe_sample_shots, bit for bit, for callers that cannot allocate device memory:
 * a program whose memory pool has already reserved the GPU, a fixed-footprint deployment that
 * plans every byte up front, or a latency-critical loop that must not hit the device-wide
 * synchronisation a cudaFree implies. (The paper has no counterpart; this is an interface choice
 * of the library.) The call's scratch -- the work-item list for n <= 17, the CDF workspace for
 * 18 <= n <= 21 -- lives in a fixed 40 MiB device array compiled into the library, which every
 * GPU that loads the library holds until the process exits; no cudaMalloc, cudaFree or other
 * allocating routine is called. Requests that need more (more than 2^20 = 1,048,576 work items --
 * a work item is a set, or a range of at least 65,536 of its shots above 14 qubits and of at
 * least 2^n (1,024 at the least) up to 14 -- or n > 21) return
 * PTSBE_ERR_UNSUPPORTED with the sizes in the message. The first call on a device looks up the
 * array's device address (a one-time driver query): make that first call before any stream
 * capture. For n <= 17 the work items go up through one of the context's pinned staging slots
 * (asynchronous) when that slot, allocated by earlier calls, already has room for them (up to
 * 2 MiB: 52,428 items); a larger list is copied from pageable host memory, and the call then
 * waits for the work already queued on the context stream before it returns. Every call shares the one
 * array and overwrites what the previous call left there (nothing is read before this call writes
 * it); calls whose work can overlap on the GPU -- on different streams or contexts of the same
 * device -- race on it and must be serialised by the caller. Arguments, layout and other errors
 * as for ptsbe_sample_shots. */
PTSBE_API int ptsbe_sample_shots_noalloc(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count,
                                         const void* d_states, const uint8_t* d_status, uint64_t seed,
                                         uint32_t* d_bits, uint64_t d_bits_capacity);

/* ---------------------------------------------------------------------------------------- */
/* Many circuits in one persistent launch (Sec. 3 batched execution over uneven circuits)        */
/* ---------------------------------------------------------------------------------------- */

/* One job of a batch: sets [first, first + count) of set_id, prepared in place in d_states
 * (complex64 [count][2^n], 16-byte aligned, n >= 12) with dense passes, normalised (d_weights
 * float64 [count] and d_status uint8 [count] as for ptsbe_evolve_batch; either may be NULL), and
 * sampled into d_bits as ptsbe_sample_shots would (NULL: no shots). All buffers caller-owned, on
 * the context's device, and valid while the batch lives. */
typedef struct {
    uint32_t set_id, first, count;
    void* d_states;
    double* d_weights;
    uint8_t* d_status;
    uint64_t seed;
    uint32_t* d_bits;
    uint64_t d_bits_capacity;
} ptsbe_job;

enum {
    /* ptsbe_batch_run: capture the run into a CUDA graph on the first such call (the context's
     * stream must not be the legacy default stream) and launch that graph on this and later calls. */
    PTSBE_BATCH_GRAPH = 1u
};

/* Plans a batch: every job's dense-pass plan, Kraus-set overrides, weights, the work queue's tasks
 * and the sampler launches, copied to the device now (the jobs' sets and circuits may be released
 * afterwards). The tasks are (set, level) of every job, level by level: each dense pass of a set
 * (one work item per 2^12-amplitude tile), then its normalisation and its scaling; a task waits for
 * the same set's previous level. Host-synchronous planning, one stream-ordered upload.
 * Errors: PTSBE_ERR_INVALID, PTSBE_ERR_UNSUPPORTED (n < 12), PTSBE_ERR_BUFFER_TOO_SMALL, PTSBE_ERR_OOM. */
PTSBE_API int ptsbe_batch_plan(ptsbe_ctx* ctx, const ptsbe_job* jobs, uint32_t n_jobs, uint32_t* batch_id);

/* Runs a planned batch on the context stream: one persistent cooperative launch prepares every
 * job's states (all CTAs resident; each takes the next tile from one global counter and waits,
 * bounded by PTSBE_OPT_QUEUE_SPIN_CYCLES, for the tiles it depends on), then the samplers draw the
 * shots. Enqueues device work only (memsets and kernels), so it can be replayed as a CUDA graph
 * (PTSBE_BATCH_GRAPH). Results: the outputs of ptsbe_evolve_batch (kernel 4) and
 * ptsbe_sample_shots for every job, bit for bit. A wait that ran out makes the next
 * ptsbe_synchronize return PTSBE_ERR_TIMEOUT (the outputs are then incomplete); the context and
 * the batch stay usable. Asynchronous. */
PTSBE_API int ptsbe_batch_run(ptsbe_ctx* ctx, uint32_t batch_id, uint32_t flags);

/* Size of a planned batch: queue tasks, work items, CTAs of the persistent launch, kernels per run
 * (any pointer may be NULL). Host-only. */
PTSBE_API int ptsbe_batch_info(ptsbe_ctx* ctx, uint32_t batch_id, uint64_t* tasks, uint64_t* items, uint32_t* grid,
                               uint64_t* kernels_per_run);

/* Frees a batch's device tables, workspace and graph (stream-ordered after its runs). */
PTSBE_API int ptsbe_batch_release(ptsbe_ctx* ctx, uint32_t batch_id);

/* ---------------------------------------------------------------------------------------- */
/* Adjoint gradients of the fixed-set estimator (Sec. 3 with the Kraus sets held fixed)        */
/* ---------------------------------------------------------------------------------------- */

/* Diagonal observable O = sum_t coeffs[t] prod_{q in masks[t]} Z_q  +  sum_x diag[x] |x><x|.
 * masks/coeffs: host arrays of n_terms entries (bit q of a mask = qubit q); diag: optional device
 * float64 [2^n] indexed by the logical basis index (e.g. the indicator of one outcome, for the
 * gradient of an outcome probability). masks and coeffs are copied during the call; d_diag is
 * read by the call's kernels and must stay valid until they complete on the stream. */
typedef struct {
    uint32_t n_terms;
    const uint64_t* masks;
    const double* coeffs;
    const double* d_diag;
} ptsbe_observable;

/* Loss and gradients of the importance-weighted estimator over sets [first, first + count) of
 * set_id (Sec. 3: each set alpha prepared once; its nominal probability q_alpha and multiplicity
 * mult_alpha held fixed):
 *   L = (1 / N) sum_alpha mult_alpha <psi~_alpha| O |psi~_alpha> / q_alpha,  N = sum of mult_alpha,
 * psi~_alpha the unnormalised state with every Kraus operator applied as given (K_{s,k}, Sec. 2.2).
 * With the sets drawn by PTS this estimates Tr(O rho) and its gradient that of Tr(O rho); with
 * count = 1 it is the single trajectory's observable. circuit_id gives the gate angles and channel
 * strengths to differentiate at; it must have the structure of the set's circuit (same qubits,
 * operations, targets, channel kinds and Kraus counts), its parameters may differ.
 * Outputs (device, caller-owned, each may be NULL):
 *   d_loss        float64 [1]
 *   d_per_set     float64 [count]: <psi~_alpha|O|psi~_alpha> / q_alpha
 *   d_grad_params float64 [n_ops][3]: dL / d ops[i].params[j] (RX/RY/RZ theta, U3 theta, phi,
 *                 lambda; 0 for every other operation and parameter)
 *   d_grad_noise  float64 [n_channels]: dL / d channels[c].param (the named kinds; 0 for CUSTOM)
 * checkpoint_every: 0 stores a set's state only before operators it cannot invert (a damping
 * jump) and where the plan's conditioning rule asks for it (un-computing through the blocks since
 * the last stored copy would multiply FP32 rounding by more than 2^6: the product of their
 * condition numbers, e.g. 1 / sqrt(1 - gamma) per damping site); c > 0 also every c fused blocks
 * (the un-computed state is replaced by the stored one there). n_qubits <= 16, at most 64 (site, k) entries per set.
 * Asynchronous on the context stream. Errors: PTSBE_ERR_INVALID (range, structure, null
 * observable, a set with q_alpha = 0), PTSBE_ERR_UNSUPPORTED (n > 16, longer sets),
 * PTSBE_ERR_OOM, PTSBE_ERR_CUDA. */
/* Shape of the backward plan of a circuit (built on first use): fused blocks of one and two
 * qubits, qubit-position swaps between cluster CTAs, blocks holding a differentiable parameter,
 * blocks before which the state is stored by the conditioning rule (see ptsbe_backward).
 * Any pointer may be NULL. Host-only work. Errors: PTSBE_ERR_INVALID, PTSBE_ERR_UNSUPPORTED (n > 16). */
PTSBE_API int ptsbe_backward_plan_info(ptsbe_ctx* ctx, uint32_t circuit_id, uint32_t* blocks_1q, uint32_t* blocks_2q,
                                       uint32_t* swaps, uint32_t* differentiable_blocks,
                                       uint32_t* conditioning_checkpoints);

PTSBE_API int ptsbe_backward(ptsbe_ctx* ctx, uint32_t circuit_id, uint32_t set_id, uint32_t first, uint32_t count,
                             const ptsbe_observable* obs, uint32_t checkpoint_every, double* d_loss,
                             double* d_per_set, double* d_grad_params, double* d_grad_noise);

/* ---------------------------------------------------------------------------------------- */
/* Traditional trajectories (Algorithm 1), one prepared state per shot, for comparison        */
/* ---------------------------------------------------------------------------------------- */

/* Simulates shots [first_shot, first_shot + n_shots) of the traditional trajectory loop: at
 * noise site s shot j draws u = U53(Philox(seed; s, j_lo, j_hi, 3)); a unitary mixture picks
 * k = index(u, {q}) and applies U_k; a general channel computes p_i = <psi|K_i^dag K_i|psi> (FP64
 * accumulation), picks k = index(u, {p}) and applies K_k / sqrt(p_k). The final state is read out
 * once with u = U53(Philox(seed; j_lo, j_hi, 0, 5)) by the inverse-CDF rule of
 * ptsbe_sample_shots. Outputs: d_bits uint32 [n_shots]; d_kraus uint8 [n_shots][S] chosen k per
 * site (may be NULL). Uses library workspace for the states in flight. Asynchronous. */
PTSBE_API int ptsbe_pershot_run(ptsbe_ctx* ctx, uint32_t circuit_id, uint64_t seed, uint64_t first_shot,
                      uint64_t n_shots, uint32_t* d_bits, uint8_t* d_kraus);

/* ---------------------------------------------------------------------------------------- */
/* Options                                                                                   */
/* ---------------------------------------------------------------------------------------- */

enum {
    /* Kernel for the tile passes of ptsbe_evolve_batch: 0 auto (= 3), 1 shared-memory sweeps (one
     * pass of the tile per operator), 2 register-blocked (operators applied to amplitudes held in
     * registers, the tile re-shuffled through shared memory between register groups), 3 deferred
     * frame (permutations and diagonals tracked as an index map and factor tables; only
     * operators that mix amplitudes pass over the tile), 4 dense passes (the state streams
     * through HBM once per pass over 12-qubit tiles; the operators of a pass are fused into 1- and
     * 2-qubit blocks applied to amplitudes held in registers; the planner changes the
     * qubit-to-bit layout between passes so each pass holds the qubits it needs; a state of
     * n < 12 qubits is prepared zero-padded to 12 in a library buffer, the added qubits untouched,
     * and its 2^n amplitudes copied to d_states). */
    PTSBE_OPT_EVOLVE_KERNEL = 0,
    /* States (15 <= n <= 20) with at most this many shots are sampled by one CTA each from chunk
     * prefixes (one chunk re-read per shot); heavier ones by a thread-block cluster holding the
     * whole CDF. In ptsbe_evolve_sample with a sparse final stage, states with at most this many
     * shots are sampled inside the evolve launch and heavier ones from their exported support
     * CDF. Every choice gives the same shots; only the speed differs. Default 65,536 (measured
     * for ptsbe_sample_shots; the autotuner times 512 .. 2^20 on the one-call path). */
    PTSBE_OPT_LIGHT_SHOTS = 1,
    /* Kraus sets whose frame programs one warp of the program prepass builds (one thread per set):
     * 4, 8 or 16 (0 = default, 8: measured). The builders branch on each set's entries, so fewer
     * sets per warp diverge less and leave more warps per scheduler. Same programs; speed only. */
    PTSBE_OPT_PROGRAM_SETS_PER_WARP = 2,
    /* Fault injection for tests (no GPU fault: the failure is made on the host): value k >= 0 makes
     * the k-th allocation (0-based: device tables, workspace, pinned staging) the context attempts
     * from now on fail as if memory ran out, so the call making it returns PTSBE_ERR_OOM; -1
     * (default) turns it off. Every entry point but ptsbe_autotune (a series of calls) allocates
     * before its first kernel launch, so a call that fails this way has written none of its
     * outputs, and the context stays usable. */
    PTSBE_OPT_FAIL_ALLOC = 3,
    /* Wait budget of the batch work queue (ptsbe_batch_run), in GPU clock cycles (clock64): a CTA
     * waiting for another task's tiles gives up after this long, records the task, and every CTA
     * leaves; the next ptsbe_synchronize returns PTSBE_ERR_TIMEOUT. Default 2e10 (~10 s). */
    PTSBE_OPT_QUEUE_SPIN_CYCLES = 4,
    /* Test hook of the work queue: the task with this index waits for one tile more than its
     * predecessor has, so its wait always runs out (no GPU fault: the wait is bounded and the
     * kernel returns); -1 (default) turns it off. */
    PTSBE_OPT_QUEUE_STALL_TASK = 5,
    /* Percentage p (0..100, default 0) of each state's bytes zeroed apart from the evolve launch,
     * when a call's plan is one stage ending in the small sparse final store (each state's nonzero
     * amplitudes held on chip, as for the syndrome workload): that part of the zero fill runs as
     * its own kernel on a second stream of the context, concurrently with the program prepass, and
     * the evolve launch zeroes the rest (rounded to whole 4 KB chunks). Same outputs; speed only.
     * The second stream starts after the work the call found on the context stream and the
     * context stream waits for it, so the call stays ordered on the context stream (and a capture
     * of that stream into a CUDA graph takes both). */
    PTSBE_OPT_SPLIT_FILL = 6,
    /* Tile bits (9..14; 0 = default) of the plan ptsbe_pershot_run uses: its stages end at every
     * general noise site whatever the tile, so the tile only sets how many CTAs share an SM and
     * how many tiles a state spans. Same shots; speed only. */
    PTSBE_OPT_PERSHOT_TILE_BITS = 7,
    /* 1 (default) or 0. With 1, a frame-kernel call whose plan is one stage (every state prepared
     * in one tile pass, as for the syndrome workload) puts its table uploads and its program
     * prepass on the context's second stream without waiting for the context stream: the
     * programs depend only on the circuit and the Kraus sets, so the latency-bound prepass of
     * this call runs while the context stream still executes earlier calls (their HBM-bound
     * evolve launches). The evolve launch waits for it on the context stream, so every output is
     * still written in the context stream's order, and the caller's buffers are touched only
     * there. The library keeps two copies of the node tables and programs and reuses one only
     * after the context stream has run the launches that read it. Off while the context stream
     * is being captured into a CUDA graph, and with a split zero fill. Same outputs; speed only. */
    PTSBE_OPT_PREPASS_AHEAD = 8
};

/* Sets a context option; PTSBE_ERR_INVALID for an unknown option or value. */
PTSBE_API int ptsbe_set_option(ptsbe_ctx* ctx, int option, int64_t value);

/* Result of ptsbe_autotune: the options it chose and the measured time of every candidate
 * (milliseconds per ptsbe_evolve_batch call for the kernels, per ptsbe_evolve_sample call for the
 * shot limits; mean of `reps` calls; 0 for a candidate that does not apply). */
typedef struct {
    int32_t evolve_kernel;            /* chosen PTSBE_OPT_EVOLVE_KERNEL (1 sweeps, 2 registers, 3 frame, 4 dense) */
    uint64_t light_shots;             /* chosen PTSBE_OPT_LIGHT_SHOTS                                */
    double evolve_ms[5];              /* by kernel index (entry 0 unused; 4 only for n >= 12)       */
    uint64_t light_candidates[4];
    double sample_ms[4];              /* by light-shot candidate                                    */
} ptsbe_tuning;

/* Autotuner: runs ptsbe_evolve_batch (every evolve kernel, flags as given) and then
 * ptsbe_evolve_sample (each light-shot limit) on sets [first, first + count) of set_id, `reps`
 * timed calls each after one warm-up, times them with CUDA events on the context stream, and sets
 * the context to the fastest evolve kernel and shot limit. The kernels give the same results up
 * to rounding (the shot limit changes no shot at all), so tuning changes speed only. Buffers as
 * for the two calls; d_states, d_weights, d_status and d_bits are overwritten. Host-synchronous.
 * Errors: those of the two calls; PTSBE_ERR_INVALID for reps = 0. */
PTSBE_API int ptsbe_autotune(ptsbe_ctx* ctx, uint32_t set_id, uint32_t first, uint32_t count, void* d_states,
                             double* d_weights, uint8_t* d_status, uint32_t flags, uint64_t seed, uint32_t* d_bits,
                             uint64_t d_bits_capacity, uint32_t reps, ptsbe_tuning* out);

/* ---------------------------------------------------------------------------------------- */
/* Instrumentation                                                                           */
/* ---------------------------------------------------------------------------------------- */

/* Number of CUDA kernels the library has enqueued since it was loaded (all contexts). */
PTSBE_API int ptsbe_kernel_launches(uint64_t* count);

/* Host-to-device bytes the library has copied since it was loaded (circuit tables, Kraus-set
 * entries, per-call schedules). */
PTSBE_API int ptsbe_h2d_bytes(uint64_t* bytes);

/* Prefix-reuse accounting of the context's last ptsbe_evolve_batch / ptsbe_evolve_sample call
 * (Sec. 3 batched execution with shared prefixes): *gates_applied = gates the call's passes applied,
 * summed over its Kraus sets (a pass run once for a group of sets that share it counts once);
 * *gates_without_reuse = the circuit's gates times the number of sets. The savings are
 * 1 - applied / without. Either pointer may be NULL. Host-only. */
PTSBE_API int ptsbe_reuse_stats(ptsbe_ctx* ctx, uint64_t* gates_applied, uint64_t* gates_without_reuse);

/* Work of the context's last call that ran dense passes (evolve kernel 4, or ptsbe_evolve_sample
 * without states): *pass_launches = passes run summed over the states they ran for; *fma = the
 * FP32 multiply-adds of those passes' fused blocks (a 2x2 complex block 8 per amplitude, a 4x4
 * block 16 per amplitude), the algorithmic arithmetic for an ALU roofline. Host-only. */
PTSBE_API int ptsbe_dense_work(ptsbe_ctx* ctx, uint64_t* pass_launches, double* fma);

/* The dense-pass plan of a circuit (built if needed; n < 12 is planned zero-padded to 12 qubits):
 * passes (of which fixup_passes only restore logical qubit order at the end), fused 1- and 2-qubit
 * blocks, and FP32 multiply-adds per amplitude (of the plan's state) of one full preparation. Any
 * pointer may be NULL. Host-only. */
PTSBE_API int ptsbe_dense_plan_info(ptsbe_ctx* ctx, uint32_t circuit_id, uint32_t* passes, uint32_t* fixup_passes,
                                    uint64_t* blocks_1q, uint64_t* blocks_2q, double* fma_per_amplitude);

/* Kernel classes of the timing counters. */
enum {
    PTSBE_TIMER_EVOLVE_STAGE = 0,     /* tile passes of ptsbe_evolve_batch                        */
    PTSBE_TIMER_EVOLVE_FINALIZE = 1,  /* norm reduction / renormalisation of ptsbe_evolve_batch   */
    PTSBE_TIMER_SAMPLE = 2,           /* cluster and global samplers; support-CDF sampler          */
    PTSBE_TIMER_PERSHOT = 3,          /* stage kernels of ptsbe_pershot_run (its readout: SAMPLE)   */
    PTSBE_TIMER_EVOLVE_PROGRAM = 4,   /* per-set program prepass of the deferred-frame kernel     */
    PTSBE_TIMER_SAMPLE_LIGHT = 5,     /* ptsbe_sample_shots: one-CTA-per-state light sampler      */
    PTSBE_TIMER_BACKWARD = 6,         /* ptsbe_backward                                           */
    PTSBE_TIMER_DENSE = 7,            /* dense tile passes (evolve kernel 4, and states not returned) */
    PTSBE_TIMER_ZERO_FILL = 8,        /* zero fill of the states of a small sparse final stage, run on
                                         the context's second stream beside the program prepass      */
    PTSBE_TIMER_CLASSES = 9
};

/* enable != 0: every later launch is bracketed by CUDA events recorded on the context stream and
 * its algorithmic bytes are added up per kernel class (state bytes read and written by a pass,
 * 4 bytes per shot ...). Adds two event records per launch. */
PTSBE_API int ptsbe_set_timing(ptsbe_ctx* ctx, int enable);

/* Waits for the timed launches and returns, for one kernel class, the summed event time in
 * milliseconds, the number of launches and the algorithmic bytes (any pointer may be NULL);
 * reset != 0 clears the counters afterwards. */
PTSBE_API int ptsbe_get_timing(ptsbe_ctx* ctx, int kernel_class, double* ms, uint64_t* launches, double* bytes,
                               int reset);

#ifdef __cplusplus
}
#endif

#endif /* PTSBE_H */
