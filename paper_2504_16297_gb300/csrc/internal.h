// Internal data structures of libptsbe shared by the host code and the CUDA kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <complex>
#include <stdexcept>
#include <string>
#include <vector>
#include <array>

#include <cuda_runtime.h>

#include "../../include/ptsbe.h"
#include "dense.cuh"

namespace ptsbe {

constexpr int kMaxKraus = 16;
constexpr int kMaxQubits = 32;
constexpr int kTileMax = 14;      // largest tile: 2^14 complex64 = 128 KiB of shared memory
constexpr int kPershotTileBits = 12;   // tile of the Algorithm 1 path's plan (PTSBE_OPT_PERSHOT_TILE_BITS; measured)
constexpr int kLowBits = 4;       // low qubits every tile keeps contiguous (16 amplitudes = 128 B)
constexpr int kSmallSupportBits = 10;   // sparse final stages with a support of at most 2^10 amplitudes
                                        // run the small-buffer frame kernel

// ---------------------------------------------------------------------------------------------
// Errors: thrown inside the library, turned into a status at the ABI boundary.
// ---------------------------------------------------------------------------------------------
struct Error : std::runtime_error {
    int status;
    Error(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};
[[noreturn]] inline void fail(int status, const std::string& msg) { throw Error(status, msg); }

void cuda_check(cudaError_t e, const char* what);
void count_launch(uint64_t n = 1);   // kernels enqueued by the library (all contexts)
void count_h2d(uint64_t bytes);      // host-to-device bytes copied by the library
uint64_t launches_so_far();
#define PTSBE_CUDA(call) ::ptsbe::cuda_check((call), #call)

// ---------------------------------------------------------------------------------------------
// Device op tables. A circuit becomes a list of DevOp; a gate is one micro-kernel, a noise site
// selects the micro-op list of its chosen Kraus operator at run time.
// ---------------------------------------------------------------------------------------------
enum : uint8_t {
    DOP_G1 = 0,    // general 2x2: mat[0..3]
    DOP_D1 = 1,    // diagonal 2x2: mat[0], mat[1]
    DOP_X1 = 2,    // anti-diagonal [[0, a], [b, 0]]: mat[0] = a, mat[1] = b
    DOP_CX = 3,    // controlled-X, control q0, target q1
    DOP_CZ = 4,    // diag(1, 1, 1, -1)
    DOP_SWAP = 5,
    DOP_G2 = 6,    // general 4x4 on local index 2*bit(q0) + bit(q1): mat[0..15]
    DOP_NOISE = 7, // noise site: ch, site
    DOP_NOP = 8,   // identity
    DOP_M2 = 9     // monomial 4x4: out[l] = d[l] * in[perm_l], d = mat[0..3], perm packed 2 bits per l
};

struct DevOp {
    uint8_t kind;
    uint8_t q0, q1;
    uint8_t nt;
    uint32_t mat;    // offset into the complex64 matrix pool
    uint32_t site;   // DOP_NOISE: site index
    uint32_t ch;     // DOP_NOISE: channel index
    // A gate fused with the "no error" Kraus operators of the noise sites right after it on its
    // own qubits. Used when the state's set has no entry among those sites; otherwise the ops run
    // one by one.
    uint8_t fkind;   // DOP_NOP when nothing is fused (kind of the fused operator otherwise)
    uint8_t fperm;   // DOP_M2 permutation
    uint8_t fsep;    // DOP_M2: 1 when d[2 l_a + l_b] = alpha[l_a] beta[l_b]; fmat[4..7] = alpha, beta
    uint8_t pad;
    uint32_t fmat;   // fused operator in the matrix pool
    uint32_t fend;   // op index after the absorbed noise ops
    uint32_t fsite1; // one past the last absorbed site
};

struct DevMicro {
    uint8_t kind;     // DOP_G1 / D1 / X1 / G2 / NOP
    uint8_t operand;  // 0: first target, 1: second target, 2: both (G2)
    uint16_t pad;
    uint32_t mat;
};

struct DevChannel {
    uint32_t micro_off[kMaxKraus + 1];  // micro ops of Kraus k: [micro_off[k], micro_off[k+1])
    uint32_t herm_mat[kMaxKraus];       // K_k^dag K_k (for Algorithm 1 probabilities), pool offset
    double q[kMaxKraus];                // nominal probabilities (unitary mixture: exact mixing weights)
    uint8_t nk, arity, mixture, pad;
};

// One pass of the tiled evolution: ops [op_begin, op_end) all act inside the qubit set of the
// tile. Tile index l (tb bits): bits [0, lb) are global qubits [0, lb) (contiguous in memory),
// bits [lb, tb) are the global qubits listed in tile_q[lb..tb); the remaining n - tb qubits
// (outer_q) enumerate the 2^(n-tb) tiles of a state.
struct DevStage {
    uint32_t op_begin, op_end;
    uint32_t group_begin, group_end; // register groups of this stage
    uint32_t hi_off;                 // offset of this stage's hi table (2^(tb-lb) uint32)
    uint32_t flags;                  // bit 0: ends right before a general noise site (Algorithm 1 mode)
    uint32_t probe_op;               // Algorithm 1 mode: the general noise op whose probabilities
                                     // the epilogue accumulates
    uint8_t pos[kMaxQubits];         // global qubit -> tile bit, 0xFF if outer
    uint8_t outer_q[kMaxQubits];     // outer bit b -> global qubit
};

// Register group: consecutive ops of a stage that only touch kRegBits tile positions. Each thread
// of the CTA holds the 2^kRegBits amplitudes whose tile index has its thread id spread over
// lane_pos and runs over every combination of reg_pos, so the ops apply without shared memory.
constexpr int kRegBits = 4;
struct DevGroup {
    uint32_t op_begin, op_end;
    uint8_t reg_pos[kRegBits];       // register bit b <- tile position reg_pos[b]
    uint8_t rbit[kTileMax];          // tile position -> register bit (0xFF when it is a lane bit)
    uint8_t lane_pos[kTileMax];      // thread-id bit i -> tile position lane_pos[i] (ascending)
    uint8_t pad[3];
};

// Deferred-frame plan, per stage. Between stages the state of logical index l is stored at global
// index A_j l (A_j invertible over GF(2), the same for every Kraus set); a stage's tile is a set of
// global index bits (DevStage::pos/outer_q/hi) that holds the directions of its mixing operators.
struct DevFrameStage {
    uint32_t col[kMaxQubits];        // A at the stage start: global image of logical bit q
    uint32_t row[kMaxQubits];        // rows of A^-1: logical bit q = <row[q], global index>
    // Stages that end in logical order (the last one, and any stage after which the frame restarts
    // at the identity because a permutation spread a mixing direction wider than a tile): tile-local
    // index t holds logical l = l0 ^ sum_k t_k w[k] at tile-local address sum_k t_k m[k];
    // l0 = R b ^ (xor of ox[i] over the set outer bits i of the tile index); w[k] = e_k for k < lbf,
    // so runs of 2^lbf amplitudes stay contiguous.
    uint32_t w[kTileMax];
    uint16_t m[kTileMax];
    uint32_t ox[kMaxQubits];
    uint32_t last, lbf;              // last: the stage ends in logical order
    // Sparse final store (a one-stage plan of a multi-tile state, every set from |0...0>): one CTA
    // per state holds all nonzero amplitudes (they stay in the tile holding index 0), so it
    // computes the norm, zero-fills the state and scatters each amplitude to its logical index
    // l = R_end (x ^ b) (rowe = rows of A^-1 at the stage end). No other tile runs.
    uint32_t sparse_final;
    uint32_t rowe[kMaxQubits];
    // Sparse final stage whose nonzero amplitudes all sit at tile addresses below 2^sbits (the
    // stage is entered in a layout that maps the span of its mixing directions to the low bits);
    // 0 when only the tile bound holds.
    uint32_t sbits;
};

struct Plan {
    int tb = 0, lb = 0;              // tile bits, contiguous low bits
    std::vector<DevStage> stages;
    std::vector<DevGroup> groups;
    std::vector<uint32_t> hi;        // concatenated hi tables: global offset of tile bits [lb, tb)
    std::vector<int32_t> op_stage;   // op index -> stage
    std::vector<DevFrameStage> fstages;   // deferred-frame plans only
};

// ---------------------------------------------------------------------------------------------
// Adjoint backward. The circuit becomes a list of fused blocks ("items", the consecutive
// operators of one or two qubits, noise sites included); a set's state lives in the shared memory
// of a thread-block cluster (local bits = low qubit positions, cluster rank = high positions) and
// the plan swaps qubit positions between CTAs so that every item acts on local bits.
// ---------------------------------------------------------------------------------------------
constexpr int kBwMaxErr = 64;        // (site, k) entries per set
constexpr int kBwMaxMembers = 48;    // operators fused into one item
constexpr int kBwLocalBits = 13;     // local bits of a cluster CTA (two complex64 vectors: 128 KiB)
constexpr int kBwMaxQubits = 16;     // clusters of at most 8 CTAs
constexpr uint32_t kBwNone = 0xFFFFFFFFu;

struct BwMember {
    uint32_t mat;      // FP32 pool block of variant 0 (variant k at mat + k); a block = 16 float2
    uint32_t inv;      // FP32 pool block of the inverse of variant 0 (zeros where singular)
    uint32_t m64;      // FP64 pool block of variant 0 (variant k at m64 + k)
    uint32_t d64;      // FP64 pool block of the first derivative matrix (gate: angle j at d64 + j;
                       // general channel: d(variant k)/d strength at d64 + k)
    uint32_t sing;     // bit k: variant k cannot be inverted (its input comes from a checkpoint)
    uint32_t dslot;    // gradient slot of the first angle (gate) or of the site (general channel)
    uint8_t noise, nk, nd, pad;   // nd: gate angles, or 1 for a differentiable site, else 0
};

struct BwItem {
    uint8_t nq, p0, p1, diff;   // 1 or 2 qubits at physical positions p0 (high matrix bit), p1
    uint32_t mbeg, mend;        // members
    uint32_t def, definv;       // FP32 pool blocks of the default product (every variant 0) and inverse
    uint32_t defsing;           // the default product cannot be inverted
    uint32_t gslot;             // slot of its outer-product accumulator (differentiable items)
    uint32_t ckpt;              // store phi before this block: un-computing through the blocks since
                                // the last stored copy would amplify rounding too much (see kBwCondLog2)
};

struct BwStep {
    uint32_t kind;              // 0 item, 1 swap local position a with global position g
    uint32_t a, g, item;
};

// Un-computing phi_{t-1} = B_t^-1 phi_t multiplies the rounding error of phi_t by up to the
// condition number kappa(B_t) (relative to the state's norm); through a run of blocks the factors
// multiply. The plan stores phi before a block once the product of kappa over the blocks that would
// be un-computed since the last stored copy would exceed 2^kBwCondLog2 (damping K0 = diag(1,
// sqrt(1 - gamma)) has kappa = 1 / sqrt(1 - gamma); unitary blocks have kappa = 1).
constexpr double kBwCondLog2 = 6.0;

struct BwPlan {
    bool built = false;
    int nl = 0;
    uint32_t cond_ckpts = 0;             // blocks marked ckpt
    // Kraus variants of general channels are stored scaled to spectral norm 1 (a damping jump
    // K1 = [[0, sqrt g], [0, 0]] would otherwise shrink the FP32 state by sqrt g per jump, and a
    // set with tens of jumps underflows into subnormals); their derivative matrices carry the same
    // constant. A set's state, loss and gradients are then all multiplied by C = prod over its
    // general sites of c_k^2, which the host divides out of its weight in FP64. logc[logc_off[m] + k]
    // = ln c_k^2 of member m's variant k (kBwNone: a gate or a unitary mixture, c = 1);
    // logc_default = sum over every general site of its variant-0 term.
    std::vector<double> logc;
    std::vector<uint32_t> logc_off;
    double logc_default = 0.0;
    std::vector<BwStep> steps;
    std::vector<BwItem> items;
    std::vector<BwMember> members;
    std::vector<float2> pool;            // 16 per block
    std::vector<double> pool64;          // 32 per block (complex as re, im)
    std::vector<uint32_t> site_item, site_mem;
    std::vector<uint32_t> dslot_out;     // dslot -> 3 op + j (gate angle) or 0x80000000 | channel (site)
    std::vector<uint8_t> pos_final;      // logical qubit -> physical position after the last step
    uint32_t ngs = 0, ndslots = 0, first_diff_step = 0;
    std::vector<uint32_t> defsing_items; // items whose default product cannot be inverted
    double P0mix = 1.0;                  // prod over unitary-mixture sites of q_{s,0}
    void* dev = nullptr;                 // device copy (one allocation)
    const BwStep* d_steps = nullptr;
    const BwItem* d_items = nullptr;
    const BwMember* d_members = nullptr;
    const float2* d_pool = nullptr;
    const double* d_pool64 = nullptr;
    const uint32_t* d_site_item = nullptr;
    const uint32_t* d_site_mem = nullptr;
    const uint32_t* d_dslot_out = nullptr;
    const uint8_t* d_pos_final = nullptr;
};

// ---------------------------------------------------------------------------------------------
// Dense tile passes (dense.cuh): the circuit cut into passes over kT-bit tiles, each pass's
// operators fused into 1- and 2-qubit blocks and grouped by register bits. Built on first use.
// ---------------------------------------------------------------------------------------------
struct DensePlan {
    bool built = false;
    int n = 0;
    std::vector<dense::Pass> passes;
    std::vector<dense::Group> groups;
    std::vector<dense::Block> blocks;         // execution order; blocks[i].id == i
    std::vector<uint32_t> hi;
    std::vector<uint16_t> omap;
    std::vector<float2> mats;                 // default block matrices (every site at Kraus operator 0)
    // host records for the per-set override blocks
    std::vector<uint32_t> site_block;         // noise site -> block id
    std::vector<uint32_t> blk_pass;           // block id -> pass
    std::vector<uint32_t> blk_op_off;         // block id -> its ops [blk_op_off[b], blk_op_off[b+1]) in blk_ops
    std::vector<uint32_t> blk_ops;
    std::vector<uint8_t> blk_nq;              // 1 or 2
    std::vector<uint32_t> blk_qa, blk_qb;     // logical qubits; block basis index 2 bit(qa) + bit(qb)
    std::vector<uint8_t> blk_swap;            // kernel local index = bit(qa) + 2 bit(qb) (else 2 bit(qa) + bit(qb))
    // Phases carried between blocks (diagonal-times-real form): the state after block b is
    // D_out(b) times what the kernel holds, D_out a product of one diagonal per qubit. blk_pin: the
    // per-qubit diagonals (qa entries 0, 1; qb entries 2, 3) the block absorbs on its input;
    // blk_pout: those it leaves (identity for a general block).
    std::vector<std::array<std::complex<double>, 4>> blk_pin, blk_pout;
    std::vector<uint32_t> pass_gates;         // gates applied by each pass (prefix-reuse accounting)
    std::vector<uint32_t> pass_fma;           // FP32 multiply-adds per amplitude of each pass's blocks
                                              // (a 2x2 block 8, a 4x4 block 16: complex products of 4)
    uint32_t fixup_passes = 0;                // trailing passes that only restore logical order
    void* dev = nullptr;                      // device copy (one allocation)
    const dense::Pass* d_passes = nullptr;
    const dense::Group* d_groups = nullptr;
    const dense::Block* d_blocks = nullptr;
    const uint32_t* d_hi = nullptr;
    const uint16_t* d_omap = nullptr;
    const float2* d_mats = nullptr;
};

// ---------------------------------------------------------------------------------------------
// Host-side circuit and Kraus-set records.
// ---------------------------------------------------------------------------------------------
using cd = std::complex<double>;

struct HostChannel {
    uint32_t kind = 0, arity = 1, nk = 0, dim = 2;
    double param = 0;
    std::vector<cd> K;       // nk * dim * dim, row-major
    std::vector<double> q;   // nominal probabilities
    std::vector<cd> U;       // unitary-mixture: K_k / sqrt(q_k)
    bool mixture = false;
};

// Channels the adjoint backward applies as U_k = K_k / sqrt(q_k) with the scale q_k kept apart:
// unitary mixtures other than damping (whose derivative is not a multiple of K_k).
inline bool bw_unit_channel(const HostChannel& ch) { return ch.mixture && ch.kind != PTSBE_CH_AMPDAMP; }

struct DeviceCircuit {
    void* base = nullptr;            // one device allocation holding every table below
    DevOp* ops = nullptr;
    DevMicro* micro = nullptr;
    float2* mats = nullptr;
    DevChannel* chans = nullptr;
    uint32_t* site_op = nullptr;
    DevStage* stages = nullptr;
    DevGroup* groups = nullptr;
    uint32_t* hi = nullptr;
    DevFrameStage* fstages = nullptr;
    size_t bytes = 0;
    cudaEvent_t ready = nullptr;     // recorded after the upload, on the stream that made it
};

struct Circuit {
    uint32_t n = 0;
    std::vector<ptsbe_op> ops;
    std::vector<double> custom;      // custom gate rows, 4x4 complex128 as (re, im)
    std::vector<HostChannel> ch;
    std::vector<uint32_t> site_op, site_ch;
    uint64_t n_gates = 0;
    double Q0 = 1.0;                 // prod_s q_{s,0}, site order
    bool k0_strict_mode = true;      // q_{s,0} > q_{s,k} for all k at every site
    // device form
    std::vector<DevOp> dops;
    std::vector<DevMicro> dmicro;
    std::vector<float2> dmats;
    std::vector<DevChannel> dchans;
    Plan plan;                       // PTSBE evolution plan (ops inside each stage's qubit set)
    Plan plan_pershot;               // Algorithm 1 plan (stage break before every general site)
    Plan plan_frame;                 // deferred-frame plan (mixing directions inside each tile)
    BwPlan bw;                       // adjoint backward plan (built on the first backward call)
    DensePlan dense;                 // dense tile passes (built on first use)
    bool pershot_planned = false;
    int pershot_tb = 0;              // tile bits plan_pershot was made for
    bool frame_planned = false;
    bool op_planned = false;         // per-operator plan (sweep and register-blocked kernels) built
    DeviceCircuit dev;
    DeviceCircuit dev_pershot;
    DeviceCircuit dev_frame;
};

struct KSet {
    uint32_t circuit = 0;
    std::vector<uint32_t> off;       // [count + 1]
    std::vector<uint32_t> site;
    std::vector<uint8_t> k;
    std::vector<uint64_t> mult, shots, shot_off;
    std::vector<double> q, key;
    // device copies of the entries (uploaded on first use)
    uint32_t* d_site = nullptr;
    uint8_t* d_k = nullptr;
    cudaEvent_t ready = nullptr;     // recorded after the upload, on the stream that made it
    uint32_t count() const { return (uint32_t)(off.size() - 1); }
};

// PTS (host) ----------------------------------------------------------------------------------
void pts_run(const Circuit& c, const ptsbe_pts_params& p, uint64_t seed, KSet& out);
void apportion_counts(const std::vector<uint64_t>& c, uint64_t M, std::vector<uint64_t>& out);
void apportion_weights(const std::vector<double>& w, uint64_t M, std::vector<uint64_t>& out);
double set_key(const Circuit& c, const uint32_t* sites, const uint8_t* ks, uint32_t len);

// Registration and planning (host) -----------------------------------------------------------------
void gate_matrix_of(uint32_t g, const double* params, const double* custom, cd* m, int& dim);
void embed_pair(const cd* m, int dim, const uint32_t* qs, uint32_t q0, uint32_t q1, cd* out);
void make_backward_plan(const Circuit& c, BwPlan& P);
void build_channel(const ptsbe_channel& in, HostChannel& c);
void register_ops(Circuit& c, const ptsbe_op* ops, uint64_t n_ops, const double* custom, uint32_t n_custom);
void build_device_ops(Circuit& c);
Plan make_plan(const Circuit& c, int tile_bits, bool pershot);
Plan make_frame_plan(const Circuit& c, int tile_bits);
void make_dense_plan(const Circuit& c, DensePlan& P);
// Override matrix of block b (kernel layout, complex64, a general 2x2 or 4x4; *code its block code)
// with Kraus operator ks[i] at site sites[i] (sites inside the block, increasing) and operator 0 at
// its other sites, including the phases the block takes in and leaves (blk_pin, blk_pout).
void dense_block_matrix(const Circuit& c, const DensePlan& P, uint32_t b, const uint32_t* sites, const uint8_t* ks,
                        uint32_t len, float2* out, uint32_t* code);

// ---------------------------------------------------------------------------------------------
// Kernel launch interface (evolve.cu / sample.cu / pershot.cu).
// ---------------------------------------------------------------------------------------------
struct EvolveArgs {
    // circuit
    const DevOp* ops;
    const DevMicro* micro;
    const float2* mats;
    uint32_t n_mats;                 // entries of mats
    uint32_t stage_mats;             // per-operator kernel: entries of mats staged in shared memory (0: none)
    const DevChannel* chans;
    const uint32_t* site_op;
    const DevStage* stages;
    const DevGroup* groups;
    const uint32_t* hi;
    const DevFrameStage* fstages;
    int n, tb, lb;
    // Kraus-set entries (whole set, on device)
    const uint32_t* ent_site;
    const uint8_t* ent_k;
    // per-node tables (range-local node index). A node runs stages node_sstage .. J-1; in its first
    // stage it reads the state of slot node_src (its prefix parent's input of that stage, or its
    // own slot), later its own slot; node_fresh: it starts from |0...0> in stage 0.
    const uint32_t* node_ebeg;
    const uint32_t* node_eend;
    const uint32_t* node_sstage;
    const uint32_t* node_src;
    const uint8_t* node_fresh;
    const double* wmix;              // prod of unitary-mixture q over all sites
    const double* qalpha;
    // states: a stage reads states_in and writes states ([count][2^n] each; the same buffer
    // without prefix reuse, alternating buffers with it)
    const float2* states_in;
    float2* states;
    double* part;                    // [count][2^(n-tb)] last-stage partial norms
    double* weights;
    uint8_t* status;
    void* frame_progs;               // frame kernel: one program per node of a launch
    int store_norm;                  // frame kernel: stage-end stores also leave tile norm partials in part
    int sparse_final_stage;          // frame kernel: stage with the sparse final store (one CTA per state), or -1
    const float* scale_in;           // frame kernel: the last stage writes psi * scale_in[node] (norm known)
    int small_bits;                  // frame kernel: support bits of the sparse final stage (0: tile-sized buffer)
    // Shots drawn by the small sparse final stage from the support it holds on chip (null
    // shot_bits: none). Node i draws node_shots[i] shots (0: drawn later by a sampler kernel) into
    // shot_bits[node_shot_out[i] ...], with Philox counter word 2 = shot_alpha0 + i.
    uint32_t* shot_bits;
    const uint32_t* node_shots;
    const uint64_t* node_shot_out;
    uint64_t shot_seed;
    uint32_t shot_alpha0;
    uint32_t* fault;                 // set nonzero when a launch could not do its work (checked by the host)
    // Heavy states of the small sparse final stage: node i with node_export[i] != ~0 leaves its
    // support CDF in slot node_export[i] of support_out (SupportCdf layout) for k_sample_support.
    const uint32_t* node_export;
    unsigned char* support_out;
    // Small sparse final stage: the first prefill_bytes of every state were zeroed by
    // k_zero_states before the launch; the launch's bulk copies zero the rest.
    uint64_t prefill_bytes;
};

// A state's outcome CDF over its support, in increasing outcome order (2^-62 fixed point), as the
// small sparse final stage leaves it for heavy states: header, then cdf[2^sbits], then lidx[2^sbits].
struct SupportCdfHeader {
    unsigned long long T;            // total (inclusive prefix of the last entry)
    uint32_t n;                      // entries (a power of two)
    uint32_t mark_all;               // 1: every shot is `mark` (null state, or a support not ordered)
    uint32_t mark;
    uint32_t nq;                     // qubits: outcome 2^nq - 1 when T = 0 (as the dense samplers)
    uint32_t pad[2];
};
#ifdef __CUDACC__
__host__ __device__
#endif
inline size_t support_slot_bytes(int sbits) { return sizeof(SupportCdfHeader) + ((size_t)12 << sbits); }

struct SupportItem {                 // a shot range of one exported state
    uint32_t slot, alpha;
    uint64_t j0, j1, out0;
};
void launch_sample_support(const unsigned char* slots, size_t slot_bytes, const SupportItem* d_items, uint32_t n_items,
                           uint64_t seed, uint32_t* bits, cudaStream_t s);

// kernel: 0 auto (= 3), 1 shared-memory sweeps, 2 register-blocked, 3 deferred frame
void launch_evolve_stage(const EvolveArgs& a, int stage, bool last, const uint32_t* d_nodes, uint32_t n_nodes,
                         cudaStream_t s, int kernel = 0);
// Frame kernel (kernel 0 or 3): builds the per-node programs of a stage; must precede
// launch_evolve_stage of the same stage and nodes.
// Zero fill of the first `prefix` bytes (a multiple of 4096) of each of `count` states of
// `state_bytes` from the 16-byte aligned `base`: bulk copies of a zeroed shared buffer, at most one
// one-warp CTA per SM (it shares the SMs with a running program prepass).
// Copies the first 2^n_out amplitudes of each of `count` states of 2^n_in amplitudes (a dense
// plan zero-padded to kT qubits) to the caller's buffer of 2^n_out-amplitude states.
void launch_dense_unpad(const float2* src, int n_in, float2* dst, int n_out, uint32_t count, int n_sm, cudaStream_t s);
void launch_zero_states(void* base, uint64_t state_bytes, uint64_t prefix, uint32_t count, int n_sm, cudaStream_t s);
void launch_frame_program(const EvolveArgs& a, int stage, const uint32_t* d_nodes, uint32_t n_nodes, cudaStream_t s,
                          int sets_per_warp);
// Reduce (weights, flags, scales) and scale; for n == tb only with one_tile_too (the dense passes:
// the other kernels normalise a one-tile state themselves).
void launch_evolve_finalize(const EvolveArgs& a, uint32_t count, float* d_scale, cudaStream_t s,
                            bool one_tile_too = false);
void launch_evolve_reduce(const EvolveArgs& a, uint32_t count, float* d_scale, cudaStream_t s);
size_t evolve_frame_program_bytes();   // workspace per node of a frame-kernel launch

struct SampleItem {                  // one cluster's share of one state's shots
    uint32_t state;                  // range-local state index
    uint32_t alpha;                  // global set index (Philox counter word 2)
    uint64_t j0, j1;                 // shot interval within the set
    uint64_t out0;                   // output slot of shot j0
    uint32_t dom;                    // Philox counter word 3 (counter domain)
    uint32_t pad;
};

struct SampleArgs {
    int n;
    const float2* states;
    const uint8_t* status;
    uint64_t seed;
    uint32_t* bits;
    unsigned long long* scratch;     // n > 17: per-state global CDF workspace (2^-62 fixed point)
    unsigned long long* scratch_tot; // n > 17: per-block totals / offsets
};

void launch_sample_cluster(const SampleArgs& a, const SampleItem* d_items, uint32_t n_items, cudaStream_t s);
void launch_sample_global(const SampleArgs& a, uint32_t state, uint32_t alpha, uint64_t j0, uint64_t j1,
                          uint64_t out0, cudaStream_t s, uint32_t dom = 2);

// Algorithm 1: one trajectory per shot, Kraus operators drawn while the state evolves.
struct PershotArgs {
    const DevOp* ops;
    const DevMicro* micro;
    const float2* mats;
    const DevChannel* chans;
    const DevStage* stages;
    const uint32_t* hi;
    int n, tb, lb;
    uint64_t seed;
    uint64_t first_shot;             // global index of the batch's first shot
    float2* states;                  // [batch][2^n]
    double* part;                    // [2][batch][2^(n-tb)][kMaxKraus] branch-probability partials
    uint8_t* kraus;                  // optional [batch][n_sites] chosen Kraus index per site
    uint64_t n_sites;
};
void launch_pershot_stage(const PershotArgs& a, int stage, uint32_t batch, cudaStream_t s);
// Adjoint backward kernels (backward.cu).
struct BwArgs {
    int n, nl, cl;
    uint32_t nslots, count;
    const BwStep* steps; uint32_t nsteps, first_diff_step;
    const BwItem* items; uint32_t nitems;
    const BwMember* members;
    const float2* pool;
    const double* pool64;
    const uint32_t* site_item;
    const uint32_t* site_mem;
    const uint32_t* dslot_out;
    const uint8_t* pos_final;
    // Kraus-set entries (whole set) and per-set tables of the range
    const uint32_t* ent_site;
    const uint8_t* ent_k;
    const uint32_t* ebeg;          // [count + 1] absolute entry offsets
    const double* W;               // mult s^2 / (N q): weight of a set's <phi|O|phi>
    const double* s2q;             // s^2 / q: per-set output factor
    const double* gmix;            // [count][nch]: d log s^2 / d strength of channel c
    int nch;
    // observable (physical masks of the final layout)
    uint32_t nterms;
    const uint32_t* pmask;
    const double* coeff;
    const double* diag;            // logical-index diagonal or nullptr
    uint32_t ckpt_every, maxck, ngs, ndslots, n_ops;
    // workspace
    float2* ckpt;                  // [nslots][maxck][2^n]
    double* Ga;                    // [nslots][cl][ngs][32]: a set's outer products
    double* Gbar;                  // [nslots][cl][ngs][32]: weighted sums over default items
    double* acc_err;               // [nslots][ndslots]
    double* acc_mix;               // [nslots][nch]
    double* acc_loss;              // [nslots]
    double* dtot;                  // [ndslots] finish-kernel scratch
    // outputs
    double* per_set;
    double* loss;
    double* grad_params;
    double* grad_noise;
};
uint32_t backward_slots(int n, uint32_t count, int n_sm);
void launch_backward(const BwArgs& a, cudaStream_t s);

struct DenseArgs {
    const dense::Pass* passes;
    const dense::Group* groups;
    const dense::Block* blocks;
    const uint32_t* hi;
    const uint16_t* omap;
    const float2* mats;
    const dense::Node* nodes;
    uint32_t n_nodes;
    const dense::Override* ovr;
    const float2* opool;
    int n, pass, last;
    double* part;                    // last pass: [rows][2^(n - kT)] tile squared norms
    uint32_t stage_bytes;            // dynamic shared memory: the pass's staged tables (0: read from global)
};
void launch_dense_pass(const DenseArgs& a, int n_sm, cudaStream_t s);
int dense_ctas_per_sm();

// One persistent launch over many circuits' dense passes (a device work queue, dense.cu).
struct QJob {                        // one circuit's range of Kraus sets, prepared in place
    const dense::Pass* passes;
    const dense::Group* groups;
    const dense::Block* blocks;
    const uint32_t* hi;
    const uint16_t* omap;
    const float2* mats;
    const dense::Override* ovr;
    const float2* opool;
    const uint32_t* ov_begin;        // [count] override range of each set
    const uint32_t* ov_end;
    float2* states;                  // [count][2^n]
    double* part;                    // [count][2^(n - kT)] tile norms of the last pass
    const double* wmix;              // [count] prod of unitary-mixture q
    const double* qalpha;            // [count]
    double* weights;                 // [count] or null
    uint8_t* status;                 // [count] or null
    float* scale;                    // [count]
    uint32_t n, J, count, pad;
};
struct QTask {
    uint64_t item0;                  // first global work item
    uint32_t job, set;               // set: job-local index
    uint32_t level;                  // pass j < J; J: finalisation; J + 1: scaling
    uint32_t items;                  // work items of this task
    uint32_t pred;                   // task that must finish first (~0: none)
    uint32_t pred_items;             // its work items
};
struct QueueArgs {
    const QJob* jobs;
    const QTask* tasks;
    uint32_t n_tasks;
    uint64_t n_items;
    unsigned long long* next;        // global item counter (zero before the launch)
    uint32_t* done;                  // [n_tasks] finished items (zero before the launch)
    uint32_t* err;                   // nonzero: a wait ran out (the task index + 1)
    long long spin_cycles;           // wait budget in clock64 cycles
    uint32_t stall_task;             // test hook: this task waits for one item more than its predecessor has
};
void launch_dense_queue(const QueueArgs& a, int n_sm, cudaStream_t s);
int dense_queue_grid(int n_sm);

int unique_max_qubits();
size_t unique_bitmap_bytes(int n);
void launch_unique(const uint32_t* bits, const uint64_t* d_pieces, uint32_t n_pieces, uint32_t count, int n,
                   uint32_t* d_bitmaps, unsigned long long* out, cudaStream_t s);
int sample_cluster_max_qubits();
void configure_samplers();
int sample_light_max_qubits();
// Default shot limit of the one-CTA-per-state light sampler (15 <= n <= 20); heavier states go to
// the cluster sampler. Both give the same shots (exact integer prefix sums), so the limit only
// moves work between the kernels (PTSBE_OPT_LIGHT_SHOTS).
constexpr uint64_t kLightShotLimit = 65536;
constexpr uint64_t kSupportChunk = 1ull << 16;   // shots per k_sample_support work item
void launch_sample_light(const SampleArgs& a, const SampleItem* d_items, uint32_t n_items, cudaStream_t s);

}  // namespace ptsbe
