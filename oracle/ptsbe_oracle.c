/*
 * PTSBE CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, complex128 implementation of Pre-Trajectory Sampling with Batched
 * Execution (Patti et al., "Augmenting Simulated Noisy Quantum Data Collection by Orders
 * of Magnitude Using Pre-Trajectory Sampling with Batched Execution", SC'25). It exists
 * to check the CUDA library; only the tests, the package's smoke check and the bench's
 * CPU-baseline leg may load it. It shares no code, header or table with the library.
 *
 * Passages followed:
 *   trajectory method (Kraus branch K_i chosen with probability <psi|K_i^dag K_i|psi>,
 *     applied, state renormalised)                                    -- Sec. 2.2
 *   unitary-mixture channels K_i = sqrt(p_i) U_i (the paper prints "p_i U_i")
 *                                                                     -- Sec. 2.2, item 2
 *   traditional per-operator trajectory loop                          -- Algorithm 1
 *   probabilistic pre-trajectory sampling, compatible / uniqueKraus   -- Algorithm 2
 *   proportional shot reallocation p'_a = p_a / sum p, probability bands,
 *     most-likely combinations above a cutoff                         -- Sec. 3.1
 *   batched execution: prepare each Kraus set once, draw all m_a shots -- Sec. 3
 *   fixed-set estimator of a diagonal observable (sets and q_a held fixed), the loss the
 *     adjoint backward differentiates; its gradient here is central finite differences
 *     (oracle.py, loss_grad_fd)                                       -- Sec. 3, Sec. 2.2
 *   counter-based RNG: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 *     numbers: as easy as 1, 2, 3", SC'11)
 *
 * Readings where the paper is silent are stated at each function. No compiler
 * floating-point contraction: build with -ffp-contract=off.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define OR_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011): 10 rounds of two 32x32->64 multiplies with a      */
/* Weyl-sequence key schedule.                                                           */
/* ------------------------------------------------------------------------------------ */
OR_API void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform in [0,1): the top 32 bits come from x0, the next 21 from x1. */
OR_API double or_u53(uint32_t x0, uint32_t x1) {
    uint64_t m = ((uint64_t)x0 << 21) | (uint64_t)(x1 >> 11);
    return (double)m * (1.0 / 9007199254740992.0);
}

static double uniform(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
    uint32_t ctr[4] = {c0, c1, c2, c3}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, o[4];
    or_philox(ctr, key, o);
    return or_u53(o[0], o[1]);
}

/* Counter domains (low byte of the fourth counter word). */
enum { DOM_PTS = 1, DOM_SHOT = 2, DOM_PERSHOT_KRAUS = 3, DOM_LITERAL = 4, DOM_PERSHOT_READ = 5 };

/* ------------------------------------------------------------------------------------ */
/* Gates. Single-qubit matrices are textbook (OpenQASM U3 convention). Two-qubit        */
/* matrices act on the local index 2*bit(t0) + bit(t1).                                  */
/* ------------------------------------------------------------------------------------ */
enum { G_I = 0, G_X, G_Y, G_Z, G_H, G_S, G_SDG, G_T, G_TDG, G_RX, G_RY, G_RZ, G_U3,
       G_CX, G_CZ, G_SWAP, G_U1, G_U2, G_COUNT };
enum { CH_DEPOL1 = 0, CH_DEPOL2, CH_AMPDAMP, CH_BITFLIP, CH_PHASEFLIP, CH_CUSTOM };

static int gate_arity(int g) { return (g == G_CX || g == G_CZ || g == G_SWAP || g == G_U2) ? 2 : 1; }

/* Writes the gate matrix (row-major, dim 2 or 4). Returns the dimension or 0. */
OR_API int or_gate_matrix(int g, const double* par, const double* custom /* 16 complex */,
                          double* out /* re,im interleaved */) {
    cplx m[16];
    for (int i = 0; i < 16; i++) m[i] = 0;
    double th = par[0], ph = par[1], la = par[2];
    int d = 2;
    switch (g) {
    case G_I: m[0] = 1; m[3] = 1; break;
    case G_X: m[1] = 1; m[2] = 1; break;
    case G_Y: m[1] = -I; m[2] = I; break;
    case G_Z: m[0] = 1; m[3] = -1; break;
    case G_H: m[0] = M_SQRT1_2; m[1] = M_SQRT1_2; m[2] = M_SQRT1_2; m[3] = -M_SQRT1_2; break;
    case G_S: m[0] = 1; m[3] = I; break;
    case G_SDG: m[0] = 1; m[3] = -I; break;
    case G_T: m[0] = 1; m[3] = cexp(I * M_PI / 4); break;
    case G_TDG: m[0] = 1; m[3] = cexp(-I * M_PI / 4); break;
    case G_RX: m[0] = cos(th / 2); m[1] = -I * sin(th / 2); m[2] = -I * sin(th / 2); m[3] = cos(th / 2); break;
    case G_RY: m[0] = cos(th / 2); m[1] = -sin(th / 2); m[2] = sin(th / 2); m[3] = cos(th / 2); break;
    case G_RZ: m[0] = cexp(-I * th / 2); m[3] = cexp(I * th / 2); break;
    case G_U3:
        m[0] = cos(th / 2);
        m[1] = -cexp(I * la) * sin(th / 2);
        m[2] = cexp(I * ph) * sin(th / 2);
        m[3] = cexp(I * (ph + la)) * cos(th / 2);
        break;
    case G_U1:
        m[0] = custom[0] + I * custom[1]; m[1] = custom[2] + I * custom[3];
        m[2] = custom[8] + I * custom[9]; m[3] = custom[10] + I * custom[11];
        break;
    case G_CX: d = 4; m[0] = 1; m[5] = 1; m[11] = 1; m[14] = 1; break;
    case G_CZ: d = 4; m[0] = 1; m[5] = 1; m[10] = 1; m[15] = -1; break;
    case G_SWAP: d = 4; m[0] = 1; m[6] = 1; m[9] = 1; m[15] = 1; break;
    case G_U2: d = 4; for (int i = 0; i < 16; i++) m[i] = custom[2 * i] + I * custom[2 * i + 1]; break;
    default: return 0;
    }
    for (int i = 0; i < d * d; i++) { out[2 * i] = creal(m[i]); out[2 * i + 1] = cimag(m[i]); }
    return d;
}

/* ------------------------------------------------------------------------------------ */
/* Channels: Kraus matrices, nominal probabilities q_k and unitary-mixture detection.    */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int kind, arity, dim, nk;
    cplx* K;        /* nk matrices, dim x dim, row-major */
    double* q;      /* nominal probability of Kraus k */
    int mixture;    /* 1 if every K_k = sqrt(q_k) U_k with U_k unitary (Sec. 2.2 item 2) */
    double param;
} or_channel;

static void pauli(int a, cplx* m) {
    double par[3] = {0, 0, 0}, buf[8];
    static const int code[4] = {G_I, G_X, G_Y, G_Z};
    or_gate_matrix(code[a], par, NULL, buf);
    for (int i = 0; i < 4; i++) m[i] = buf[2 * i] + I * buf[2 * i + 1];
}

/* Builds channel Kraus matrices. Depolarising (Nielsen & Chuang): {sqrt(1-p) I,
 * sqrt(p/3) X, Y, Z}. Two-qubit depolarising (reading of "16 Pauli Kraus"): sqrt(1-p) I(x)I
 * and sqrt(p/15) P_a (x) P_b for the 15 non-identity pairs, index k = 4a + b with P_a on
 * the first operand. Amplitude damping: K0 = [[1,0],[0,sqrt(1-g)]], K1 = [[0,sqrt(g)],[0,0]].
 * Bit flip {sqrt(1-p) I, sqrt(p) X}; phase flip {sqrt(1-p) I, sqrt(p) Z}. */
static int channel_build(or_channel* c, int kind, int arity, int nk, double param, const double* kraus) {
    if (arity < 1 || arity > 2 || nk < 1 || nk > 16) return -1;
    c->kind = kind; c->arity = arity; c->dim = 1 << arity; c->nk = nk; c->param = param;
    int d = c->dim, dd = d * d;
    c->K = (cplx*)calloc((size_t)nk * dd, sizeof(cplx));
    c->q = (double*)calloc((size_t)nk, sizeof(double));
    double p = param;
    cplx P[4][4];
    for (int a = 0; a < 4; a++) pauli(a, P[a]);
    switch (kind) {
    case CH_DEPOL1:
        if (arity != 1 || nk != 4) return -1;
        for (int a = 0; a < 4; a++) {
            double s = a == 0 ? sqrt(1 - p) : sqrt(p / 3);
            for (int i = 0; i < 4; i++) c->K[a * 4 + i] = s * P[a][i];
            c->q[a] = a == 0 ? 1 - p : p / 3;
        }
        break;
    case CH_DEPOL2:
        if (arity != 2 || nk != 16) return -1;
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) {
                int k = 4 * a + b;
                double s = k == 0 ? sqrt(1 - p) : sqrt(p / 15);
                for (int r = 0; r < 4; r++)
                    for (int col = 0; col < 4; col++)
                        c->K[k * 16 + r * 4 + col] = s * P[a][(r >> 1) * 2 + (col >> 1)] * P[b][(r & 1) * 2 + (col & 1)];
                c->q[k] = k == 0 ? 1 - p : p / 15;
            }
        break;
    case CH_AMPDAMP:
        if (arity != 1 || nk != 2) return -1;
        c->K[0] = 1; c->K[3] = sqrt(1 - p);
        c->K[4 + 1] = sqrt(p);
        c->q[0] = 1 - p / 2; c->q[1] = p / 2;
        break;
    case CH_BITFLIP:
    case CH_PHASEFLIP: {
        if (arity != 1 || nk != 2) return -1;
        int e = kind == CH_BITFLIP ? 1 : 3;
        for (int i = 0; i < 4; i++) { c->K[i] = sqrt(1 - p) * P[0][i]; c->K[4 + i] = sqrt(p) * P[e][i]; }
        c->q[0] = 1 - p; c->q[1] = p;
        break;
    }
    case CH_CUSTOM:
        for (int k = 0; k < nk; k++) {
            double s = 0;
            for (int i = 0; i < dd; i++) {
                double re = kraus[2 * (k * dd + i)], im = kraus[2 * (k * dd + i) + 1];
                c->K[k * dd + i] = re + I * im;
                s += re * re + im * im;
            }
            c->q[k] = s / d;
        }
        break;
    default: return -1;
    }
    /* unitary mixture: K_k^dag K_k = q_k * Identity for every k */
    c->mixture = 1;
    for (int k = 0; k < nk && c->mixture; k++) {
        for (int r = 0; r < d; r++)
            for (int col = 0; col < d; col++) {
                cplx s = 0;
                for (int i = 0; i < d; i++) s += conj(c->K[k * dd + i * d + r]) * c->K[k * dd + i * d + col];
                cplx want = (r == col) ? c->q[k] : 0;
                if (cabs(s - want) > 1e-12) c->mixture = 0;
            }
    }
    return 0;
}

/* max |sum_k K_k^dag K_k - I| : the CPTP condition of Sec. 2.2 */
static double channel_cptp_error(const or_channel* c) {
    int d = c->dim, dd = d * d;
    double worst = 0;
    for (int r = 0; r < d; r++)
        for (int col = 0; col < d; col++) {
            cplx s = 0;
            for (int k = 0; k < c->nk; k++)
                for (int i = 0; i < d; i++) s += conj(c->K[k * dd + i * d + r]) * c->K[k * dd + i * d + col];
            double e = cabs(s - (r == col ? 1.0 : 0.0));
            if (e > worst) worst = e;
        }
    return worst;
}

/* ------------------------------------------------------------------------------------ */
/* Circuit                                                                                */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int kind, id, nt, t0, t1;
    double par[3];
    int site;          /* noise-site index for NOISE ops, -1 for gates */
    int dim;           /* gate dimension */
    cplx M[16];        /* gate matrix */
} or_op;

typedef struct {
    int n;
    int n_ops, n_sites, n_ch;
    or_op* ops;
    or_channel* ch;
    int* site_op;      /* op index of each site */
    int* site_ch;      /* channel of each site */
    double Q0;         /* product over sites of q_{s,0}, site order */
} or_circuit;

OR_API void or_circuit_free(or_circuit* c) {
    if (!c) return;
    for (int i = 0; i < c->n_ch; i++) { free(c->ch[i].K); free(c->ch[i].q); }
    free(c->ch); free(c->ops); free(c->site_op); free(c->site_ch); free(c);
}

/* Returns NULL on malformed input. */
OR_API or_circuit* or_circuit_new(int n, int n_ops, const int32_t* op_ints, const double* op_params,
                                  int n_ch, const int32_t* ch_ints, const double* ch_params,
                                  const double* ch_kraus /* complex128 as re,im */, const int64_t* ch_kraus_off,
                                  const double* custom_gates /* [*][4][4] complex128 */, int n_custom) {
    if (n < 1 || n > 34) return NULL;
    or_circuit* c = (or_circuit*)calloc(1, sizeof(or_circuit));
    c->n = n; c->n_ops = n_ops; c->n_ch = n_ch;
    c->ops = (or_op*)calloc((size_t)(n_ops > 0 ? n_ops : 1), sizeof(or_op));
    c->ch = (or_channel*)calloc((size_t)(n_ch > 0 ? n_ch : 1), sizeof(or_channel));
    for (int j = 0; j < n_ch; j++) {
        const double* kr = (ch_kraus_off && ch_kraus_off[j] >= 0) ? ch_kraus + 2 * ch_kraus_off[j] : NULL;
        if (ch_ints[3 * j] == CH_CUSTOM && !kr) { or_circuit_free(c); return NULL; }
        if (channel_build(&c->ch[j], ch_ints[3 * j], ch_ints[3 * j + 1], ch_ints[3 * j + 2], ch_params[j], kr)) {
            c->n_ch = j + 1; or_circuit_free(c); return NULL;
        }
    }
    int s = 0;
    for (int i = 0; i < n_ops; i++) if (op_ints[5 * i] == 1) s++;
    c->n_sites = s;
    c->site_op = (int*)calloc((size_t)(s > 0 ? s : 1), sizeof(int));
    c->site_ch = (int*)calloc((size_t)(s > 0 ? s : 1), sizeof(int));
    s = 0;
    for (int i = 0; i < n_ops; i++) {
        or_op* o = &c->ops[i];
        o->kind = op_ints[5 * i]; o->id = op_ints[5 * i + 1]; o->nt = op_ints[5 * i + 2];
        o->t0 = op_ints[5 * i + 3]; o->t1 = op_ints[5 * i + 4];
        for (int k = 0; k < 3; k++) o->par[k] = op_params[3 * i + k];
        o->site = -1;
        if (o->nt < 1 || o->nt > 2 || o->t0 < 0 || o->t0 >= n || (o->nt == 2 && (o->t1 < 0 || o->t1 >= n || o->t1 == o->t0))) {
            or_circuit_free(c); return NULL;
        }
        if (o->kind == 0) {
            if (o->id < 0 || o->id >= G_COUNT || gate_arity(o->id) != o->nt) { or_circuit_free(c); return NULL; }
            const double* cu = NULL;
            if (o->id == G_U1 || o->id == G_U2) {
                int idx = (int)o->par[0];
                if (idx < 0 || idx >= n_custom) { or_circuit_free(c); return NULL; }
                cu = custom_gates + 32 * idx;
            }
            double buf[32];
            o->dim = or_gate_matrix(o->id, o->par, cu, buf);
            for (int k = 0; k < o->dim * o->dim; k++) o->M[k] = buf[2 * k] + I * buf[2 * k + 1];
        } else if (o->kind == 1) {
            if (o->id < 0 || o->id >= n_ch || c->ch[o->id].arity != o->nt) { or_circuit_free(c); return NULL; }
            o->site = s; c->site_op[s] = i; c->site_ch[s] = o->id; s++;
        } else { or_circuit_free(c); return NULL; }
    }
    c->Q0 = 1.0;
    for (int t = 0; t < c->n_sites; t++) c->Q0 *= c->ch[c->site_ch[t]].q[0];
    return c;
}

OR_API int or_circuit_sites(const or_circuit* c) { return c->n_sites; }
OR_API double or_circuit_Q0(const or_circuit* c) { return c->Q0; }

/* Channel introspection for the tests: Kraus matrices, q_k, mixture flag, CPTP error. */
OR_API int or_channel_info(const or_circuit* c, int j, double* kraus_out, double* q_out, int* mixture, double* cptp_err) {
    if (j < 0 || j >= c->n_ch) return -1;
    const or_channel* ch = &c->ch[j];
    int dd = ch->dim * ch->dim;
    if (kraus_out) for (int i = 0; i < ch->nk * dd; i++) { kraus_out[2 * i] = creal(ch->K[i]); kraus_out[2 * i + 1] = cimag(ch->K[i]); }
    if (q_out) for (int k = 0; k < ch->nk; k++) q_out[k] = ch->q[k];
    if (mixture) *mixture = ch->mixture;
    if (cptp_err) *cptp_err = channel_cptp_error(ch);
    return ch->nk;
}

/* ------------------------------------------------------------------------------------ */
/* State-vector kernels (complex128, plain loops).                                        */
/* ------------------------------------------------------------------------------------ */
static void apply1(cplx* psi, int n, int q, const cplx* M) {
    uint64_t N = 1ull << n, m = 1ull << q;
    for (uint64_t i = 0; i < N; i++) {
        if (i & m) continue;
        cplx a = psi[i], b = psi[i | m];
        psi[i] = M[0] * a + M[1] * b;
        psi[i | m] = M[2] * a + M[3] * b;
    }
}

static void apply2(cplx* psi, int n, int q0, int q1, const cplx* M) {
    uint64_t N = 1ull << n, m0 = 1ull << q0, m1 = 1ull << q1;
    for (uint64_t i = 0; i < N; i++) {
        if ((i & m0) || (i & m1)) continue;
        uint64_t idx[4] = {i, i | m1, i | m0, i | m0 | m1};  /* local index 2*b0 + b1 */
        cplx v[4], w[4];
        for (int l = 0; l < 4; l++) v[l] = psi[idx[l]];
        for (int r = 0; r < 4; r++) { w[r] = 0; for (int l = 0; l < 4; l++) w[r] += M[4 * r + l] * v[l]; }
        for (int l = 0; l < 4; l++) psi[idx[l]] = w[l];
    }
}

static void apply_matrix(cplx* psi, int n, int nt, int t0, int t1, const cplx* M) {
    if (nt == 1) apply1(psi, n, t0, M); else apply2(psi, n, t0, t1, M);
}

static double norm2(const cplx* psi, int n) {
    uint64_t N = 1ull << n;
    double s = 0;
    for (uint64_t i = 0; i < N; i++) s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    return s;
}

/* Smallest k with u < q_0 + ... + q_k (FP64, summed in listed order); the last index if
 * rounding leaves u above the total. (Reading of "index(r, {p_i})" in Algorithm 1.) */
static int categorical(double u, const double* q, int nk) {
    double acc = 0;
    for (int k = 0; k < nk; k++) { acc += q[k]; if (u < acc) return k; }
    return nk - 1;
}

/* ------------------------------------------------------------------------------------ */
/* Kraus sets                                                                             */
/* ------------------------------------------------------------------------------------ */
typedef struct { uint32_t site; uint8_t k; } ent;

typedef struct {
    uint32_t len;
    ent* e;             /* sorted by site, k != 0 */
    uint64_t mult;
    double key;         /* product of ratios q_{s,k}/q_{s,0}, multiplied in descending order */
} aset;

typedef struct {
    uint32_t count;
    aset* a;
    double* q;          /* nominal probability Q0 * key */
    uint64_t* shots;
} or_set;

static int ent_cmp(const ent* x, const ent* y) {
    if (x->site != y->site) return x->site < y->site ? -1 : 1;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    return 0;
}

/* Canonical order of Kraus sets: lexicographic over the (site, k) list, a proper prefix
 * before its extensions (so the empty set is first). */
static int aset_cmp(const aset* x, const aset* y) {
    uint32_t m = x->len < y->len ? x->len : y->len;
    for (uint32_t i = 0; i < m; i++) { int c = ent_cmp(&x->e[i], &y->e[i]); if (c) return c; }
    if (x->len != y->len) return x->len < y->len ? -1 : 1;
    return 0;
}
static int aset_qcmp(const void* a, const void* b) { return aset_cmp((const aset*)a, (const aset*)b); }

static double ratio(const or_circuit* c, uint32_t s, int k) {
    const or_channel* ch = &c->ch[c->site_ch[s]];
    return ch->q[k] / ch->q[0];
}

static int dbl_desc(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return x > y ? -1 : (x < y ? 1 : 0);
}

/* key(alpha): product of the ratios r_{s,k} = q_{s,k}/q_{s,0} of its entries, multiplied
 * from 1.0 in descending order of value, so equal multisets give identical keys. */
static double set_key(const or_circuit* c, const aset* a) {
    if (a->len == 0) return 1.0;
    double* r = (double*)malloc(sizeof(double) * a->len);
    for (uint32_t i = 0; i < a->len; i++) r[i] = ratio(c, a->e[i].site, a->e[i].k);
    qsort(r, a->len, sizeof(double), dbl_desc);
    double key = 1.0;
    for (uint32_t i = 0; i < a->len; i++) key *= r[i];
    free(r);
    return key;
}

static or_set* set_new(uint32_t count) {
    or_set* s = (or_set*)calloc(1, sizeof(or_set));
    s->count = count;
    s->a = (aset*)calloc(count ? count : 1, sizeof(aset));
    s->q = (double*)calloc(count ? count : 1, sizeof(double));
    s->shots = (uint64_t*)calloc(count ? count : 1, sizeof(uint64_t));
    return s;
}

OR_API void or_set_free(or_set* s) {
    if (!s) return;
    for (uint32_t i = 0; i < s->count; i++) free(s->a[i].e);
    free(s->a); free(s->q); free(s->shots); free(s);
}

OR_API uint32_t or_set_count(const or_set* s) { return s->count; }
OR_API uint64_t or_set_entries(const or_set* s) {
    uint64_t t = 0;
    for (uint32_t i = 0; i < s->count; i++) t += s->a[i].len;
    return t;
}
OR_API void or_set_export(const or_set* s, uint32_t* offsets, uint32_t* sites, uint8_t* kidx,
                          uint64_t* mult, double* q, uint64_t* shots) {
    uint64_t o = 0;
    for (uint32_t i = 0; i < s->count; i++) {
        offsets[i] = (uint32_t)o;
        for (uint32_t j = 0; j < s->a[i].len; j++) { sites[o] = s->a[i].e[j].site; kidx[o] = s->a[i].e[j].k; o++; }
        mult[i] = s->a[i].mult; q[i] = s->q[i]; shots[i] = s->shots[i];
    }
    offsets[s->count] = (uint32_t)o;
}

/* Sort into canonical order and merge duplicates (uniqueKraus of Algorithm 2): the
 * multiplicity c_alpha counts how often a set was drawn. Takes ownership of `a`. */
static or_set* finish_sets(const or_circuit* c, aset* a, uint64_t n) {
    qsort(a, n, sizeof(aset), aset_qcmp);
    uint64_t u = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (u > 0 && aset_cmp(&a[u - 1], &a[i]) == 0) { a[u - 1].mult += a[i].mult; free(a[i].e); continue; }
        a[u++] = a[i];
    }
    or_set* s = set_new((uint32_t)u);
    for (uint64_t i = 0; i < u; i++) {
        s->a[i] = a[i];
        s->a[i].key = set_key(c, &a[i]);
        s->q[i] = c->Q0 * s->a[i].key;
    }
    free(a);
    return s;
}

/* ------------------------------------------------------------------------------------ */
/* Shot allocation (Sec. 3.1 "redistributing ... according to the relative populations"). */
/* Reading: deterministic largest-remainder (Hamilton) apportionment of the total.       */
/* ------------------------------------------------------------------------------------ */
typedef struct { double rem; uint64_t rem_int; uint32_t idx; } remrec;
static int rem_desc(const void* a, const void* b) {
    const remrec* x = (const remrec*)a; const remrec* y = (const remrec*)b;
    if (x->rem != y->rem) return x->rem > y->rem ? -1 : 1;
    return x->idx < y->idx ? -1 : 1;
}
static int remint_desc(const void* a, const void* b) {
    const remrec* x = (const remrec*)a; const remrec* y = (const remrec*)b;
    if (x->rem_int != y->rem_int) return x->rem_int > y->rem_int ? -1 : 1;
    return x->idx < y->idx ? -1 : 1;
}
static int rem_asc_idx_desc(const void* a, const void* b) {
    const remrec* x = (const remrec*)a; const remrec* y = (const remrec*)b;
    if (x->rem != y->rem) return x->rem < y->rem ? -1 : 1;
    return x->idx > y->idx ? -1 : 1;
}

/* Integer weights: exact. out[i] = floor(M c_i / N) plus one for the R largest
 * remainders (M c_i mod N), ties to the lower index. */
OR_API void or_apportion_counts(uint32_t n, const uint64_t* c, uint64_t M, uint64_t* out) {
    unsigned __int128 N = 0;
    for (uint32_t i = 0; i < n; i++) N += c[i];
    if (n == 0) return;
    if (N == 0) { for (uint32_t i = 0; i < n; i++) out[i] = 0; return; }
    remrec* r = (remrec*)malloc(sizeof(remrec) * n);
    uint64_t used = 0;
    for (uint32_t i = 0; i < n; i++) {
        unsigned __int128 p = (unsigned __int128)M * c[i];
        out[i] = (uint64_t)(p / N);
        r[i].rem_int = (uint64_t)(p % N); r[i].rem = 0; r[i].idx = i;
        used += out[i];
    }
    uint64_t R = M - used;
    qsort(r, n, sizeof(remrec), remint_desc);
    for (uint64_t j = 0; j < R; j++) out[r[j].idx] += 1;
    free(r);
}

/* FP64 weights: quota_i = (M * w_i) / W, W summed in index order; floor; the R largest
 * remainders (quota - floor) get one more, ties to the lower index. If rounding makes the
 * floors exceed M, one is taken back from the smallest remainders (ties: higher index). */
OR_API void or_apportion_weights(uint32_t n, const double* w, uint64_t M, uint64_t* out) {
    if (n == 0) return;
    double W = 0;
    for (uint32_t i = 0; i < n; i++) W += w[i];
    remrec* r = (remrec*)malloc(sizeof(remrec) * n);
    uint64_t used = 0;
    for (uint32_t i = 0; i < n; i++) {
        double quota = W > 0 ? ((double)M * w[i]) / W : 0.0;
        double fl = floor(quota);
        out[i] = (uint64_t)fl;
        r[i].rem = quota - fl; r[i].idx = i; r[i].rem_int = 0;
        used += out[i];
    }
    if (used <= M) {
        uint64_t R = M - used;
        qsort(r, n, sizeof(remrec), rem_desc);
        for (uint64_t j = 0; j < R && j < n; j++) out[r[j].idx] += 1;
    } else {
        uint64_t R = used - M;
        qsort(r, n, sizeof(remrec), rem_asc_idx_desc);
        for (uint32_t j = 0; j < n && R > 0; j++) if (out[r[j].idx] > 0) { out[r[j].idx] -= 1; R--; }
    }
    free(r);
}

/* ------------------------------------------------------------------------------------ */
/* PTS: probabilistic sampling (Algorithm 2).                                             */
/* Reading: the per-operator draw "r <= p, then compatible" of the printed algorithm does */
/* not reproduce a multi-Kraus channel's distribution; "in much the same way as at state  */
/* preparation runtime" is read as one categorical draw per noise site: sample i, site s  */
/* draws u = U53(Philox(seed; s, i_lo, i_hi, 1)) and picks the smallest k with           */
/* u < q_0 + ... + q_k. k = 0 is "no error" and is not stored. Each site picks exactly one */
/* Kraus operator, so compatible() holds by construction.                                 */
/* ------------------------------------------------------------------------------------ */
static void aset_push(aset* a, uint32_t* cap, uint32_t s, int k) {
    if (a->len == *cap) { *cap = *cap ? 2 * *cap : 4; a->e = (ent*)realloc(a->e, sizeof(ent) * *cap); }
    a->e[a->len].site = s; a->e[a->len].k = (uint8_t)k; a->len++;
}

OR_API or_set* or_pts_proportional(const or_circuit* c, uint64_t nsamples, uint64_t seed, uint64_t total_shots,
                                   int alloc /* 0 counts, 1 uniform per set, 2 by q */, uint64_t nshots) {
    aset* a = (aset*)calloc(nsamples ? nsamples : 1, sizeof(aset));
    for (uint64_t i = 0; i < nsamples; i++) {
        uint32_t cap = 0;
        for (int s = 0; s < c->n_sites; s++) {
            const or_channel* ch = &c->ch[c->site_ch[s]];
            double u = uniform(seed, (uint32_t)s, (uint32_t)i, (uint32_t)(i >> 32), DOM_PTS);
            int k = categorical(u, ch->q, ch->nk);
            if (k != 0) aset_push(&a[i], &cap, (uint32_t)s, k);
        }
        a[i].mult = 1;
    }
    or_set* s = finish_sets(c, a, nsamples);
    if (alloc == 0) {
        uint64_t* m = (uint64_t*)malloc(sizeof(uint64_t) * (s->count ? s->count : 1));
        for (uint32_t i = 0; i < s->count; i++) m[i] = s->a[i].mult;
        or_apportion_counts(s->count, m, total_shots, s->shots);
        free(m);
    } else if (alloc == 1) {
        for (uint32_t i = 0; i < s->count; i++) s->shots[i] = nshots;
    } else {
        or_apportion_weights(s->count, s->q, total_shots, s->shots);
    }
    return s;
}

/* Algorithm 2 as printed: every (site, k != 0) draws r = U53(Philox(seed; s, i_lo, i_hi,
 * 4 | k << 8)); if r <= q_{s,k} and no operator was already taken at that site
 * (compatible), it is appended. Duplicates are merged; each unique set gets `nshots`. */
OR_API or_set* or_pts_literal(const or_circuit* c, uint64_t nsamples, uint64_t seed, uint64_t nshots) {
    aset* a = (aset*)calloc(nsamples ? nsamples : 1, sizeof(aset));
    for (uint64_t i = 0; i < nsamples; i++) {
        uint32_t cap = 0;
        for (int s = 0; s < c->n_sites; s++) {
            const or_channel* ch = &c->ch[c->site_ch[s]];
            int taken = 0;
            for (int k = 1; k < ch->nk; k++) {
                double r = uniform(seed, (uint32_t)s, (uint32_t)i, (uint32_t)(i >> 32), DOM_LITERAL | ((uint32_t)k << 8));
                if (r <= ch->q[k] && !taken) { aset_push(&a[i], &cap, (uint32_t)s, k); taken = 1; }
            }
        }
        a[i].mult = 1;
    }
    or_set* s = finish_sets(c, a, nsamples);
    for (uint32_t i = 0; i < s->count; i++) s->shots[i] = nshots;
    return s;
}

/* ------------------------------------------------------------------------------------ */
/* PTS: most likely combinations (Sec. 3.1). Options are all (s, k != 0) with q_{s,k} > 0, */
/* ordered by ratio descending then (s, k) ascending. A set's key is the product of its    */
/* option ratios in that order. The oracle enumerates every set whose key passes a         */
/* threshold by depth-first search over increasing option indices (pruning once the        */
/* product drops below the threshold) and then sorts; top-K finds the K-th largest key by   */
/* bisection on the threshold.                                                              */
/* ------------------------------------------------------------------------------------ */
typedef struct { uint32_t site; int k; double r; } opt;
static int opt_cmp(const void* a, const void* b) {
    const opt* x = (const opt*)a; const opt* y = (const opt*)b;
    if (x->r != y->r) return x->r > y->r ? -1 : 1;
    if (x->site != y->site) return x->site < y->site ? -1 : 1;
    return x->k < y->k ? -1 : 1;
}

typedef struct {
    const or_circuit* c;
    opt* o; uint32_t no;
    double tau;            /* keep key >= tau (top-K) */
    double pmin, pmax;     /* keep Q0*key in [pmin, pmax] (cutoff/band); pmin < 0 disables */
    uint64_t count, cap;   /* count visited sets; stop when count >= cap */
    int collect;
    aset* out; uint64_t nout, capout;
    uint8_t* used;         /* site -> taken */
    ent* stack; uint32_t depth;
} dfs_t;

static int keep(const dfs_t* d, double key) {
    if (d->pmin >= 0) { double q = d->c->Q0 * key; return q >= d->pmin && q <= d->pmax; }
    return key >= d->tau;
}
static int prune(const dfs_t* d, double key) {
    if (d->pmin >= 0) return d->c->Q0 * key < d->pmin;
    return key < d->tau;
}

static void dfs_record(dfs_t* d, double key) {
    d->count++;
    if (!d->collect) return;
    if (d->nout == d->capout) { d->capout = d->capout ? 2 * d->capout : 1024; d->out = (aset*)realloc(d->out, sizeof(aset) * d->capout); }
    aset* a = &d->out[d->nout++];
    a->len = d->depth; a->mult = 1; a->key = key;
    a->e = (ent*)malloc(sizeof(ent) * (d->depth ? d->depth : 1));
    memcpy(a->e, d->stack, sizeof(ent) * d->depth);
    /* sort entries by site (they were pushed in option order) */
    for (uint32_t i = 1; i < a->len; i++)
        for (uint32_t j = i; j > 0 && ent_cmp(&a->e[j], &a->e[j - 1]) < 0; j--) { ent t = a->e[j]; a->e[j] = a->e[j - 1]; a->e[j - 1] = t; }
}

static void dfs(dfs_t* d, uint32_t start, double key) {
    for (uint32_t j = start; j < d->no; j++) {
        if (d->count >= d->cap) return;
        double nk = key * d->o[j].r;
        if (prune(d, nk)) return;
        if (d->used[d->o[j].site]) continue;
        d->used[d->o[j].site] = 1;
        d->stack[d->depth].site = d->o[j].site; d->stack[d->depth].k = (uint8_t)d->o[j].k; d->depth++;
        if (keep(d, nk)) dfs_record(d, nk);
        dfs(d, j + 1, nk);
        d->depth--;
        d->used[d->o[j].site] = 0;
    }
}

static void dfs_init(dfs_t* d, const or_circuit* c) {
    memset(d, 0, sizeof(*d));
    d->c = c;
    uint32_t no = 0;
    for (int s = 0; s < c->n_sites; s++) no += c->ch[c->site_ch[s]].nk - 1;
    d->o = (opt*)malloc(sizeof(opt) * (no ? no : 1));
    no = 0;
    for (int s = 0; s < c->n_sites; s++) {
        const or_channel* ch = &c->ch[c->site_ch[s]];
        for (int k = 1; k < ch->nk; k++) {
            if (!(ch->q[k] > 0)) continue;
            d->o[no].site = (uint32_t)s; d->o[no].k = k; d->o[no].r = ch->q[k] / ch->q[0]; no++;
        }
    }
    d->no = no;
    qsort(d->o, no, sizeof(opt), opt_cmp);
    d->used = (uint8_t*)calloc(c->n_sites ? c->n_sites : 1, 1);
    d->stack = (ent*)malloc(sizeof(ent) * (c->n_sites + 1));
    d->pmin = -1;
}
static void dfs_free(dfs_t* d) { free(d->o); free(d->used); free(d->stack); }

static uint64_t count_above(const or_circuit* c, double tau, uint64_t cap) {
    dfs_t d; dfs_init(&d, c);
    d.tau = tau; d.cap = cap; d.collect = 0;
    if (keep(&d, 1.0)) d.count = 1;
    dfs(&d, 0, 1.0);
    uint64_t r = d.count;
    dfs_free(&d);
    return r;
}

static int key_then_canon(const void* x, const void* y) {
    const aset* a = (const aset*)x; const aset* b = (const aset*)y;
    if (a->key != b->key) return a->key > b->key ? -1 : 1;
    return aset_cmp(a, b);
}

/* Returns NULL if q_{s,0} is not the strict maximum at some site (ratios must be < 1). */
static int check_mode_k0(const or_circuit* c) {
    for (int s = 0; s < c->n_sites; s++) {
        const or_channel* ch = &c->ch[c->site_ch[s]];
        if (!(ch->q[0] > 0)) return 0;
        for (int k = 1; k < ch->nk; k++) if (!(ch->q[k] < ch->q[0])) return 0;
    }
    return 1;
}

static void dfs_collect(dfs_t* d) {
    if (keep(d, 1.0)) { d->depth = 0; dfs_record(d, 1.0); }
    dfs(d, 0, 1.0);
}

OR_API or_set* or_pts_topk(const or_circuit* c, uint64_t K, uint64_t total_shots, int alloc, uint64_t nshots) {
    if (!check_mode_k0(c)) return NULL;
    /* Largest tau with count(key >= tau) >= K, by bisection over the ordered bit patterns
     * of doubles in [0, 1]. */
    uint64_t lo, hi;
    double one = 1.0, zero = 0.0;
    memcpy(&hi, &one, 8); memcpy(&lo, &zero, 8);
    if (count_above(c, 1.0, K) >= K) lo = hi;
    else if (count_above(c, 0.0, K) < K) { /* fewer than K sets with positive key: take them all */ }
    else {
        while (hi - lo > 1) {
            uint64_t mid = lo + (hi - lo) / 2;
            double t; memcpy(&t, &mid, 8);
            if (count_above(c, t, K) >= K) lo = mid; else hi = mid;
        }
    }
    double tau; memcpy(&tau, &lo, 8);
    dfs_t d; dfs_init(&d, c);
    d.tau = tau; d.cap = UINT64_MAX; d.collect = 1;
    dfs_collect(&d);
    qsort(d.out, d.nout, sizeof(aset), key_then_canon);
    uint64_t keepn = d.nout < K ? d.nout : K;
    for (uint64_t i = keepn; i < d.nout; i++) free(d.out[i].e);
    dfs_free(&d);
    or_set* s = finish_sets(c, d.out, keepn);
    if (alloc == 1) for (uint32_t i = 0; i < s->count; i++) s->shots[i] = nshots;
    else or_apportion_weights(s->count, s->q, total_shots, s->shots);
    return s;
}

/* Every set with p_min <= q_alpha <= p_max (cutoff: p_max = 1). */
OR_API or_set* or_pts_band(const or_circuit* c, double pmin, double pmax, uint64_t total_shots, int alloc, uint64_t nshots) {
    if (!check_mode_k0(c) || !(pmin > 0)) return NULL;
    dfs_t d; dfs_init(&d, c);
    d.pmin = pmin; d.pmax = pmax; d.cap = UINT64_MAX; d.collect = 1;
    dfs_collect(&d);
    dfs_free(&d);
    or_set* s = finish_sets(c, d.out, d.nout);
    if (alloc == 1) for (uint32_t i = 0; i < s->count; i++) s->shots[i] = nshots;
    else or_apportion_weights(s->count, s->q, total_shots, s->shots);
    return s;
}

/* Caller-given sets (targeted error sets, Sec. 3.1 "selection criteria"). Entries of a set
 * must have strictly increasing sites and 0 < k < n_kraus. Duplicate sets are merged (their
 * multiplicities and shots add). shots == NULL: apportion total_shots in proportion to q. */
typedef struct { aset a; uint64_t s; } tpair;
static int tpair_cmp(const void* x, const void* y) { return aset_cmp(&((const tpair*)x)->a, &((const tpair*)y)->a); }

OR_API or_set* or_pts_targeted(const or_circuit* c, uint32_t count, const uint32_t* offsets, const uint32_t* sites,
                               const uint8_t* kidx, const uint64_t* shots, uint64_t total_shots) {
    tpair* p = (tpair*)calloc(count ? count : 1, sizeof(tpair));
    for (uint32_t i = 0; i < count; i++) {
        uint32_t b = offsets[i], e = offsets[i + 1];
        int bad = e < b;
        for (uint32_t j = b; j < e && !bad; j++)
            bad = sites[j] >= (uint32_t)c->n_sites || kidx[j] == 0 || kidx[j] >= c->ch[c->site_ch[sites[j]]].nk ||
                  (j > b && sites[j] <= sites[j - 1]);
        if (bad) { for (uint32_t t = 0; t < i; t++) free(p[t].a.e); free(p); return NULL; }
        p[i].a.len = e - b; p[i].a.mult = 1; p[i].s = shots ? shots[i] : 0;
        p[i].a.e = (ent*)malloc(sizeof(ent) * (e > b ? e - b : 1));
        for (uint32_t j = b; j < e; j++) { p[i].a.e[j - b].site = sites[j]; p[i].a.e[j - b].k = kidx[j]; }
    }
    qsort(p, count, sizeof(tpair), tpair_cmp);
    uint32_t u = 0;
    for (uint32_t i = 0; i < count; i++) {
        if (u > 0 && aset_cmp(&p[u - 1].a, &p[i].a) == 0) { p[u - 1].a.mult++; p[u - 1].s += p[i].s; free(p[i].a.e); continue; }
        p[u++] = p[i];
    }
    or_set* s = set_new(u);
    for (uint32_t i = 0; i < u; i++) {
        s->a[i] = p[i].a;
        s->a[i].key = set_key(c, &s->a[i]);
        s->q[i] = c->Q0 * s->a[i].key;
        s->shots[i] = p[i].s;
    }
    if (!shots) or_apportion_weights(s->count, s->q, total_shots, s->shots);
    free(p);
    return s;
}

/* ------------------------------------------------------------------------------------ */
/* Batched execution, preparation step (Sec. 3): evolve |0...0> through the circuit with  */
/* the Kraus operators of alpha fixed. Unitary-mixture sites apply U_k = K_k / sqrt(q_k)   */
/* and multiply the weight by q_k; other sites apply K_k, renormalise, and multiply the     */
/* weight by the squared norm (Sec. 2.2). Reading (null rule): a set whose weight is below */
/* 1e-6 of its nominal probability is marked null (status 1).                              */
/* ------------------------------------------------------------------------------------ */
static int kraus_at(const aset* a, uint32_t site, uint32_t* ptr) {
    while (*ptr < a->len && a->e[*ptr].site < site) (*ptr)++;
    if (*ptr < a->len && a->e[*ptr].site == site) return a->e[*ptr].k;
    return 0;
}

static void apply_site(const or_circuit* c, cplx* psi, const or_op* o, int k, double* w, int* dead) {
    const or_channel* ch = &c->ch[o->id];
    int dd = ch->dim * ch->dim;
    if (ch->mixture) {
        cplx U[16];
        double s = sqrt(ch->q[k]);
        for (int i = 0; i < dd; i++) U[i] = ch->K[k * dd + i] / s;
        apply_matrix(psi, c->n, o->nt, o->t0, o->t1, U);
        *w *= ch->q[k];
    } else {
        apply_matrix(psi, c->n, o->nt, o->t0, o->t1, &ch->K[k * dd]);
        double n2 = norm2(psi, c->n);
        *w *= n2;
        if (n2 > 0) {
            double inv = 1.0 / sqrt(n2);
            uint64_t N = 1ull << c->n;
            for (uint64_t i = 0; i < N; i++) psi[i] *= inv;
        } else *dead = 1;
    }
}

OR_API int or_evolve(const or_circuit* c, const or_set* s, uint32_t idx, double* state_out /* 2^n complex */,
                     double* w_out, int* status_out) {
    if (idx >= s->count) return -1;
    const aset* a = &s->a[idx];
    uint64_t N = 1ull << c->n;
    cplx* psi = (cplx*)calloc(N, sizeof(cplx));
    psi[0] = 1;
    double w = 1.0;
    int dead = 0;
    uint32_t ptr = 0;
    for (int i = 0; i < c->n_ops && !dead; i++) {
        const or_op* o = &c->ops[i];
        if (o->kind == 0) apply_matrix(psi, c->n, o->nt, o->t0, o->t1, o->M);
        else apply_site(c, psi, o, kraus_at(a, (uint32_t)o->site, &ptr), &w, &dead);
    }
    if (dead) { memset(psi, 0, N * sizeof(cplx)); w = 0; }
    int status = (w == 0 || w / s->q[idx] < 1e-6) ? 1 : 0;
    memcpy(state_out, psi, N * sizeof(cplx));
    *w_out = w; *status_out = status;
    free(psi);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Batched execution, sampling step (Sec. 3: "sampling all m_alpha desired bitstrings at   */
/* once"). P_i = |psi_i|^2 in FP64, C = inclusive prefix summed sequentially, T = C[last]. */
/* Shot j of set alpha: u = U53(Philox(seed; j_lo, j_hi, alpha, 2)), outcome = smallest i  */
/* with u*T < C[i] (the last index if none).                                               */
/* ------------------------------------------------------------------------------------ */
static uint64_t search(const double* C, uint64_t N, double t) {
    uint64_t lo = 0, hi = N;  /* smallest i with t < C[i] */
    while (lo < hi) { uint64_t mid = lo + (hi - lo) / 2; if (t < C[mid]) hi = mid; else lo = mid + 1; }
    return lo < N ? lo : N - 1;
}

OR_API void or_cdf(int n, const double* state, double* C) {
    uint64_t N = 1ull << n;
    double acc = 0;
    for (uint64_t i = 0; i < N; i++) {
        double re = state[2 * i], im = state[2 * i + 1];
        acc += re * re + im * im;
        C[i] = acc;
    }
}

OR_API void or_sample(int n, const double* state, uint64_t m, uint64_t seed, uint32_t alpha, uint64_t first_shot,
                      uint64_t* out) {
    uint64_t N = 1ull << n;
    double* C = (double*)malloc(sizeof(double) * N);
    or_cdf(n, state, C);
    double T = C[N - 1];
    for (uint64_t j = first_shot; j < first_shot + m; j++) {
        double u = uniform(seed, (uint32_t)j, (uint32_t)(j >> 32), alpha, DOM_SHOT);
        out[j - first_shot] = search(C, N, u * T);
    }
    free(C);
}

/* Uniform of shot j (so the tests can apply the boundary rule). */
OR_API double or_shot_uniform(uint64_t seed, uint32_t alpha, uint64_t j) {
    return uniform(seed, (uint32_t)j, (uint32_t)(j >> 32), alpha, DOM_SHOT);
}

/* ------------------------------------------------------------------------------------ */
/* Traditional trajectory, one shot (Algorithm 1). At each noise site draw                */
/* u = U53(Philox(seed; s, j_lo, j_hi, 3)). Unitary mixture: k = index(u, {q}) and apply   */
/* U_k. General channel: p_i = <psi|K_i^dag K_i|psi> (the printed "<Psi|K_i^dag K|psi>" is */
/* read as this), k = index(u, {p}), apply K_k / sqrt(p_k). The final state is read out    */
/* with u = U53(Philox(seed; j_lo, j_hi, 0, 5)) by the inverse-CDF rule above.              */
/* kraus_out (optional) receives the chosen k of every site.                               */
/* ------------------------------------------------------------------------------------ */
OR_API uint64_t or_pershot(const or_circuit* c, uint64_t seed, uint64_t j, uint8_t* kraus_out) {
    uint64_t N = 1ull << c->n;
    cplx* psi = (cplx*)calloc(N, sizeof(cplx));
    cplx* tmp = (cplx*)calloc(N, sizeof(cplx));
    psi[0] = 1;
    for (int i = 0; i < c->n_ops; i++) {
        const or_op* o = &c->ops[i];
        if (o->kind == 0) { apply_matrix(psi, c->n, o->nt, o->t0, o->t1, o->M); continue; }
        const or_channel* ch = &c->ch[o->id];
        int dd = ch->dim * ch->dim;
        double u = uniform(seed, (uint32_t)o->site, (uint32_t)j, (uint32_t)(j >> 32), DOM_PERSHOT_KRAUS);
        int k;
        if (ch->mixture) {
            k = categorical(u, ch->q, ch->nk);
            cplx U[16];
            double s = sqrt(ch->q[k]);
            for (int t = 0; t < dd; t++) U[t] = ch->K[k * dd + t] / s;
            apply_matrix(psi, c->n, o->nt, o->t0, o->t1, U);
        } else {
            double p[16];
            for (int kk = 0; kk < ch->nk; kk++) {
                memcpy(tmp, psi, N * sizeof(cplx));
                apply_matrix(tmp, c->n, o->nt, o->t0, o->t1, &ch->K[kk * dd]);
                p[kk] = norm2(tmp, c->n);
            }
            k = categorical(u, p, ch->nk);
            while (k > 0 && !(p[k] > 0)) k--;  /* rounding fallback landed on an impossible branch */
            apply_matrix(psi, c->n, o->nt, o->t0, o->t1, &ch->K[k * dd]);
            double inv = 1.0 / sqrt(p[k]);
            for (uint64_t t = 0; t < N; t++) psi[t] *= inv;
        }
        if (kraus_out) kraus_out[o->site] = (uint8_t)k;
    }
    double* C = (double*)malloc(sizeof(double) * N);
    or_cdf(c->n, (const double*)psi, C);
    double u = uniform(seed, (uint32_t)j, (uint32_t)(j >> 32), 0, DOM_PERSHOT_READ);
    uint64_t out = search(C, N, u * C[N - 1]);
    free(C); free(psi); free(tmp);
    return out;
}

/* ------------------------------------------------------------------------------------ */
/* Estimator for the adjoint backward: L = (1/N) sum_alpha c_alpha <psi~_a|O|psi~_a> / q_a */
/* with psi~_a the unnormalised state (every Kraus operator applied as given, K_k not U_k) */
/* and O = sum_t coeff_t prod_{q in mask_t} Z_q diagonal. With alpha and q_alpha fixed     */
/* this is an importance-sampling estimate of Tr(O rho); its derivatives with respect to   */
/* gate angles and channel strengths are what the backward computes.                        */
/* ------------------------------------------------------------------------------------ */
/* Shared body: O(x) = diag[x] when diag is given, plus the Z-string terms. */
static double loss_body(const or_circuit* c, const or_set* s, uint32_t nterms, const uint64_t* masks,
                        const double* coeffs, const double* diag, double* per_set) {
    uint64_t N = 1ull << c->n;
    cplx* psi = (cplx*)malloc(N * sizeof(cplx));
    double total = 0, Ntot = 0;
    for (uint32_t a = 0; a < s->count; a++) Ntot += (double)s->a[a].mult;
    for (uint32_t a = 0; a < s->count; a++) {
        memset(psi, 0, N * sizeof(cplx));
        psi[0] = 1;
        uint32_t ptr = 0;
        for (int i = 0; i < c->n_ops; i++) {
            const or_op* o = &c->ops[i];
            if (o->kind == 0) apply_matrix(psi, c->n, o->nt, o->t0, o->t1, o->M);
            else {
                const or_channel* ch = &c->ch[o->id];
                int k = kraus_at(&s->a[a], (uint32_t)o->site, &ptr);
                apply_matrix(psi, c->n, o->nt, o->t0, o->t1, &ch->K[k * ch->dim * ch->dim]);
            }
        }
        double e = 0;
        for (uint64_t x = 0; x < N; x++) {
            double pr = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
            double ov = diag ? diag[x] : 0.0;
            for (uint32_t t = 0; t < nterms; t++) ov += (__builtin_popcountll(x & masks[t]) & 1) ? -coeffs[t] : coeffs[t];
            e += pr * ov;
        }
        double v = (double)s->a[a].mult * e / s->q[a];
        if (per_set) per_set[a] = e / s->q[a];
        total += v;
    }
    free(psi);
    return total / Ntot;
}

OR_API double or_loss(const or_circuit* c, const or_set* s, uint32_t nterms, const uint64_t* masks, const double* coeffs,
                      double* per_set /* optional [count] */) {
    return loss_body(c, s, nterms, masks, coeffs, NULL, per_set);
}

/* Same estimator for a caller-given diagonal observable O = sum_x diag[x] |x><x| (2^n values,
 * e.g. the indicator of one outcome for the gradient of an outcome probability), plus terms. */
OR_API double or_loss_diag(const or_circuit* c, const or_set* s, uint32_t nterms, const uint64_t* masks,
                           const double* coeffs, const double* diag, double* per_set) {
    return loss_body(c, s, nterms, masks, coeffs, diag, per_set);
}
