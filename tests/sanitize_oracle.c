/* Sanitizer run of the oracle (test infrastructure): built with -fsanitize=address,undefined by
 * tests/test_sanitizers.py and run on circuit dumps written by that test. It calls every oracle
 * entry point the tests use -- circuit construction, PTS in four modes, evolution, CDF and
 * sampling, Algorithm 1, the loss -- and frees everything, so the sanitizers see every path. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

typedef struct or_circuit or_circuit;
typedef struct or_set or_set;
or_circuit* or_circuit_new(int n, int n_ops, const int32_t* op_ints, const double* op_params, int n_ch,
                           const int32_t* ch_ints, const double* ch_params, const double* ch_kraus,
                           const int64_t* ch_kraus_off, const double* custom_gates, int n_custom);
void or_circuit_free(or_circuit* c);
or_set* or_pts_proportional(const or_circuit* c, uint64_t nsamples, uint64_t seed, uint64_t total_shots, int alloc,
                            uint64_t nshots);
or_set* or_pts_literal(const or_circuit* c, uint64_t nsamples, uint64_t seed, uint64_t nshots);
or_set* or_pts_topk(const or_circuit* c, uint64_t K, uint64_t total_shots, int alloc, uint64_t nshots);
or_set* or_pts_band(const or_circuit* c, double pmin, double pmax, uint64_t total_shots, int alloc, uint64_t nshots);
uint32_t or_set_count(const or_set* s);
void or_set_free(or_set* s);
int or_evolve(const or_circuit* c, const or_set* s, uint32_t idx, double* state_out, double* w_out, int* status_out);
void or_cdf(int n, const double* state, double* C);
void or_sample(int n, const double* state, uint64_t m, uint64_t seed, uint32_t alpha, uint64_t first_shot, uint64_t* out);
uint64_t or_pershot(const or_circuit* c, uint64_t seed, uint64_t j, uint8_t* kraus_out);
double or_loss(const or_circuit* c, const or_set* s, uint32_t nterms, const uint64_t* masks, const double* coeffs,
               double* per_set);

static void* rd(FILE* f, size_t n, size_t size) {
    void* p = calloc(n ? n : 1, size);
    if (n && fread(p, size, n, f) != n) { fprintf(stderr, "short dump\n"); exit(2); }
    return p;
}

static void exercise(const or_circuit* c, or_set* s, int n, uint64_t* shots, double* state, double* C) {
    if (!s) return;
    const uint32_t cnt = or_set_count(s);
    for (uint32_t i = 0; i < cnt && i < 6; ++i) {
        double w = 0;
        int st = 0;
        if (or_evolve(c, s, i, state, &w, &st) != 0) { fprintf(stderr, "evolve failed\n"); exit(3); }
        or_cdf(n, state, C);
        or_sample(n, state, 500, 11, i, 0, shots);
    }
    const uint64_t mask = n > 1 ? 3u : 1u;
    const double coeff = 0.5;
    double* per = (double*)calloc(cnt ? cnt : 1, sizeof(double));
    (void)or_loss(c, s, 1, &mask, &coeff, per);
    free(per);
    or_set_free(s);
}

int main(int argc, char** argv) {
    if (argc < 2) return 1;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 1;
    int64_t h[5];
    if (fread(h, sizeof(int64_t), 5, f) != 5) return 2;
    const int n = (int)h[0], n_ops = (int)h[1], n_ch = (int)h[2], n_custom = (int)h[4];
    const int64_t n_kraus = h[3];
    int32_t* op_ints = (int32_t*)rd(f, (size_t)n_ops * 5, 4);
    double* op_params = (double*)rd(f, (size_t)n_ops * 3, 8);
    int32_t* ch_ints = (int32_t*)rd(f, (size_t)n_ch * 3, 4);
    double* ch_params = (double*)rd(f, (size_t)n_ch, 8);
    double* kraus = (double*)rd(f, (size_t)n_kraus * 2, 8);
    int64_t* koff = (int64_t*)rd(f, (size_t)n_ch, 8);
    double* custom = (double*)rd(f, (size_t)n_custom * 32, 8);
    fclose(f);
    or_circuit* c = or_circuit_new(n, n_ops, op_ints, op_params, n_ch, ch_ints, ch_params, kraus, koff,
                                   n_custom ? custom : NULL, n_custom);
    if (!c) { fprintf(stderr, "circuit rejected\n"); return 4; }
    double* state = (double*)calloc((size_t)2 << n, sizeof(double));
    double* C = (double*)calloc((size_t)1 << n, sizeof(double));
    uint64_t* shots = (uint64_t*)calloc(500, sizeof(uint64_t));
    exercise(c, or_pts_proportional(c, 120, 7, 2000, 0, 0), n, shots, state, C);
    exercise(c, or_pts_literal(c, 60, 3, 1), n, shots, state, C);
    exercise(c, or_pts_topk(c, 40, 1000, 2, 0), n, shots, state, C);    /* NULL when not strictly ordered */
    exercise(c, or_pts_band(c, 1e-3, 1.0, 1000, 2, 0), n, shots, state, C);   /* a band of a few sets */
    uint8_t* kr = (uint8_t*)calloc(1u << 16, 1);
    for (uint64_t j = 0; j < 8; ++j) (void)or_pershot(c, 9, j, kr);
    free(kr); free(shots); free(C); free(state);
    or_circuit_free(c);
    free(op_ints); free(op_params); free(ch_ints); free(ch_params); free(kraus); free(koff); free(custom);
    printf("oracle sanitizer run ok\n");
    return 0;
}
