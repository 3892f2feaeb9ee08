// Sanitizer run of the library's host-side planning and builder code (test infrastructure): built
// with -fsanitize=address,undefined by tests/test_sanitizers.py together with the CPU harnesses of
// the frame and dense kernels (tests/frame_host.cpp, tests/dense_host.cpp) and the library's host
// sources. Runs registration, the frame plan at a small and the full tile size, every set's frame
// program and tile steps, and the dense plan (zero-padded below 12 qubits) with every set's
// override blocks, on circuit and Kraus-set dumps written by the test.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "ptsbe.h"
#include <cuda_runtime.h>

extern "C" {
int fh_register(uint32_t n, const ptsbe_op* ops, uint64_t n_ops, const ptsbe_channel* chans, uint32_t n_ch,
                const double* custom, uint32_t n_custom, int tile_bits);
int fh_evolve(uint32_t count, const uint32_t* off, const uint32_t* site, const uint8_t* kk, const double* q, int reuse,
              float2* states, double* weights, uint8_t* status);
int dh_register(uint32_t n, const ptsbe_op* ops, uint64_t n_ops, const ptsbe_channel* chans, uint32_t n_ch,
                const double* custom, uint32_t n_custom);
double dh_evolve(const uint32_t* sites, const uint8_t* ks, uint32_t len, float* out);
int dh_pad_errors();
}

template <class T>
static std::vector<T> rd(FILE* f, size_t n) {
    std::vector<T> v(n ? n : 1);
    if (n && fread(v.data(), sizeof(T), n, f) != n) { std::fprintf(stderr, "short dump\n"); std::exit(2); }
    return v;
}

int main(int argc, char** argv) {
    if (argc < 2) return 1;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 1;
    int64_t h[5];
    if (std::fread(h, sizeof(int64_t), 5, f) != 5) return 2;
    const uint32_t n = (uint32_t)h[0], n_ops = (uint32_t)h[1], n_ch = (uint32_t)h[2], n_custom = (uint32_t)h[4];
    auto op_ints = rd<int32_t>(f, (size_t)n_ops * 5);
    auto op_params = rd<double>(f, (size_t)n_ops * 3);
    auto ch_ints = rd<int32_t>(f, (size_t)n_ch * 3);
    auto ch_params = rd<double>(f, n_ch);
    auto kraus = rd<double>(f, (size_t)h[3] * 2);
    auto koff = rd<int64_t>(f, n_ch);
    auto custom = rd<double>(f, (size_t)n_custom * 32);
    int64_t cnt64 = 0;
    if (std::fread(&cnt64, sizeof(int64_t), 1, f) != 1) return 2;
    const uint32_t count = (uint32_t)cnt64;
    auto off = rd<uint32_t>(f, count + 1);
    const size_t E = off[count];
    auto site = rd<uint32_t>(f, E);
    auto kk = rd<uint8_t>(f, E);
    auto q = rd<double>(f, count);
    std::fclose(f);
    std::vector<ptsbe_op> ops(n_ops);
    for (uint32_t i = 0; i < n_ops; ++i) {
        ops[i].kind = (uint32_t)op_ints[5 * i]; ops[i].id = (uint32_t)op_ints[5 * i + 1];
        ops[i].n_targets = (uint32_t)op_ints[5 * i + 2];
        ops[i].targets[0] = (uint32_t)op_ints[5 * i + 3]; ops[i].targets[1] = (uint32_t)op_ints[5 * i + 4];
        for (int j = 0; j < 3; ++j) ops[i].params[j] = op_params[3 * i + j];
    }
    std::vector<ptsbe_channel> ch(n_ch);
    for (uint32_t j = 0; j < n_ch; ++j) {
        ch[j].kind = (uint32_t)ch_ints[3 * j]; ch[j].arity = (uint32_t)ch_ints[3 * j + 1];
        ch[j].n_kraus = (uint32_t)ch_ints[3 * j + 2]; ch[j].param = ch_params[j];
        ch[j].kraus = koff[j] >= 0 ? kraus.data() + 2 * koff[j] : nullptr;
    }
    const double* cg = n_custom ? custom.data() : nullptr;
    std::vector<float2> states((size_t)count << n);
    std::vector<double> w(count);
    std::vector<uint8_t> st(count);
    for (int tb : {7, 14}) {   // a small tile (many stages, layout changes between them) and the full one
        const int stages = fh_register(n, ops.data(), n_ops, ch.data(), n_ch, cg, n_custom, tb);
        if (stages <= 0) { std::fprintf(stderr, "frame plan failed (%d) at tile bits %d\n", -stages, tb); return 3; }
        for (int reuse : {0, 1})
            if (fh_evolve(count, off.data(), site.data(), kk.data(), q.data(), reuse, states.data(), w.data(), st.data()) != 0) {
                std::fprintf(stderr, "frame evolve reported a guard violation\n");
                return 4;
            }
    }
    const int passes = dh_register(n, ops.data(), n_ops, ch.data(), n_ch, cg, n_custom);
    if (passes <= 0) { std::fprintf(stderr, "dense plan failed (%d)\n", -passes); return 5; }
    std::vector<float> out((size_t)2 << n);
    for (uint32_t a = 0; a < count; ++a) (void)dh_evolve(site.data() + off[a], kk.data() + off[a], off[a + 1] - off[a], out.data());
    if (dh_pad_errors() != 0) { std::fprintf(stderr, "dense padding amplitudes not zero\n"); return 6; }
    std::printf("host sanitizer run ok: %u sets, %d dense passes\n", count, passes);
    return 0;
}
