// Kernel-choice table and its autotuner.
//
// Every choice the library makes between equivalent kernels or launch shapes reads this table
// (one copy per state dtype): the Fourier/Walsh-Hadamard pass kernel (bulk-copy tiles or
// thread loads, and the latter's lane count and L2 prefetch distance), which dense gate widths
// run on the tensor cores (complex64), and the fusion width qsim_fuse(max_k = 0) uses.  The
// entries start at defaults measured on GB300; qsim_autotune times the alternatives on the
// caller's state buffer and writes the fastest; qsim_tune_set fixes an entry (to compare
// variants).  Nothing is read from the environment.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <chrono>
#include <cmath>
#include <random>
#include <vector>

#include "common.h"

namespace qsim {
namespace {

// [dtype][size class][key]: the pass-kernel entries depend on the state size (a 31-qubit state
// spans 8192 pages of 2 MiB, and passes on its top qubits meet other bounds than a 27-qubit one),
// so each entry is kept per size class: up to 24 qubits, 25..28, 29 and more
constexpr int kClasses = 3;
std::atomic<int> g_tune[2][kClasses][QSIM_TUNE_COUNT];
std::atomic<bool> g_tune_init{false};
std::mutex g_tune_mu;

int class_of(int n) { return n <= 24 ? 0 : (n <= 28 ? 1 : 2); }

int default_value(int slot, int key) {
    switch (key) {
        case QSIM_TUNE_DFT_TMA: return slot == 0 ? 4 : 0;  // complex64 only
        case QSIM_TUNE_DFT_LANES: return 0;                // 0: 128-byte lane runs
        case QSIM_TUNE_DFT_PREFETCH: return slot == 0 ? 0 : 1;  // bulk-copy passes: no L2 prefetch
        case QSIM_TUNE_DENSE_TC: return slot == 0 ? ((1 << 4) | (1 << 5) | (1 << 6) | (1 << 7)) : 0;
        case QSIM_TUNE_FUSE_WIDTH: return slot == 0 ? 4 : 2;
        case QSIM_TUNE_DFT_L2PROMO: return 2;
        case QSIM_TUNE_DFT_MERGE: return 1;  // two-transform merges measured slower on GB300
        case QSIM_TUNE_TUNED: return 0;
        default: return 0;
    }
}

void ensure_init() {
    if (g_tune_init.load(std::memory_order_acquire)) return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune_init.load(std::memory_order_relaxed)) return;
    for (int s = 0; s < 2; s++)
        for (int c = 0; c < kClasses; c++)
            for (int k = 0; k < QSIM_TUNE_COUNT; k++) g_tune[s][c][k].store(default_value(s, k));
    g_tune_init.store(true, std::memory_order_release);
}

int slot_of(int dtype) { return dtype == QSIM_C128 ? 1 : 0; }

bool valid_value(int key, int v) {
    switch (key) {
        case QSIM_TUNE_DFT_TMA: return v >= 0 && v <= 4;
        case QSIM_TUNE_DFT_L2PROMO: return v >= 0 && v <= 3;
        case QSIM_TUNE_DFT_MERGE: return v >= 0 && v <= 7;
        case QSIM_TUNE_DFT_LANES: return v >= 0 && v <= 8;
        case QSIM_TUNE_DFT_PREFETCH: return v >= 0 && v <= 4;
        case QSIM_TUNE_DENSE_TC: return v >= 0 && v < 256;
        case QSIM_TUNE_FUSE_WIDTH: return v >= 1 && v <= 6;
        case QSIM_TUNE_TUNED: return v == 0 || v == 1;
        default: return false;
    }
}

}  // namespace

int tune_get(int dtype, int key, int n) {
    ensure_init();
    return g_tune[slot_of(dtype)][class_of(n)][key].load(std::memory_order_relaxed);
}

}  // namespace qsim

using namespace qsim;

extern "C" int qsim_tune_get(int dtype, int key, int n_qubits, int *value) {
    return guarded([&] {
        QSIM_REQUIRE(value != nullptr, "NULL argument");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        QSIM_REQUIRE(key >= 0 && key < QSIM_TUNE_COUNT, "unknown tuning key");
        QSIM_REQUIRE(n_qubits >= 1 && n_qubits <= 34, "n_qubits must be in 1..34");
        *value = tune_get(dtype, key, n_qubits);
    });
}

extern "C" int qsim_tune_set(int dtype, int key, int n_qubits, int value) {
    return guarded([&] {
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        QSIM_REQUIRE(key >= 0 && key < QSIM_TUNE_COUNT, "unknown tuning key");
        QSIM_REQUIRE(n_qubits >= 0 && n_qubits <= 34, "n_qubits must be in 0..34");
        QSIM_REQUIRE(valid_value(key, value), "value out of range for this tuning key");
        ensure_init();
        for (int c = 0; c < kClasses; c++)
            if (n_qubits == 0 || c == class_of(n_qubits))
                g_tune[slot_of(dtype)][c][key].store(value, std::memory_order_relaxed);
    });
}

extern "C" int qsim_tune_reset(void) {
    return guarded([&] {
        ensure_init();
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (int s = 0; s < 2; s++)
            for (int c = 0; c < kClasses; c++)
                for (int k = 0; k < QSIM_TUNE_COUNT; k++) g_tune[s][c][k].store(default_value(s, k));
    });
}

namespace qsim {
namespace {

#define TUNE_CUDA_OK(call)                                                                          \
    do {                                                                                            \
        cudaError_t e__ = (call);                                                                   \
        if (e__ != cudaSuccess) throw Error(QSIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

// Average time of `reps` applications of circuit c to the state, CUDA events on `st`, after
// one warm-up application.
double time_apply(void *state, int n, int dtype, qsim_circuit *c, cudaStream_t st, int reps) {
    apply_ops(state, n, dtype, c, st);
    cudaEvent_t e0, e1;
    TUNE_CUDA_OK(cudaEventCreate(&e0));
    TUNE_CUDA_OK(cudaEventCreate(&e1));
    TUNE_CUDA_OK(cudaEventRecord(e0, st));
    for (int i = 0; i < reps; i++) apply_ops(state, n, dtype, c, st);
    TUNE_CUDA_OK(cudaEventRecord(e1, st));
    TUNE_CUDA_OK(cudaEventSynchronize(e1));
    float ms = 0.f;
    TUNE_CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (double)ms / reps;
}

std::vector<cd> haar(std::mt19937_64 &rng, int d) {
    // Ginibre matrix, Gram-Schmidt columns with the phase fix of Mezzadri (2007)
    std::normal_distribution<double> g(0.0, 1.0);
    std::vector<cd> Q((size_t)d * d);
    for (auto &z : Q) z = cd(g(rng), g(rng));
    for (int j = 0; j < d; j++) {
        for (int i = 0; i < j; i++) {
            cd dot = 0;
            for (int r = 0; r < d; r++) dot += std::conj(Q[(size_t)r * d + i]) * Q[(size_t)r * d + j];
            for (int r = 0; r < d; r++) Q[(size_t)r * d + j] -= dot * Q[(size_t)r * d + i];
        }
        double nn = 0;
        for (int r = 0; r < d; r++) nn += std::norm(Q[(size_t)r * d + j]);
        nn = std::sqrt(nn);
        for (int r = 0; r < d; r++) Q[(size_t)r * d + j] /= nn;
    }
    return Q;
}

struct CircuitHolder {
    qsim_circuit *c = nullptr;
    explicit CircuitHolder(int n) {
        if (qsim_circuit_create(n, &c) != QSIM_OK) throw Error(QSIM_ENOMEM, qsim_last_error());
    }
    ~CircuitHolder() { qsim_circuit_free(c); }
};

}  // namespace
}  // namespace qsim

extern "C" int qsim_autotune(void *state, int n_qubits, int dtype, void *stream, qsim_tune_report *out) {
    using namespace qsim;
    return guarded([&] {
        QSIM_REQUIRE(state != nullptr, "NULL state");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        QSIM_REQUIRE(n_qubits >= 20 && n_qubits <= 34, "autotune needs a state of 20..34 qubits");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        ensure_init();
        const int s = slot_of(dtype);
        const int n = n_qubits;
        std::atomic<int> *T = g_tune[s][class_of(n)];
        qsim_tune_report rep;
        std::memset(&rep, 0, sizeof(rep));
        std::mt19937_64 rng(2402);
        // 1. Fourier passes: the top field with a twiddle from the 10 qubits below it, the
        //    field right above qubit 5 without twiddle, and a Walsh-Hadamard pass
        {
            CircuitHolder ch(n);
            std::vector<int> top(10), bot(10), src(10);
            for (int j = 0; j < 10; j++) {
                top[j] = n - 10 + j;
                bot[j] = 6 + j;
                src[j] = n - 20 + j;
            }
            QSIM_REQUIRE(qsim_circuit_add_dft(ch.c, 10, top.data(), 10, src.data(), -1, 0) == QSIM_OK, qsim_last_error());
            QSIM_REQUIRE(qsim_circuit_add_dft(ch.c, 10, bot.data(), 0, nullptr, 1, 0) == QSIM_OK, qsim_last_error());
            QSIM_REQUIRE(qsim_circuit_add_walsh(ch.c, 10, top.data()) == QSIM_OK, qsim_last_error());
            struct Cand {
                int tma, lanes, pf;
            };
            std::vector<Cand> cands;
            if (dtype == QSIM_C64) {
                for (int pf : {1, 0, 2}) cands.push_back({4, 0, pf});
                for (int v : {3, 2, 1}) cands.push_back({v, 0, 1});
            }
            for (int lanes : {0, 3, 5})
                for (int pf : {0, 1}) cands.push_back({0, lanes, pf});
            double best = 1e300;
            Cand bc = cands.front();
            for (const Cand &c : cands) {
                T[QSIM_TUNE_DFT_TMA].store(c.tma);
                T[QSIM_TUNE_DFT_LANES].store(c.lanes);
                T[QSIM_TUNE_DFT_PREFETCH].store(c.pf);
                const double ms = time_apply(state, n, dtype, ch.c, st, 3);
                if (ms < best) best = ms, bc = c;
            }
            T[QSIM_TUNE_DFT_TMA].store(bc.tma);
            T[QSIM_TUNE_DFT_LANES].store(bc.lanes);
            T[QSIM_TUNE_DFT_PREFETCH].store(bc.pf);
            rep.dft_ms = best / 3.0;
        }
        // 2. dense gates of 3..6 targets (complex64): tensor cores or SIMT, per width (bit 7, the
        //    real 7-target tensor-core kernel, keeps its value)
        if (dtype == QSIM_C64) {
            int mask = T[QSIM_TUNE_DENSE_TC].load() & (1 << 7);
            for (int k = 3; k <= 6; k++) {
                CircuitHolder ch(n);
                for (int g = 0; g < 3; g++) {
                    std::vector<int> perm(n);
                    for (int q = 0; q < n; q++) perm[q] = q;
                    std::shuffle(perm.begin(), perm.end(), rng);
                    std::vector<cd> U = haar(rng, 1 << k);
                    std::vector<double> Ud(2 * U.size());
                    for (size_t i = 0; i < U.size(); i++) Ud[2 * i] = U[i].real(), Ud[2 * i + 1] = U[i].imag();
                    QSIM_REQUIRE(qsim_circuit_add_gate(ch.c, k, perm.data(), 0, nullptr, Ud.data()) == QSIM_OK,
                                 qsim_last_error());
                }
                double t[2];
                for (int use = 0; use < 2; use++) {
                    T[QSIM_TUNE_DENSE_TC].store(mask | (use ? (1 << k) : 0));
                    t[use] = time_apply(state, n, dtype, ch.c, st, 2);
                }
                if (t[1] < t[0]) mask |= 1 << k;
                rep.dense_ms[k - 3] = std::min(t[0], t[1]) / 3.0;
            }
            T[QSIM_TUNE_DENSE_TC].store(mask);
        }
        // 3. fusion width for gate-level circuits: a layer of random 1- and 2-qubit gates on the
        //    lowest 12 qubits (the shape of the phase estimation's gate-level QFT), fused at each
        //    width and applied
        {
            CircuitHolder ch(n);
            std::uniform_int_distribution<int> qd(0, 11);
            for (int g = 0; g < 48; g++) {
                const int k = (g % 3 == 0) ? 1 : 2;
                int t[2] = {qd(rng), qd(rng)};
                while (k == 2 && t[1] == t[0]) t[1] = qd(rng);
                std::vector<cd> U = haar(rng, 1 << k);
                std::vector<double> Ud(2 * U.size());
                for (size_t i = 0; i < U.size(); i++) Ud[2 * i] = U[i].real(), Ud[2 * i + 1] = U[i].imag();
                QSIM_REQUIRE(qsim_circuit_add_gate(ch.c, k, t, 0, nullptr, Ud.data()) == QSIM_OK, qsim_last_error());
            }
            double best = 1e300;
            int bk = 4;
            for (int k = 2; k <= 6; k++) {
                qsim_circuit *f = nullptr;
                QSIM_REQUIRE(qsim_fuse(ch.c, k, &f) == QSIM_OK, qsim_last_error());
                double ms = 0;
                try {
                    ms = time_apply(state, n, dtype, f, st, 2);
                } catch (...) {
                    qsim_circuit_free(f);
                    throw;
                }
                qsim_circuit_free(f);
                rep.fuse_ms[k - 2] = ms;
                if (ms < best) best = ms, bk = k;
            }
            T[QSIM_TUNE_FUSE_WIDTH].store(bk);
        }
        T[QSIM_TUNE_TUNED].store(1);
        for (int k = 0; k < QSIM_TUNE_COUNT; k++) rep.values[k] = T[k].load();
        rep.n_qubits = n;
        if (out) *out = rep;
    });
}
