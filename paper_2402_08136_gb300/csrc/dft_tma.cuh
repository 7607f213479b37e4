// Shared pieces of the bulk-copy (TMA) Fourier-pass kernels (dft_tma.cu: one pass per launch;
// dft_merge.cu: two transforms per tile, and the pass with generated inputs): mbarrier and
// bulk-copy wrappers, the tile shape, the tensor-map encoder.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "dft_impl.cuh"

namespace qsim {
namespace dftt {


using dftk::bitrev;
using dftk::cmul;
using dftk::DftArgs;
using dftk::dft_regs;

constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
    return t;
}

// Bounded wait for the mbarrier phase of the given parity; false after about one second.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    unsigned long long t0 = 0;
    for (unsigned it = 0;; it++) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 63) == 0) {
            const unsigned long long t = global_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kWaitLimitNs) return false;
        }
    }
}

__device__ __forceinline__ void tma_load(unsigned dst, const CUtensorMap *map, int c1, int c4, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
        "l"(map), "r"(0), "r"(c1), "r"(0), "r"(0), "r"(c4), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_l2(const CUtensorMap *map, int c1, int c4) {
    asm volatile("cp.async.bulk.prefetch.tensor.5d.L2.global [%0, {%1, %2, %3, %4, %5}];\n" ::"l"(map), "r"(0), "r"(c1),
                 "r"(0), "r"(0), "r"(c4)
                 : "memory");
}

__device__ __forceinline__ void tma_store(const CUtensorMap *map, int c1, int c4, unsigned src) {
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];\n" ::"l"(map),
                 "r"(0), "r"(c1), "r"(0), "r"(0), "r"(c4), "r"(src)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

// The bulk stores issued by this thread have finished reading shared memory.
__device__ __forceinline__ void tma_store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// ... and are complete (visible in global memory).
__device__ __forceinline__ void tma_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

struct TmaExtra {
    int gap;        // qubits between the lanes and the field (f0 - 3)
    int above;      // qubits above the field in the tensor map (includes the ancilla for KIND 2)
    int inv_c4;     // KIND 2: coordinate offset of the upper half along the "above" dimension
    long long ntiles;  // tiles to transform (the lower half only for KIND 2)
    int pf;            // > 0: L2 prefetch of the tile pf loads ahead of the next one issued
};

// L lane qubits (the lowest qubits): rows of 2^L amplitudes, 64 (L = 3) or 128 bytes (L = 4)
template <int K, int L>
struct Shape {
    static constexpr int k1 = K / 2, k2 = K - k1;
    static constexpr int N1 = 1 << k1, N2 = 1 << k2, RR = N2 / N1;
    static constexpr int NL = 1 << L;
    static constexpr int threads = N1 * NL;
    static constexpr int tile = (1 << K) * NL;  // amplitudes
    static constexpr int min_blocks = threads >= 512 ? 1 : 512 / threads;  // 128 registers a thread
};

PFN_cuTensorMapEncodeTiled_v12000 encode_fn();
int num_sms();

}  // namespace dftt
}  // namespace qsim
