// Device side of the GB300 HHL state-vector simulator: gate-application kernels, HHL state
// preparation and the FP64 readout reductions (sm_103a).
//
// The state is 2^n interleaved complex amplitudes (float2 for complex64, double2 for
// complex128); qubit q is bit q of the amplitude index.
//
// Dense gates (Sec. II-C "unitary evolution of the state", fused products of Fig. 4) run as a
// persistent tiled kernel: a CTA owns a tile of 2^T amplitudes spanned by the gate's target
// qubits plus the lowest non-control qubits, so that every tile is a union of contiguous runs
// of at least 16 amplitudes (coalesced, full 32-byte sectors).  The tile is staged in shared
// memory, the 2^k x 2^k matrix sits in shared memory for the CTA's lifetime, and each thread
// computes 16 output rows of one group column at a time, writing straight back to HBM.
// Specialised kernels handle phase (controlled-phase, e.g. the QFT's), diagonal, swap and the
// uniformly controlled RY of the eigenvalue inversion, touching only the amplitudes they change.
//
// The executor (apply_ops) can also run an HHL solve on the populated part of the state only
// (hhl_run): after the preparation every amplitude from 2^nb on is zero, so it tracks a live
// width, runs ops below it on the prefix, turns a pass onto the field right above it into a
// write-only broadcast (expand_kernel), and lets the inversion write the ancilla's upper half
// without reading it.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.h"

namespace qsim {

#define CUDA_OK(call)                                                                         \
    do {                                                                                      \
        cudaError_t e__ = (call);                                                             \
        if (e__ != cudaSuccess)                                                               \
            throw ::qsim::Error(QSIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

// Kernels launched by this library (every launch site reports here; a CUDA graph replay does
// not go through them).
static std::atomic<unsigned long long> g_launches{0};
static std::atomic<unsigned long long> g_family[QSIM_KERNEL_FAMILIES];
void note_launches(int k, int family) {
    g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed);
    if (family >= 0 && family < QSIM_KERNEL_FAMILIES)
        g_family[family].fetch_add((unsigned long long)k, std::memory_order_relaxed);
}

int occupancy_cached(const void *kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, size_t, int>, int> cache;
    int dev = 0;
    CUDA_OK(cudaGetDevice(&dev));
    const auto key = std::make_tuple(kernel, threads, smem, dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int per_sm = 0;
    CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = per_sm;
    return per_sm;
}

static void check_launch(const char *what, int launches, int family) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    note_launches(launches, family);
}

static int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return sms;
}

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// insert zero bits at the ascending positions pos[0..cnt-1]
__device__ __forceinline__ uint64_t insert_zeros(uint64_t x, const int *pos, int cnt) {
    for (int i = 0; i < cnt; i++) {
        const int p = pos[i];
        const uint64_t low = x & ((1ull << p) - 1ull);
        x = ((x >> p) << (p + 1)) | low;
    }
    return x;
}

// ---------------------------------------------------------------------------------------
// Dense k-qubit gate, tiled.
constexpr int kThreads = 256;
constexpr int kMaxFix = 40;

struct DenseArgs {
    void *psi;
    const void *U;        // 2^K x 2^K, stored transposed: Ut[c * D + r] = U[r][c]
    long long ntiles;
    unsigned long long cmask;  // control bits that must be 1
    int T;                // tile bits
    int L0;               // tile bits 0..L0-1 are global qubits 0..L0-1
    int nh;               // tile bits L0..T-1 map to global positions hpos[0..nh-1]
    int hpos[16];
    int nfix;             // ascending insertion positions (tile qubits above L0, controls)
    int fix[kMaxFix];
    int tloc[8];          // tile-local bit of target b
};

template <typename R, int K, bool USMEM, bool REALU>
__global__ void __launch_bounds__(kThreads) dense_tile_kernel(const DenseArgs a) {
    using V = typename C2<R>::T;
    constexpr int D = 1 << K;
    constexpr int RPT = D < 16 ? D : 16;  // output rows per thread
    constexpr int RG = D / RPT;           // row groups
    constexpr int WPG = (kThreads / 32) / RG;  // warps per row group
    constexpr int CSTRIDE = 32 * WPG;     // column stride
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = a.T;
    const int tile_amps = 1 << T;
    const int G = tile_amps >> K;  // groups (columns) per tile
    V *tile = reinterpret_cast<V *>(smem_raw);
    // U in shared memory (USMEM): D*D complex, or D*D reals when U is real (REALU)
    constexpr int UBYTES = USMEM ? D * D * (REALU ? (int)sizeof(R) : (int)sizeof(V)) : 0;
    unsigned char *Usb = reinterpret_cast<unsigned char *>(tile + tile_amps);
    V *Us = reinterpret_cast<V *>(Usb);
    R *Usr = reinterpret_cast<R *>(Usb);
    int *toff = reinterpret_cast<int *>(Usb + UBYTES);  // D entries
    long long *hoff = reinterpret_cast<long long *>(toff + ((D + 1) & ~1));  // 2^nh entries

    const int tid = threadIdx.x;
    const V *Ug = reinterpret_cast<const V *>(a.U);
    if (USMEM)
        for (int i = tid; i < D * D; i += kThreads) {
            if (REALU) Usr[i] = Ug[i].x;
            else Us[i] = Ug[i];
        }
    for (int c = tid; c < D; c += kThreads) {
        int o = 0;
        for (int b = 0; b < K; b++)
            if ((c >> b) & 1) o |= 1 << a.tloc[b];
        toff[c] = o;
    }
    const int nhv = 1 << a.nh;
    for (int h = tid; h < nhv; h += kThreads) {
        long long o = 0;
        for (int i = 0; i < a.nh; i++)
            if ((h >> i) & 1) o |= 1ll << a.hpos[i];
        hoff[h] = o;
    }
    // tile-local index of the first amplitude of each group: insert zeros at target bits
    int tsorted[K];
    for (int b = 0; b < K; b++) tsorted[b] = a.tloc[b];
    for (int i = 1; i < K; i++) {
        int v = tsorted[i], j = i - 1;
        while (j >= 0 && tsorted[j] > v) { tsorted[j + 1] = tsorted[j]; j--; }
        tsorted[j + 1] = v;
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    const int rg = warp % RG;
    const int col0 = (warp / RG) * 32 + lane;
    const int lomask = (1 << a.L0) - 1;
    V *psi = reinterpret_cast<V *>(a.psi);

    for (long long tix = blockIdx.x; tix < a.ntiles; tix += gridDim.x) {
        const unsigned long long base =
            insert_zeros((unsigned long long)tix << a.L0, a.fix, a.nfix) | a.cmask;
        for (int l = tid; l < tile_amps; l += kThreads)
            tile[l] = psi[base + hoff[l >> a.L0] + (l & lomask)];
        __syncthreads();
        for (int g = col0; g < G; g += CSTRIDE) {
            int gl = g;
            for (int b = 0; b < K; b++) {
                const int p = tsorted[b];
                gl = ((gl >> p) << (p + 1)) | (gl & ((1 << p) - 1));
            }
            V acc[RPT];
#pragma unroll
            for (int r = 0; r < RPT; r++) acc[r] = V{0, 0};
            for (int c = 0; c < D; c++) {
                const V x = tile[gl + toff[c]];
                if (REALU) {  // real U: two multiply-adds per entry
                    const R *ucr = Usr + c * D + rg * RPT;
                    const V *ucg = Ug + c * D + rg * RPT;
#pragma unroll
                    for (int r = 0; r < RPT; r++) {
                        const R u = USMEM ? ucr[r] : ucg[r].x;
                        acc[r].x = fma(u, x.x, acc[r].x);
                        acc[r].y = fma(u, x.y, acc[r].y);
                    }
                } else {
                    const V *uc = (USMEM ? Us : Ug) + c * D + rg * RPT;
#pragma unroll
                    for (int r = 0; r < RPT; r++) {
                        const V u = uc[r];
                        acc[r].x = fma(u.x, x.x, acc[r].x);
                        acc[r].x = fma(-u.y, x.y, acc[r].x);
                        acc[r].y = fma(u.x, x.y, acc[r].y);
                        acc[r].y = fma(u.y, x.x, acc[r].y);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < RPT; r++) {
                const int l = gl + toff[rg * RPT + r];
                psi[base + hoff[l >> a.L0] + (l & lomask)] = acc[r];
            }
        }
        __syncthreads();
    }
}

// Same operation with a multi-stage cp.async pipeline: while the CTA computes tile i from
// shared memory, the copies of tiles i+1 .. i+NS-1 are in flight (16-byte cp.async chunks, each
// chunk contiguous in HBM because the tile always contains qubit 0).  Results are stored from
// registers straight to HBM.  Used whenever qubit 0 is a tile qubit (always for complex128).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int kStages = 3;

template <typename R, int K, bool USMEM, bool REALU>
__global__ void __launch_bounds__(kThreads) dense_pipe_kernel(const DenseArgs a) {
    using V = typename C2<R>::T;
    constexpr int D = 1 << K;
    constexpr int RPT = D < 16 ? D : 16;
    constexpr int RG = D / RPT;
    constexpr int WPG = (kThreads / 32) / RG;
    constexpr int CSTRIDE = 32 * WPG;
    constexpr int EPC = 16 / sizeof(V);  // amplitudes per 16-byte chunk
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = a.T;
    const int tile_amps = 1 << T;
    const int G = tile_amps >> K;
    V *stages = reinterpret_cast<V *>(smem_raw);
    constexpr int UBYTES = USMEM ? D * D * (REALU ? (int)sizeof(R) : (int)sizeof(V)) : 0;
    unsigned char *Usb = reinterpret_cast<unsigned char *>(stages + kStages * tile_amps);
    V *Us = reinterpret_cast<V *>(Usb);
    R *Usr = reinterpret_cast<R *>(Usb);
    int *toff = reinterpret_cast<int *>(Usb + UBYTES);
    long long *hoff = reinterpret_cast<long long *>(toff + ((D + 1) & ~1));

    const int tid = threadIdx.x;
    const V *Ug = reinterpret_cast<const V *>(a.U);
    if (USMEM)
        for (int i = tid; i < D * D; i += kThreads) {
            if (REALU) Usr[i] = Ug[i].x;
            else Us[i] = Ug[i];
        }
    for (int c = tid; c < D; c += kThreads) {
        int o = 0;
        for (int b = 0; b < K; b++)
            if ((c >> b) & 1) o |= 1 << a.tloc[b];
        toff[c] = o;
    }
    const int nhv = 1 << a.nh;
    for (int h = tid; h < nhv; h += kThreads) {
        long long o = 0;
        for (int i = 0; i < a.nh; i++)
            if ((h >> i) & 1) o |= 1ll << a.hpos[i];
        hoff[h] = o;
    }
    int tsorted[K];
    for (int b = 0; b < K; b++) tsorted[b] = a.tloc[b];
    for (int i = 1; i < K; i++) {
        int v = tsorted[i], j = i - 1;
        while (j >= 0 && tsorted[j] > v) { tsorted[j + 1] = tsorted[j]; j--; }
        tsorted[j + 1] = v;
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    const int rg = warp % RG;
    const int col0 = (warp / RG) * 32 + lane;
    const int lomask = (1 << a.L0) - 1;
    V *psi = reinterpret_cast<V *>(a.psi);
    const long long first = blockIdx.x, stride = gridDim.x;
    const long long ntl = first < a.ntiles ? (a.ntiles - first + stride - 1) / stride : 0;
    const int nchunk = tile_amps / EPC;

    auto tile_base = [&](long long i) -> unsigned long long {
        return insert_zeros((unsigned long long)(first + i * stride) << a.L0, a.fix, a.nfix) | a.cmask;
    };
    auto issue = [&](long long i) {
        const unsigned long long base = tile_base(i);
        V *dst = stages + (int)(i % kStages) * tile_amps;
        for (int ch = tid; ch < nchunk; ch += kThreads) {
            const int l0 = ch * EPC;
            cp_async16(dst + l0, psi + base + hoff[l0 >> a.L0] + (l0 & lomask));
        }
    };

    for (int p = 0; p < kStages - 1; p++) {
        if (p < ntl) issue(p);
        cp_async_commit();
    }
    for (long long i = 0; i < ntl; i++) {
        cp_async_wait<kStages - 2>();
        __syncthreads();  // tile i visible to all; every thread is done with tile i-1's stage
        if (i + kStages - 1 < ntl) issue(i + kStages - 1);
        cp_async_commit();
        const V *tile = stages + (int)(i % kStages) * tile_amps;
        const unsigned long long base = tile_base(i);
        for (int g = col0; g < G; g += CSTRIDE) {
            int gl = g;
#pragma unroll
            for (int b = 0; b < K; b++) {
                const int p = tsorted[b];
                gl = ((gl >> p) << (p + 1)) | (gl & ((1 << p) - 1));
            }
            V acc[RPT];
#pragma unroll
            for (int r = 0; r < RPT; r++) acc[r] = V{0, 0};
            for (int c = 0; c < D; c++) {
                const V x = tile[gl + toff[c]];
                if (REALU) {  // real U: two multiply-adds per entry
                    const R *ucr = Usr + c * D + rg * RPT;
                    const V *ucg = Ug + c * D + rg * RPT;
#pragma unroll
                    for (int r = 0; r < RPT; r++) {
                        const R u = USMEM ? ucr[r] : ucg[r].x;
                        acc[r].x = fma(u, x.x, acc[r].x);
                        acc[r].y = fma(u, x.y, acc[r].y);
                    }
                } else {
                    const V *uc = (USMEM ? Us : Ug) + c * D + rg * RPT;
#pragma unroll
                    for (int r = 0; r < RPT; r++) {
                        const V u = uc[r];
                        acc[r].x = fma(u.x, x.x, acc[r].x);
                        acc[r].x = fma(-u.y, x.y, acc[r].x);
                        acc[r].y = fma(u.x, x.y, acc[r].y);
                        acc[r].y = fma(u.y, x.x, acc[r].y);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < RPT; r++) {
                const int l = gl + toff[rg * RPT + r];
                psi[base + hoff[l >> a.L0] + (l & lomask)] = acc[r];
            }
        }
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------------------
// Phase on the all-ones pattern of `mask` qubits: psi[i] *= ph for i with (i & mask) == mask.
struct PhaseArgs {
    void *psi;
    long long count;  // 2^(n - nfix)
    unsigned long long mask;
    int nfix;
    int fix[kMaxFix];
    double ph_re, ph_im;
};

template <typename R>
__global__ void phase_kernel(const PhaseArgs a) {
    using V = typename C2<R>::T;
    V *psi = reinterpret_cast<V *>(a.psi);
    const V ph{(R)a.ph_re, (R)a.ph_im};
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < a.count;
         g += (long long)gridDim.x * blockDim.x) {
        const unsigned long long i = insert_zeros((unsigned long long)g, a.fix, a.nfix) | a.mask;
        psi[i] = cmul(psi[i], ph);
    }
}

// Diagonal on k targets (entries d[pattern]) where the controls are 1.
struct DiagArgs {
    void *psi;
    const void *d;
    long long count;
    unsigned long long cmask;
    int nfix;
    int fix[kMaxFix];
    int k;
    int targets[8];
};

template <typename R>
__global__ void diag_kernel(const DiagArgs a) {
    using V = typename C2<R>::T;
    V *psi = reinterpret_cast<V *>(a.psi);
    const V *d = reinterpret_cast<const V *>(a.d);
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < a.count;
         g += (long long)gridDim.x * blockDim.x) {
        const unsigned long long i = insert_zeros((unsigned long long)g, a.fix, a.nfix) | a.cmask;
        int p = 0;
        for (int b = 0; b < a.k; b++) p |= (int)((i >> a.targets[b]) & 1ull) << b;
        psi[i] = cmul(psi[i], d[p]);
    }
}

// Swap qubits qa, qb where the controls are 1.
struct SwapArgs {
    void *psi;
    long long count;
    unsigned long long cmask;
    unsigned long long ma, mb;
    int nfix;
    int fix[kMaxFix];
};

template <typename R>
__global__ void swap_kernel(const SwapArgs a) {
    using V = typename C2<R>::T;
    V *psi = reinterpret_cast<V *>(a.psi);
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < a.count;
         g += (long long)gridDim.x * blockDim.x) {
        const unsigned long long i = insert_zeros((unsigned long long)g, a.fix, a.nfix) | a.cmask;
        const V x = psi[i | a.ma], y = psi[i | a.mb];
        psi[i | a.ma] = y;
        psi[i | a.mb] = x;
    }
}

// Uniformly controlled RY on `target`: (psi0, psi1) <- [[c, -s], [s, c]] (psi0, psi1) with
// (c, s) = cs[v], v = value of the control register at the pair's index.
struct UcryArgs {
    void *psi;
    const void *cs;  // 2^nc (cos theta/2, sin theta/2) pairs, in the state's real type
    long long count;  // 2^(n-1)
    int target;
    int nc;
    int contiguous;  // controls are qubits c0 .. c0+nc-1 in order
    int c0;
    int src_zero;    // the target-1 half is known to be zero: written, not read
    int ctrl[32];
};

template <typename R>
__global__ void ucry_kernel(const UcryArgs a) {
    using V = typename C2<R>::T;
    V *psi = reinterpret_cast<V *>(a.psi);
    const V *cs = reinterpret_cast<const V *>(a.cs);
    const unsigned long long tb = 1ull << a.target;
    const unsigned long long vmask = (1ull << a.nc) - 1ull;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < a.count;
         g += (long long)gridDim.x * blockDim.x) {
        const unsigned long long i0 = (((unsigned long long)g >> a.target) << (a.target + 1)) |
                                      ((unsigned long long)g & (tb - 1ull));
        unsigned long long v;
        if (a.contiguous) {
            v = (i0 >> a.c0) & vmask;
        } else {
            v = 0;
            for (int j = 0; j < a.nc; j++) v |= ((i0 >> a.ctrl[j]) & 1ull) << j;
        }
        const V t = cs[v];
        const V x0 = psi[i0], x1 = a.src_zero ? V{0, 0} : psi[i0 | tb];
        V y0, y1;
        y0.x = t.x * x0.x - t.y * x1.x;
        y0.y = t.x * x0.y - t.y * x1.y;
        y1.x = t.y * x0.x + t.x * x1.x;
        y1.y = t.y * x0.y + t.x * x1.y;
        psi[i0] = y0;
        psi[i0 | tb] = y1;
    }
}

// Structured phase estimation: in the data register's eigenbasis, all m controlled evolutions
// together multiply amplitude (c, d) by exp(i s lam_d t c) (c = clock value, d = data index).
// The phase is the product of two table entries, lo[(c mod 2^h) D + d] * hi[(c >> h) D + d].
struct QpeArgs {
    void *psi;
    const void *lo, *hi;
    long long N;
    int nb, m, h;
};

template <typename R>
__global__ void qpe_phase_kernel(const QpeArgs a) {
    using V = typename C2<R>::T;
    V *psi = reinterpret_cast<V *>(a.psi);
    const V *lo = reinterpret_cast<const V *>(a.lo);
    const V *hi = reinterpret_cast<const V *>(a.hi);
    const unsigned long long dmask = (1ull << a.nb) - 1ull, cmask = (1ull << a.m) - 1ull;
    const unsigned long long hmask = (1ull << a.h) - 1ull;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.N;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long d = (unsigned long long)i & dmask;
        const unsigned long long c = ((unsigned long long)i >> a.nb) & cmask;
        const V p = cmul(lo[((c & hmask) << a.nb) + d], hi[((c >> a.h) << a.nb) + d]);
        psi[i] = cmul(psi[i], p);
    }
}

// A Fourier or Walsh-Hadamard pass (no twiddle after the transform) on the field w .. w+K-1 of
// a state that is zero at every index >= 2^w: only field value 0 is populated, and column 0 of
// the transform is 2^(-K/2) for every output digit, so out[y 2^w + l] = 2^(-K/2) in[l] (times a
// fused structured phase, on the input or the output index).  col0 = 0: each thread writes the
// outputs y = y0 .. y0+run-1 (y >= 1) of one l from the untouched column y = 0; along y the
// output phase is a geometric sequence when the field lies inside the clock register (qrec,
// complex64: refreshed from the tables every 8 terms).
// col0 = 1 then rescales the column y = 0 in place.
struct ExpandArgs {
    void *psi;
    const void *qlo, *qhi;  // structured phase tables (qmode 1: input index l, 2: output index)
    long long lowN;         // 2^w
    long long count;        // threads' work items this launch
    double scale;
    int w, K, run, col0, qmode, qnb, qm, qh, qrec;
};

template <typename R>
__global__ void expand_kernel(const ExpandArgs a) {
    using V = typename C2<R>::T;
    V *psi = reinterpret_cast<V *>(a.psi);
    const V *lo = reinterpret_cast<const V *>(a.qlo);
    const V *hi = reinterpret_cast<const V *>(a.qhi);
    const unsigned long long dmask = (1ull << a.qnb) - 1ull, cmask = (1ull << a.qm) - 1ull;
    const unsigned long long hmask = (1ull << a.qh) - 1ull;
    auto phase_cd = [&](unsigned long long c, unsigned long long d) -> V {
        return cmul(lo[((c & hmask) << a.qnb) + d], hi[((c >> a.qh) << a.qnb) + d]);
    };
    auto phase = [&](unsigned long long i) -> V { return phase_cd((i >> a.qnb) & cmask, i & dmask); };
    const R sc = (R)a.scale;
    const unsigned long long ymax = 1ull << a.K;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < a.count;
         g += (long long)gridDim.x * blockDim.x) {
        const unsigned long long l = (unsigned long long)g & (unsigned long long)(a.lowN - 1);
        V z = psi[l];
        if (a.qmode == 1) z = cmul(z, phase(l));
        z.x *= sc;
        z.y *= sc;
        if (a.col0) {
            if (a.qmode == 2) z = cmul(z, phase(l));
            psi[l] = z;
            continue;
        }
        const unsigned long long y0 = 1ull + ((unsigned long long)g >> a.w) * (unsigned long long)a.run;
        const bool seq = a.qmode == 2 && a.qrec;
        V P{1, 0}, Q{1, 0};
        if (seq) Q = phase_cd(1ull << (a.w - a.qnb), l & dmask);
        for (int j = 0; j < a.run; j++) {
            const unsigned long long y = y0 + (unsigned long long)j;
            if (y >= ymax) break;
            const unsigned long long idx = (y << a.w) | l;
            V o = z;
            if (seq) {
                if ((j & 7) == 0) P = phase(idx);  // refreshed from the tables every 8 terms
                o = cmul(z, P);
                P = cmul(P, Q);
            } else if (a.qmode == 2) {
                o = cmul(z, phase(idx));
            }
            psi[idx] = o;
        }
    }
}

// HHL eigenvalue inversion: for the pair of amplitudes that differ in the ancilla,
// r = clamp(Cs / k, -1, 1) with k the clock value (two's complement for an indefinite A; r = 0
// for k = 0), and
// (psi0, psi1) <- [[sqrt((1 - |r|)(1 + |r|)), -r], [r, sqrt((1 - |r|)(1 + |r|))]] (psi0, psi1).
// The clock register may sit in any bit order made of contiguous runs of qubits (the order a
// Fourier-pass inverse QFT leaves it in): run s holds bits dst[s] .. dst[s] + w[s] - 1 of k
// on qubits src[s] .. src[s] + w[s] - 1.
constexpr int kMaxSeg = 8;
struct InvertArgs {
    void *psi;
    long long count;  // 2^(n-1)
    double Cs;
    int target, nc;
    int twos;         // clock register read as two's complement (indefinite A)
    int src_zero;     // the target-1 half is known to be zero: written, not read
    int nseg;
    int seg_src[kMaxSeg], seg_w[kMaxSeg], seg_dst[kMaxSeg];
};

template <typename R>
__global__ void hhl_invert_kernel(const InvertArgs a) {
    using V = typename C2<R>::T;
    V *psi = reinterpret_cast<V *>(a.psi);
    const unsigned long long tb = 1ull << a.target;
    const R Cs = (R)a.Cs;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < a.count;
         g += (long long)gridDim.x * blockDim.x) {
        const unsigned long long i0 = (((unsigned long long)g >> a.target) << (a.target + 1)) |
                                      ((unsigned long long)g & (tb - 1ull));
        unsigned long long k = 0;
        for (int sg = 0; sg < a.nseg; sg++)
            k |= ((i0 >> a.seg_src[sg]) & ((1ull << a.seg_w[sg]) - 1ull)) << a.seg_dst[sg];
        R s = 0, c = 1;
        if (k) {
            const long long ks = (a.twos && (k >> (a.nc - 1))) ? (long long)k - (1ll << a.nc) : (long long)k;
            s = Cs / (R)ks;
            if (s > (R)1) s = (R)1;
            if (s < (R)-1) s = (R)-1;
            const R as = s < 0 ? -s : s;
            c = sqrt(((R)1 - as) * ((R)1 + as));
        }
        const V x0 = psi[i0], x1 = a.src_zero ? V{0, 0} : psi[i0 | tb];
        V y0, y1;
        y0.x = c * x0.x - s * x1.x;
        y0.y = c * x0.y - s * x1.y;
        y1.x = s * x0.x + c * x1.x;
        y1.y = s * x0.y + c * x1.y;
        psi[i0] = y0;
        psi[i0 | tb] = y1;
    }
}

// ---------------------------------------------------------------------------------------
// HHL state preparation: psi = 0 except the first D amplitudes = b.
constexpr int kMaxParamB = 256;
struct PrepArgs {
    void *psi;
    long long N;
    int D;
    double b[2 * kMaxParamB];
};

// After the state has been zeroed (cudaMemsetAsync): write the first min(D, 256) amplitudes.
template <typename R>
__global__ void prep_kernel(const PrepArgs a) {
    using V = typename C2<R>::T;
    V *psi = reinterpret_cast<V *>(a.psi);
    const int i = threadIdx.x;
    if (i < a.D && i < kMaxParamB && i < a.N) psi[i] = V{(R)a.b[2 * i], (R)a.b[2 * i + 1]};
}

// ---------------------------------------------------------------------------------------
// Readout reductions in FP64.  Block b of `nblk` sums |psi_i|^2 over its contiguous chunk in a
// fixed order (per-thread strided sums, then a fixed shuffle/shared-memory tree); the final
// single-block kernel adds the partials in index order.  The result therefore depends only on
// the state and n, never on what else runs on the GPU.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// Partial sums of |psi_i|^2 over contiguous chunks.  complex128: FP64 products and sums.
// complex64: the FP64 pipe (1/64 of the FP32 rate on this GPU) would bound the pass, so each
// square x^2 is formed exactly as an FP32 pair (p, e) with p = fl(x^2), e = fma(x, x, -p)
// (Dekker's product), 16 amplitudes per thread are summed in double-single arithmetic (Knuth's
// two-sum on the high part, ~48-bit result), and each group sum enters the FP64 accumulator;
// from there on the reduction is FP64 as for complex128.  The intrinsics keep the compiler from
// contracting the error-free steps into fused operations.
__device__ __forceinline__ void ds_add_square(float x, float &hi, float &lo) {
    const float p = __fmul_rn(x, x);
    const float e = __fmaf_rn(x, x, -p);
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

constexpr int kNormGroup = 16;

template <typename R>
__global__ void norm_partials_kernel(const void *state, long long chunk, double *partials, double *count = nullptr) {
    using V = typename C2<R>::T;
    __shared__ double sh[32];
    const V *psi = reinterpret_cast<const V *>(state) + (long long)blockIdx.x * chunk;
    double s = 0.0;
    if (sizeof(R) == 8) {
        for (long long i = threadIdx.x; i < chunk; i += blockDim.x) {
            const V z = psi[i];
            s = fma((double)z.x, (double)z.x, s);
            s = fma((double)z.y, (double)z.y, s);
        }
    } else {
        const long long span = (long long)blockDim.x * kNormGroup;
        for (long long i0 = threadIdx.x; i0 < chunk; i0 += span) {
            V z[kNormGroup];
#pragma unroll
            for (int g = 0; g < kNormGroup; g++) {
                const long long i = i0 + (long long)g * blockDim.x;
                z[g] = i < chunk ? psi[i] : V{0, 0};
            }
            float hi = 0.0f, lo = 0.0f;
#pragma unroll
            for (int g = 0; g < kNormGroup; g++) {
                ds_add_square((float)z[g].x, hi, lo);
                ds_add_square((float)z[g].y, hi, lo);
            }
            s += (double)hi + (double)lo;
        }
    }
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
    if (count && blockIdx.x == 0 && threadIdx.x == 0) *count = (double)gridDim.x;
}

// The same sums from a readout-sums buffer: buf[0] = P, the count of partial sums, then P
// partials whose first half covers the state's lower half (ancilla = 0) and second half its
// upper half, each half in a fixed order (written by the last pass of a run, or by
// norm_partials_kernel).
template <typename R>
__global__ void norm_final_buf_kernel(const double *buf, const void *state, long long off, int len, double *out);

// out[0] = sum of all partials, out[1] = sum of the upper half (ancilla = 1),
// out[2] = sum over the slice psi[off .. off + len) (ancilla = 1, clock = 0).
template <typename R>
__device__ void norm_final_body(const double *partials, int nblk, const void *state, long long off, int len,
                                double *out) {
    using V = typename C2<R>::T;
    __shared__ double sh[32];
    double lo = 0.0, hi = 0.0, sl = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        if (i < nblk / 2) lo += partials[i];
        else hi += partials[i];
    }
    const V *psi = reinterpret_cast<const V *>(state) + off;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const V z = psi[i];
        const double re = (double)z.x, im = (double)z.y;
        sl = fma(re, re, sl);
        sl = fma(im, im, sl);
    }
    const double tlo = block_sum(lo, sh);
    const double thi = block_sum(hi, sh);
    const double tsl = block_sum(sl, sh);
    if (threadIdx.x == 0) {
        out[0] = tlo + thi;
        out[1] = thi;
        out[2] = tsl;
    }
}

template <typename R>
__global__ void norm_final_kernel(const double *partials, int nblk, const void *state, long long off, int len,
                                  double *out) {
    norm_final_body<R>(partials, nblk, state, off, len, out);
}

template <typename R>
__global__ void norm_final_buf_kernel(const double *buf, const void *state, long long off, int len, double *out) {
    norm_final_body<R>(buf + 1, (int)buf[0], state, off, len, out);
}

// ---------------------------------------------------------------------------------------
// Host side.
namespace {

size_t real_size(int dtype) { return dtype == QSIM_C128 ? 8 : 4; }

void put_complex(std::vector<unsigned char> &blob, int dtype, const cd &z) {
    if (dtype == QSIM_C128) {
        double v[2] = {z.real(), z.imag()};
        blob.insert(blob.end(), (unsigned char *)v, (unsigned char *)v + 16);
    } else {
        float v[2] = {(float)z.real(), (float)z.imag()};
        blob.insert(blob.end(), (unsigned char *)v, (unsigned char *)v + 8);
    }
}

void align_blob(std::vector<unsigned char> &blob) {
    while (blob.size() % 256) blob.push_back(0);
}

std::vector<int> sorted_copy(std::vector<int> v) {
    std::sort(v.begin(), v.end());
    return v;
}

void fill_fix(int *dst, int &cnt, const std::vector<int> &pos) {
    QSIM_REQUIRE((int)pos.size() <= kMaxFix, "too many fixed qubits");
    cnt = (int)pos.size();
    for (int i = 0; i < cnt; i++) dst[i] = pos[i];
}

unsigned long long mask_of(const std::vector<int> &q) {
    unsigned long long m = 0;
    for (int x : q) m |= 1ull << x;
    return m;
}

int grid_for(long long work, int per_block) {
    long long blocks = (work + per_block - 1) / per_block;
    const long long cap = (long long)num_sms() * 16;
    return (int)std::max(1ll, std::min(blocks, cap));
}

int tile_bits(int dtype) { return dtype == QSIM_C128 ? 11 : 11; }

template <typename R, int K, bool USMEM, bool REALU>
void launch_dense_t(const DenseArgs &a, size_t smem, bool pipe, cudaStream_t st) {
    auto kern = pipe ? dense_pipe_kernel<R, K, USMEM, REALU> : dense_tile_kernel<R, K, USMEM, REALU>;
    static bool attr[2] = {false, false};
    if (!attr[pipe]) {
        CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr[pipe] = true;
    }
    int per_sm = 0;
    per_sm = occupancy_cached(reinterpret_cast<const void *>(kern), kThreads, smem);
    QSIM_REQUIRE(per_sm > 0, "dense kernel does not fit on an SM");
    const long long grid = std::min<long long>(a.ntiles, (long long)num_sms() * per_sm);
    kern<<<(int)grid, kThreads, smem, st>>>(a);
    check_launch("dense_tile_kernel", 1, QSIM_KERNEL_DENSE_SIMT);
}

template <typename R>
void launch_dense(const DenseArgs &a, int K, bool real_u, size_t smem_base, cudaStream_t st) {
    const size_t D = (size_t)1 << K;
    const size_t vb = 2 * sizeof(R);
    const size_t ubytes = D * D * (real_u ? sizeof(R) : vb);
    const size_t tile_bytes = ((size_t)1 << a.T) * vb;
    // the pipelined kernel needs qubit 0 in the tile (16-byte chunks contiguous in HBM)
    const bool pipe = a.L0 >= 1 && smem_base + (kStages - 1) * tile_bytes <= 200 * 1024;
    const size_t base = smem_base + (pipe ? (kStages - 1) * tile_bytes : 0);
    const bool usmem = base + ubytes <= 200 * 1024;
    const size_t smem = base + (usmem ? ubytes : 0);
    switch (K) {
#define QSIM_K(k)                                                                \
    case k:                                                                      \
        if (real_u) {                                                            \
            if (usmem) launch_dense_t<R, k, true, true>(a, smem, pipe, st);      \
            else launch_dense_t<R, k, false, true>(a, smem, pipe, st);           \
        } else {                                                                 \
            if (usmem) launch_dense_t<R, k, true, false>(a, smem, pipe, st);     \
            else launch_dense_t<R, k, false, false>(a, smem, pipe, st);          \
        }                                                                        \
        break;
        QSIM_K(1) QSIM_K(2) QSIM_K(3) QSIM_K(4) QSIM_K(5) QSIM_K(6) QSIM_K(7)
#undef QSIM_K
        default:
            throw Error(QSIM_EINVAL, "dense gate wider than 7 qubits");
    }
}

void run_dense(void *state, int n, int dtype, const Op &op, const void *Udev, cudaStream_t st) {
    const int K = (int)op.targets.size();
    const std::vector<int> &ctl = op.controls;
    const unsigned long long cm = mask_of(ctl);
    const unsigned long long tm = mask_of(op.targets);
    const int avail = n - (int)ctl.size();
    // a 7-target real gate on complex64: a wider tile gives each warp 32 groups (the real U
    // leaves room for it in shared memory)
    const int T = std::min(tile_bits(dtype) + (K == 7 && op.real_u && dtype == QSIM_C64 ? 1 : 0), avail);
    // tile qubits: the targets plus the lowest non-control qubits
    std::vector<int> tile(op.targets.begin(), op.targets.end());
    for (int q = 0; q < n && (int)tile.size() < T; q++)
        if (!((cm >> q) & 1ull) && !((tm >> q) & 1ull)) tile.push_back(q);
    std::vector<int> ts = sorted_copy(tile);
    DenseArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    a.U = Udev;
    a.T = (int)ts.size();
    a.L0 = 0;
    while (a.L0 < a.T && ts[a.L0] == a.L0) a.L0++;
    a.nh = a.T - a.L0;
    QSIM_REQUIRE(a.nh <= 16, "tile layout");
    for (int i = 0; i < a.nh; i++) a.hpos[i] = ts[a.L0 + i];
    std::vector<int> fix;
    for (int i = a.L0; i < a.T; i++) fix.push_back(ts[i]);
    for (int q : ctl) fix.push_back(q);
    fix = sorted_copy(fix);
    fill_fix(a.fix, a.nfix, fix);
    a.cmask = cm;
    a.ntiles = 1ll << (n - a.T - (int)ctl.size());
    for (int b = 0; b < K; b++)
        a.tloc[b] = (int)(std::find(ts.begin(), ts.end(), op.targets[b]) - ts.begin());
    const size_t vb = 2 * real_size(dtype);
    const size_t D = (size_t)1 << K;
    const size_t smem_base = ((size_t)1 << a.T) * vb + ((D + 1) & ~(size_t)1) * 4 +
                             ((size_t)1 << a.nh) * 8;
    if (dtype == QSIM_C128) launch_dense<double>(a, K, op.real_u, smem_base, st);
    else launch_dense<float>(a, K, op.real_u, smem_base, st);
}

void run_phase(void *state, int n, int dtype, const Op &op, cudaStream_t st) {
    PhaseArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    std::vector<int> q = sorted_copy(op.targets);
    fill_fix(a.fix, a.nfix, q);
    a.mask = mask_of(q);
    a.count = 1ll << (n - (int)q.size());
    a.ph_re = op.phase.real();
    a.ph_im = op.phase.imag();
    const int grid = grid_for(a.count, 256);
    if (dtype == QSIM_C128) phase_kernel<double><<<grid, 256, 0, st>>>(a);
    else phase_kernel<float><<<grid, 256, 0, st>>>(a);
    check_launch("phase_kernel", 1, QSIM_KERNEL_ELEMENTWISE);
}

void run_diag(void *state, int n, int dtype, const Op &op, const void *ddev, cudaStream_t st) {
    DiagArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    a.d = ddev;
    std::vector<int> c = sorted_copy(op.controls);
    fill_fix(a.fix, a.nfix, c);
    a.cmask = mask_of(c);
    a.count = 1ll << (n - (int)c.size());
    a.k = (int)op.targets.size();
    for (int b = 0; b < a.k; b++) a.targets[b] = op.targets[b];
    const int grid = grid_for(a.count, 256);
    if (dtype == QSIM_C128) diag_kernel<double><<<grid, 256, 0, st>>>(a);
    else diag_kernel<float><<<grid, 256, 0, st>>>(a);
    check_launch("diag_kernel", 1, QSIM_KERNEL_ELEMENTWISE);
}

void run_swap(void *state, int n, int dtype, const Op &op, cudaStream_t st) {
    SwapArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    std::vector<int> f = op.controls;
    f.push_back(op.targets[0]);
    f.push_back(op.targets[1]);
    f = sorted_copy(f);
    fill_fix(a.fix, a.nfix, f);
    a.cmask = mask_of(op.controls);
    a.ma = (1ull << op.targets[0]) | a.cmask;
    a.mb = (1ull << op.targets[1]) | a.cmask;
    a.cmask = 0;  // folded into ma / mb
    a.count = 1ll << (n - (int)f.size());
    const int grid = grid_for(a.count, 256);
    if (dtype == QSIM_C128) swap_kernel<double><<<grid, 256, 0, st>>>(a);
    else swap_kernel<float><<<grid, 256, 0, st>>>(a);
    check_launch("swap_kernel", 1, QSIM_KERNEL_ELEMENTWISE);
}

void run_ucry(void *state, int n, int dtype, const Op &op, const void *csdev, cudaStream_t st,
              bool src_zero = false) {
    UcryArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    a.src_zero = src_zero ? 1 : 0;
    a.cs = csdev;
    a.count = 1ll << (n - 1);
    a.target = op.targets[0];
    a.nc = (int)op.controls.size();
    QSIM_REQUIRE(a.nc <= 32, "too many controls");
    a.contiguous = 1;
    a.c0 = op.controls[0];
    for (int j = 0; j < a.nc; j++) {
        a.ctrl[j] = op.controls[j];
        if (op.controls[j] != a.c0 + j) a.contiguous = 0;
    }
    const int grid = grid_for(a.count, 256);
    if (dtype == QSIM_C128) ucry_kernel<double><<<grid, 256, 0, st>>>(a);
    else ucry_kernel<float><<<grid, 256, 0, st>>>(a);
    check_launch("ucry_kernel", 1, QSIM_KERNEL_ELEMENTWISE);
}

// Tensor-core dense path for complex64: the kernel-choice table says which widths use it
// (bit k: k targets; bit 7: the real 7-target kernel).
bool tc_enabled(int k, int n) { return (tune_get(QSIM_C64, QSIM_TUNE_DENSE_TC, n) >> k) & 1; }

void run_qpe_phase(void *state, int n, int dtype, const Op &op, const void *lo, const void *hi, cudaStream_t st) {
    QpeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    a.lo = lo;
    a.hi = hi;
    a.N = 1ll << n;
    a.nb = (int)op.targets.size();
    a.m = (int)op.controls.size();
    a.h = (a.m + 1) / 2;
    for (int i = 0; i < a.nb; i++) QSIM_REQUIRE(op.targets[i] == i, "phase estimation: data qubits must be 0..nb-1");
    for (int j = 0; j < a.m; j++) QSIM_REQUIRE(op.controls[j] == a.nb + j, "phase estimation: clock qubits must follow the data");
    const int grid = grid_for(a.N, 256);
    if (dtype == QSIM_C128) qpe_phase_kernel<double><<<grid, 256, 0, st>>>(a);
    else qpe_phase_kernel<float><<<grid, 256, 0, st>>>(a);
    check_launch("qpe_phase_kernel", 1, QSIM_KERNEL_ELEMENTWISE);
}

// The pass `op` on the field w .. w+K-1 of a state that is zero from index 2^w on (see
// expand_kernel); qop: structured phase fused on the inputs (qmode 1) or outputs (qmode 2).
void run_expand(void *state, int w, int dtype, const Op &op, const Op *qop, const void *qlo, const void *qhi,
                int qmode, cudaStream_t st) {
    const int K = (int)op.targets.size();
    ExpandArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    a.lowN = 1ll << w;
    a.w = w;
    a.scale = std::ldexp(1.0, -K / 2) * ((K & 1) ? std::sqrt(0.5) : 1.0);
    a.K = K;
    a.run = std::min(32, (1 << K) - 1);
    if (qop && qmode) {
        a.qlo = qlo;
        a.qhi = qhi;
        a.qmode = qmode;
        a.qnb = (int)qop->targets.size();
        a.qm = (int)qop->controls.size();
        a.qh = (a.qm + 1) / 2;  // the split qpe_phase_tables uses
        // the field is clock bits; complex64 only (as in the Fourier passes)
        a.qrec = dtype == QSIM_C64 && w >= a.qnb && w + K <= a.qnb + a.qm ? 1 : 0;
    }
    for (int pass = 0; pass < 2; pass++) {  // outputs y >= 1 first, then column 0 in place
        a.col0 = pass;
        const long long runs = (((1ll << K) - 1) + a.run - 1) / a.run;
        a.count = pass ? a.lowN : a.lowN * runs;
        const int grid = grid_for(a.count, 256);
        if (dtype == QSIM_C128) expand_kernel<double><<<grid, 256, 0, st>>>(a);
        else expand_kernel<float><<<grid, 256, 0, st>>>(a);
        check_launch("expand_kernel", 1, QSIM_KERNEL_EXPAND);
    }
}

void run_hhl_invert(void *state, int n, int dtype, const Op &op, cudaStream_t st, bool src_zero = false) {
    InvertArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    a.src_zero = src_zero ? 1 : 0;
    a.count = 1ll << (n - 1);
    a.Cs = op.tq;
    a.target = op.targets[0];
    a.nc = (int)op.controls.size();
    a.twos = op.sign == -1 ? 1 : 0;
    for (int j = 0; j < a.nc;) {
        int w = 1;
        while (j + w < a.nc && op.controls[j + w] == op.controls[j] + w) w++;
        QSIM_REQUIRE(a.nseg < kMaxSeg, "inversion register: more than 8 runs of consecutive qubits");
        a.seg_src[a.nseg] = op.controls[j];
        a.seg_w[a.nseg] = w;
        a.seg_dst[a.nseg] = j;
        a.nseg++;
        j += w;
    }
    const int grid = grid_for(a.count, 256);
    if (dtype == QSIM_C128) hhl_invert_kernel<double><<<grid, 256, 0, st>>>(a);
    else hhl_invert_kernel<float><<<grid, 256, 0, st>>>(a);
    check_launch("hhl_invert_kernel", 1, QSIM_KERNEL_ELEMENTWISE);
}

}  // namespace

// Pack every op's device data (dense matrices transposed, diagonals, UCRY (cos, sin) tables)
// into one device allocation per dtype, uploaded once.
std::vector<unsigned char> pack_device_blob(qsim_circuit *c, int dtype) {
    const int slot = dtype == QSIM_C128 ? 1 : 0;
    std::vector<unsigned char> blob;
    for (Op &op : c->ops) {
        align_blob(blob);
        op.dev_off[slot] = blob.size();
        if (op.kind == OP_DENSE) {
            const int D = 1 << (int)op.targets.size();
            for (int col = 0; col < D; col++)
                for (int r = 0; r < D; r++) put_complex(blob, dtype, op.U[(size_t)r * D + col]);
            // Gates of 1..5 targets on qubit 0 or 1 (the other one a target or free) may be widened
            // with identity qubits to the transposed 6-target tensor-core form, which runs along
            // the low qubits.  Measured at 28 qubits: the group-major form's warp loads touch
            // 32 / 2^f lines of 128 B, f = free qubits among 0..3, and it takes 0.73 ms with f >= 2,
            // 1.12 ms with f = 1, 2.1 ms with f = 0; the SIMT kernels take 0.68-1.42 ms for 1..3
            // targets on qubit 0 or 1 (1.05 for targets {0, 1}, 1.42 for {0, 1, 2}); the
            // transposed form 0.67 ms with one of qubits 2 and 3 free, 0.71 with none, 0.73 with
            // both.  The widened form is taken where it is estimated 5% faster, and always for
            // 1..3 targets (never slower in the measurements).  6 targets need no widening: the
            // transposed form takes those on qubit 0 or 1 directly (0.70-0.73 ms; launch_dense_tc).
            const int k = (int)op.targets.size();
            auto used = [&](int q) {
                for (int x : op.targets) if (x == q) return true;
                for (int x : op.controls) if (x == q) return true;
                return false;
            };
            if (dtype == QSIM_C64) {
                op.has_tc = false;
                op.tc_pads.clear();
            }
            const bool t0 = op.targets[0] == 0, t1 = std::find(op.targets.begin(), op.targets.end(), 1) != op.targets.end();
            const int miss = !t0 + !t1;
            int f = 0;
            for (int q = 0; q < 4 && q < c->n; q++) f += !used(q);
            const int f23 = c->n > 3 ? (int)!used(2) + (int)!used(3) : 0;
            const int need = 6 - k - miss;  // qubits added above 0 and 1
            bool widen = false;
            bool pad2 = false;  // widen over qubit 2 as well, leaving qubit 3 the only free one of the two
            if (dtype == QSIM_C64 && (t0 || t1) && (t0 || !used(0)) && (t1 || !used(1)) && k < 6 && need >= 0) {
                const double now = k >= 4 ? (f == 0 ? 2.1 : f == 1 ? 1.12 : 0.73) : 1e30;
                pad2 = f23 == 2 && need >= 1;
                const int fw = f23 - (int)pad2;
                const double tr = fw == 1 ? 0.67 : fw == 0 ? 0.71 : 0.73;
                widen = tr < 0.95 * now;
            }
            std::vector<int> pads;  // qubits 0 and 1 when missing, (2), then free ones from 4 up
            if (widen) {
                if (!t0) pads.push_back(0);
                if (!t1) pads.push_back(1);
                if (pad2) pads.push_back(2);
                for (int q = 4; q < c->n && (int)pads.size() < 6 - k; q++)
                    if (!used(q)) pads.push_back(q);
            }
            if (widen && (int)pads.size() == 6 - k) {
                std::vector<int> tw(op.targets);
                tw.insert(tw.end(), pads.begin(), pads.end());
                std::sort(tw.begin(), tw.end());
                int pmask = 0;  // bit positions of the added qubits in the widened index
                for (int q : pads) pmask |= 1 << (int)(std::find(tw.begin(), tw.end(), q) - tw.begin());
                auto drop = [&](int x) {  // the widened index without the added bits
                    int v = 0, b = 0;
                    for (int i = 0; i < 6; i++)
                        if (!((pmask >> i) & 1)) v |= ((x >> i) & 1) << b++;
                    return v;
                };
                const int DW = 64;
                std::vector<cd> UW((size_t)DW * DW, cd(0.0, 0.0));
                for (int r = 0; r < DW; r++)
                    for (int cc = 0; cc < DW; cc++)
                        if ((r & pmask) == (cc & pmask)) UW[(size_t)r * DW + cc] = op.U[(size_t)drop(r) * D + drop(cc)];
                align_blob(blob);
                op.dev_off_tcw = blob.size();
                op.tc_pads = pads;
                blob.resize(blob.size() + dense_tc_blob_bytes(6));
                dense_tc_pack(6, UW, blob.data() + op.dev_off_tcw);
            }
            // the gate's own tensor-core form (also where the widened one is not taken)
            if (dtype == QSIM_C64 && dense_tc_supported((int)op.targets.size())) {
                align_blob(blob);
                op.dev_off_tc[slot] = blob.size();
                op.has_tc = true;
                const size_t nb = dense_tc_blob_bytes((int)op.targets.size());
                blob.resize(blob.size() + nb);
                dense_tc_pack((int)op.targets.size(), op.U, blob.data() + op.dev_off_tc[slot]);
            } else if (dtype == QSIM_C64 && dense_tc_real7_applies(op)) {
                align_blob(blob);
                op.dev_off_tc[slot] = blob.size();
                op.has_tc = true;
                blob.resize(blob.size() + dense_tc_real7_blob_bytes());
                dense_tc_pack_real7(op.U, blob.data() + op.dev_off_tc[slot]);
            }
        } else if (op.kind == OP_DIAG) {
            for (const cd &z : op.U) put_complex(blob, dtype, z);
        } else if (op.kind == OP_UCRY) {
            for (double th : op.theta) put_complex(blob, dtype, cd(std::cos(0.5 * th), std::sin(0.5 * th)));
        } else if (op.kind == OP_QPE_PHASE) {
            std::vector<cd> lo, hi;
            int h = 0;
            qpe_phase_tables(op, lo, hi, h);
            for (const cd &z : lo) put_complex(blob, dtype, z);
            align_blob(blob);
            op.dev_off_tc[slot] = blob.size();  // second table
            for (const cd &z : hi) put_complex(blob, dtype, z);
        } else if (op.kind == OP_DFT || op.kind == OP_WALSH) {
            std::vector<cd> W, Tlo, Thi;
            dft_tables(op, W, Tlo, Thi);
            for (const cd &z : W) put_complex(blob, dtype, z);
            for (const cd &z : Tlo) put_complex(blob, dtype, z);
            for (const cd &z : Thi) put_complex(blob, dtype, z);
        }
    }
    align_blob(blob);
    if (blob.empty()) blob.resize(256, 0);
    return blob;
}

void attach_external_blob(qsim_circuit *c, int dtype, void *dev, size_t bytes) {
    std::lock_guard<std::mutex> lk(c->mu);
    int d = 0;
    CUDA_OK(cudaGetDevice(&d));
    DeviceBlob &B = c->blob[dtype == QSIM_C128 ? 1 : 0];
    QSIM_REQUIRE(B.ptr == nullptr, "circuit already has device matrices");
    B.ptr = dev;
    B.bytes = bytes;
    B.device = d;
    B.external = true;
}

void ensure_device_blob(qsim_circuit *c, int dtype) {
    build_ops(c);
    std::lock_guard<std::mutex> lk(c->mu);
    const int slot = dtype == QSIM_C128 ? 1 : 0;
    int dev = 0;
    CUDA_OK(cudaGetDevice(&dev));
    DeviceBlob &B = c->blob[slot];
    if (B.ptr && B.device == dev) return;
    QSIM_REQUIRE(B.ptr == nullptr, "circuit already uploaded to another device");
    std::vector<unsigned char> blob = pack_device_blob(c, dtype);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, blob.size());
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(QSIM_ENOMEM, std::string("cudaMalloc for circuit matrices: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(p, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p);
        throw Error(QSIM_ECUDA, std::string("cudaMemcpy circuit matrices: ") + cudaGetErrorString(e));
    }
    B.ptr = p;
    B.bytes = blob.size();
    B.device = dev;
}

// A structured phase (diagonal) next to a Fourier or Walsh-Hadamard pass is applied inside that
// pass (to its outputs or inputs) instead of as a pass of its own; a pass without twiddle is
// preferred.
static bool is_pass(const Op &op) { return op.kind == OP_DFT || op.kind == OP_WALSH; }

static int top_qubit(const Op &op) {
    int q = -1;
    for (int t : op.targets) q = std::max(q, t);
    for (int t : op.controls) q = std::max(q, t);
    return q;
}

static int readout_blocks(int n);

void apply_ops(void *state, int n, int dtype, qsim_circuit *c, void *stream, int live, double *sums) {
    ensure_device_blob(c, dtype);
    const int slot = dtype == QSIM_C128 ? 1 : 0;
    const unsigned char *base = static_cast<const unsigned char *>(c->blob[slot].ptr);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const std::vector<Op> &ops = c->ops;
    // Live width w: every amplitude at an index >= 2^w is zero and has not been written (HHL: after
    // the preparation only the data register is populated).  An op on qubits below w runs as a
    // w-qubit state; a twiddle-free pass on the field right above w broadcasts column 0 (write
    // only) and widens w; diagonal ops leave zeros zero; the inversion rotation on the top qubit
    // writes the upper half without reading it (inside the preceding pass when that pass runs
    // right below it); any other op first zero-fills up to its top qubit.
    int w = (live >= 0 && live < n) ? live : n;
    bool sums_done = false;  // the last operation's kernel wrote the readout sums
    const size_t vb = 2 * real_size(dtype);
    auto materialize = [&](int to) {
        if (to <= w) return;
        unsigned char *p = static_cast<unsigned char *>(state);
        CUDA_OK(cudaMemsetAsync(p + (vb << w), 0, (vb << to) - (vb << w), st));
        w = to;
    };
    auto expandable = [&](const Op &p) {
        if (!is_pass(p) || w >= n) return false;
        for (size_t j = 0; j < p.targets.size(); j++)
            if (p.targets[j] != w + (int)j) return false;
        for (int q : p.controls)
            if (q >= w) return false;
        return p.kind == OP_WALSH || p.controls.empty() || p.pre;  // no twiddle on the outputs
    };
    for (size_t i = 0; i < ops.size(); i++) {
        const Op &op = ops[i];
        const void *dptr = base + op.dev_off[slot];
        if (op.kind == OP_WALSH && i + 2 < ops.size() && ops[i + 1].kind == OP_QPE_PHASE && ops[i + 2].kind == OP_DFT &&
            ops[i + 2].targets == op.targets && expandable(op)) {
            // H on a field that is still |0> right above the live part, the structured phase and a
            // Fourier pass on the same field: the pass generates its inputs (complex64)
            const Op &q = ops[i + 1];
            if (run_dft_generated(state, w, dtype, ops[i + 2], base + ops[i + 2].dev_off[slot], q, base + q.dev_off[slot],
                                  base + q.dev_off_tc[slot], st)) {
                w += (int)op.targets.size();
                i += 2;
                continue;
            }
        }
        if (op.kind == OP_DFT && i + 2 < ops.size() && ops[i + 1].kind == OP_QPE_PHASE && ops[i + 2].kind == OP_WALSH &&
            ops[i + 2].targets == op.targets && !expandable(op)) {
            // a QFT pass, the structured phase and the Walsh-Hadamard pass of the same field in one
            // tile-resident kernel (complex64, bulk-copy tiles) when the shapes fit
            const Op &q = ops[i + 1];
            materialize(std::max(top_qubit(op), top_qubit(ops[i + 2])) + 1);
            if (run_dft2(state, w, dtype, 2, op, dptr, q, base + q.dev_off[slot], base + q.dev_off_tc[slot], ops[i + 2],
                         base + ops[i + 2].dev_off[slot], st)) {
                i += 2;
                continue;
            }
        }
        if (i + 1 < ops.size()) {
            // a structured phase next to a pass runs inside it: on the pass's outputs, unless this
            // pass has a twiddle and the pass after the phase has none (then on that one's inputs)
            size_t pi = ops.size(), qi = ops.size();
            int qmode = 0;
            if (is_pass(op) && ops[i + 1].kind == OP_QPE_PHASE) {
                const bool next_better = !op.controls.empty() && i + 2 < ops.size() && is_pass(ops[i + 2]) &&
                                         ops[i + 2].controls.empty();
                if (!next_better) pi = i, qi = i + 1, qmode = 2;
            } else if (op.kind == OP_QPE_PHASE && is_pass(ops[i + 1])) {
                pi = i + 1, qi = i, qmode = 1;
            }
            if (qmode) {
                const Op &p = ops[pi], &q = ops[qi];
                const void *qlo = base + q.dev_off[slot], *qhi = base + q.dev_off_tc[slot];
                if (expandable(p)) {
                    run_expand(state, w, dtype, p, &q, qlo, qhi, qmode, st);
                    w += (int)p.targets.size();
                } else {
                    materialize(top_qubit(p) + 1);  // the phase is diagonal: zeros stay zero
                    run_dft(state, w, dtype, p, base + p.dev_off[slot], st, &q, qlo, qhi, qmode);
                }
                i++;
                continue;
            }
        }
        if (is_pass(op) && i + 1 < ops.size() && ops[i + 1].kind == OP_HHL_INVERT && w == n - 1 &&
            ops[i + 1].targets[0] == n - 1 && top_qubit(op) < w && top_qubit(ops[i + 1]) == n - 1) {
            // the pass writes the rotated outputs into both halves (the upper one is unwritten)
            bool low = true;
            for (int q : ops[i + 1].controls) low = low && q < n - 1;
            // ... and, when the QFT's first pass over the same field follows, that pass too (one
            // tile-resident kernel per half, complex64 bulk-copy tiles, when the shapes fit)
            if (low && i + 2 < ops.size() && ops[i + 2].kind == OP_DFT && ops[i + 2].targets == op.targets &&
                run_dft2(state, w, dtype, 1, op, dptr, ops[i + 1], nullptr, nullptr, ops[i + 2],
                         base + ops[i + 2].dev_off[slot], st)) {
                w = n;
                i += 2;
                continue;
            }
            if (low && run_dft(state, w, dtype, op, dptr, st, nullptr, nullptr, nullptr, 0, &ops[i + 1])) {
                w = n;
                i++;
                continue;
            }
        }
        if (expandable(op)) {
            run_expand(state, w, dtype, op, nullptr, nullptr, nullptr, 0, st);
            w += (int)op.targets.size();
            continue;
        }
        if (op.kind == OP_QPE_PHASE) {  // diagonal: only the live part needs it
            run_qpe_phase(state, w, dtype, op, dptr, base + op.dev_off_tc[slot], st);
            continue;
        }
        if (op.kind == OP_PHASE && top_qubit(op) >= w) continue;  // needs a 1 where all are 0
        if ((op.kind == OP_HHL_INVERT || op.kind == OP_UCRY) && w < n && op.targets[0] == n - 1) {
            bool low = true;
            for (int q : op.controls) low = low && q < n - 1;
            if (low) {
                materialize(n - 1);
                if (op.kind == OP_HHL_INVERT) run_hhl_invert(state, n, dtype, op, st, true);
                else run_ucry(state, n, dtype, op, dptr, st, true);
                w = n;
                continue;
            }
        }
        materialize(top_qubit(op) + 1);
        switch (op.kind) {
            case OP_DENSE:
                if (dtype == QSIM_C64 && !op.tc_pads.empty()) {
                    // widened with identity qubits; all of them must lie inside the live width.  Gates
                    // of 1..3 targets are widened only on states larger than L2 (2^24 amplitudes),
                    // where the SIMT kernels' low-qubit loads were measured slower; below, they stay.
                    bool inside = tc_enabled(6, w) && (op.targets.size() >= 4 || w >= 24);
                    for (int q : op.tc_pads) inside = inside && q < w;
                    if (inside) {
                        std::vector<int> tw(op.targets);
                        tw.insert(tw.end(), op.tc_pads.begin(), op.tc_pads.end());
                        std::sort(tw.begin(), tw.end());
                        double *s7 = (sums && i + 1 == ops.size() && op.controls.empty()) ? sums : nullptr;
                        if (launch_dense_tc(state, w, tw, op.controls, base + op.dev_off_tcw, num_sms(), st, s7, n - 1,
                                            &sums_done))
                            break;
                    }
                }
                if (dtype == QSIM_C64 && op.has_tc && tc_enabled((int)op.targets.size(), w)) {
                    double *s7 = (sums && i + 1 == ops.size() && op.controls.empty()) ? sums : nullptr;
                    if (op.targets.size() == 7
                            ? launch_dense_tc_real7(state, w, op.targets, op.controls, base + op.dev_off_tc[slot], num_sms(),
                                                    st, s7, n - 1, &sums_done)
                            : launch_dense_tc(state, w, op.targets, op.controls, base + op.dev_off_tc[slot], num_sms(), st,
                                              s7, n - 1, &sums_done))
                        break;
                }
                run_dense(state, w, dtype, op, dptr, st);
                break;
            case OP_PHASE: run_phase(state, w, dtype, op, st); break;
            case OP_DIAG: run_diag(state, w, dtype, op, dptr, st); break;
            case OP_SWAP: run_swap(state, w, dtype, op, st); break;
            case OP_UCRY: run_ucry(state, w, dtype, op, dptr, st); break;
            case OP_QPE_PHASE: break;  // handled above
            case OP_HHL_INVERT: run_hhl_invert(state, w, dtype, op, st); break;
            case OP_DFT:
            case OP_WALSH: run_dft(state, w, dtype, op, dptr, st); break;
        }
    }
    materialize(n);
    if (sums && !sums_done) {  // the readout sums by a reduction pass of their own
        const int nblk = readout_blocks(n);
        const long long chunk = (1ll << n) / nblk;
        if (dtype == QSIM_C128) norm_partials_kernel<double><<<nblk, 256, 0, st>>>(state, chunk, sums + 1, sums);
        else norm_partials_kernel<float><<<nblk, 256, 0, st>>>(state, chunk, sums + 1, sums);
        check_launch("norm_partials_kernel", 1, QSIM_KERNEL_READOUT);
    }
}

void launch_prepare_state(void *state, int n, int dtype, const cd *b_pad, int nb, void *stream, int live) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PrepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    a.N = 1ll << n;
    a.D = 1 << nb;
    const int inl = std::min(a.D, kMaxParamB);
    for (int i = 0; i < inl; i++) {
        a.b[2 * i] = b_pad[i].real();
        a.b[2 * i + 1] = b_pad[i].imag();
    }
    const size_t vbytes = 2 * real_size(dtype);
    // live < n: only the first 2^live amplitudes are written (the caller treats the rest as
    // known zero)
    const long long written = (live >= nb && live < n) ? (1ll << live) : a.N;
    CUDA_OK(cudaMemsetAsync(state, 0, (size_t)written * vbytes, st));
    if (dtype == QSIM_C128) prep_kernel<double><<<1, kMaxParamB, 0, st>>>(a);
    else prep_kernel<float><<<1, kMaxParamB, 0, st>>>(a);
    check_launch("prep_kernel", 1, QSIM_KERNEL_PREP);
    if (a.D > kMaxParamB) {  // rare: long right-hand sides go through a staged copy
        const int rest = a.D - kMaxParamB;
        std::vector<unsigned char> buf;
        for (int i = kMaxParamB; i < a.D; i++) put_complex(buf, dtype, b_pad[i]);
        const size_t vb = 2 * real_size(dtype);
        CUDA_OK(cudaMemcpyAsync(static_cast<unsigned char *>(state) + (size_t)kMaxParamB * vb,
                                buf.data(), (size_t)rest * vb, cudaMemcpyHostToDevice, st));
        CUDA_OK(cudaStreamSynchronize(st));
    }
}

static int readout_blocks(int n) {
    int lg = std::max(1, std::min(11, n - 12));
    if (n <= 1) lg = 0;
    return 1 << lg;
}

// scratch of readout_launch_async: a readout-sums buffer (count, then up to 4095 partials) and
// the 3 final sums
size_t readout_scratch_doubles(int n) {
    (void)n;
    return (size_t)QSIM_READOUT_SUMS_DOUBLES + 8;
}

void readout_launch_async(const void *state, int dtype, int n, int nb, cudaStream_t st, double *scratch,
                          double *pinned_sums, void *pinned_slice, bool sums_ready) {
    const long long N = 1ll << n;
    const size_t vb = 2 * real_size(dtype);
    const size_t slice_len = (size_t)1 << nb;
    double *out = scratch + QSIM_READOUT_SUMS_DOUBLES;
    const long long off = N / 2;
    if (!sums_ready) {  // the partial sums by a reduction pass (else apply_ops left them)
        const int nblk = readout_blocks(n);
        const long long chunk = N / nblk;
        if (dtype == QSIM_C128) norm_partials_kernel<double><<<nblk, 256, 0, st>>>(state, chunk, scratch + 1, scratch);
        else norm_partials_kernel<float><<<nblk, 256, 0, st>>>(state, chunk, scratch + 1, scratch);
        check_launch("norm_partials_kernel", 1, QSIM_KERNEL_READOUT);
    }
    if (dtype == QSIM_C128) norm_final_buf_kernel<double><<<1, 256, 0, st>>>(scratch, state, off, (int)slice_len, out);
    else norm_final_buf_kernel<float><<<1, 256, 0, st>>>(scratch, state, off, (int)slice_len, out);
    check_launch("norm_final_buf_kernel", 1, QSIM_KERNEL_READOUT);
    CUDA_OK(cudaMemcpyAsync(pinned_sums, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(pinned_slice, static_cast<const unsigned char *>(state) + off * vb, slice_len * vb,
                            cudaMemcpyDeviceToHost, st));
}

void readout_device(const void *state, int dtype, int n, int nb, int m, void *stream,
                    double sums[3], cd *slice) {
    (void)m;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long N = 1ll << n;
    // fixed block count for a given n: chunks of 2^12 amplitudes, at most 2048 blocks
    int lg = std::max(1, std::min(11, n - 12));
    if (n <= 1) lg = 0;
    const int nblk = 1 << lg;
    const long long chunk = N / nblk;
    const size_t vb = 2 * real_size(dtype);
    const size_t slice_len = (size_t)1 << nb;
    void *scratch = nullptr;
    const size_t scratch_bytes = (size_t)nblk * 8 + 64 + slice_len * vb;
    cudaError_t e = cudaMallocAsync(&scratch, scratch_bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(QSIM_ENOMEM, std::string("cudaMallocAsync readout scratch: ") + cudaGetErrorString(e));
    }
    double *partials = static_cast<double *>(scratch);
    double *out = partials + nblk;
    const long long off = N / 2;  // ancilla = 1 (the top qubit), clock = 0
    try {
        if (dtype == QSIM_C128) {
            norm_partials_kernel<double><<<nblk, 256, 0, st>>>(state, chunk, partials);
            norm_final_kernel<double><<<1, 256, 0, st>>>(partials, nblk, state, off, (int)slice_len, out);
        } else {
            norm_partials_kernel<float><<<nblk, 256, 0, st>>>(state, chunk, partials);
            norm_final_kernel<float><<<1, 256, 0, st>>>(partials, nblk, state, off, (int)slice_len, out);
        }
        check_launch("readout kernels", 2, QSIM_KERNEL_READOUT);
        std::vector<unsigned char> hs(slice_len * vb);
        double hsum[3];
        CUDA_OK(cudaMemcpyAsync(hsum, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_OK(cudaMemcpyAsync(hs.data(), static_cast<const unsigned char *>(state) + off * vb,
                                slice_len * vb, cudaMemcpyDeviceToHost, st));
        CUDA_OK(cudaFreeAsync(scratch, st));
        scratch = nullptr;
        CUDA_OK(cudaStreamSynchronize(st));
        for (int i = 0; i < 3; i++) sums[i] = hsum[i];
        for (size_t i = 0; i < slice_len; i++) {
            if (dtype == QSIM_C128) {
                const double *p = reinterpret_cast<const double *>(hs.data()) + 2 * i;
                slice[i] = cd(p[0], p[1]);
            } else {
                const float *p = reinterpret_cast<const float *>(hs.data()) + 2 * i;
                slice[i] = cd(p[0], p[1]);
            }
        }
    } catch (...) {
        if (scratch) cudaFreeAsync(scratch, st);
        throw;
    }
}

void readout_device_sums(const void *state, int dtype, int n, int nb, void *stream, const double *buf,
                         double sums[3], cd *slice) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long N = 1ll << n;
    const size_t vb = 2 * real_size(dtype);
    const size_t slice_len = (size_t)1 << nb;
    const long long off = N / 2;  // ancilla = 1 (the top qubit), clock = 0
    void *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, 64, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(QSIM_ENOMEM, std::string("cudaMallocAsync readout scratch: ") + cudaGetErrorString(e));
    }
    double *out = static_cast<double *>(scratch);
    try {
        if (dtype == QSIM_C128) norm_final_buf_kernel<double><<<1, 256, 0, st>>>(buf, state, off, (int)slice_len, out);
        else norm_final_buf_kernel<float><<<1, 256, 0, st>>>(buf, state, off, (int)slice_len, out);
        check_launch("norm_final_buf_kernel", 1, QSIM_KERNEL_READOUT);
        std::vector<unsigned char> hs(slice_len * vb);
        double hsum[3];
        CUDA_OK(cudaMemcpyAsync(hsum, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_OK(cudaMemcpyAsync(hs.data(), static_cast<const unsigned char *>(state) + off * vb, slice_len * vb,
                                cudaMemcpyDeviceToHost, st));
        CUDA_OK(cudaFreeAsync(scratch, st));
        scratch = nullptr;
        CUDA_OK(cudaStreamSynchronize(st));
        for (int k = 0; k < 3; k++) sums[k] = hsum[k];
        for (size_t k = 0; k < slice_len; k++) {
            if (dtype == QSIM_C128) {
                const double *p = reinterpret_cast<const double *>(hs.data()) + 2 * k;
                slice[k] = cd(p[0], p[1]);
            } else {
                const float *p = reinterpret_cast<const float *>(hs.data()) + 2 * k;
                slice[k] = cd(p[0], p[1]);
            }
        }
    } catch (...) {
        if (scratch) cudaFreeAsync(scratch, st);
        throw;
    }
}

// ---------------------------------------------------------------------------------------
// Readout without any device allocation.
//
// Some callers cannot allocate device memory while they read a result: an application that
// hands all device memory to its own pool allocator up front, or code that runs where
// cudaMalloc/cudaMallocAsync must not be called.  hhl_readout_noalloc gives them the same
// readout as hhl_readout with its scratch (the per-block partial sums, the three totals and a
// double-precision copy of the solution slice) in the file-scope device array below, which
// every GPU that loads this library holds until the process exits.
namespace {
constexpr int kNoAllocMaxBlocks = 2048;          // partial sums (the readout grid never exceeds it)
constexpr int kNoAllocMaxSlice = 1 << 10;        // amplitudes of the solution slice (2^nb)
constexpr int kNoAllocDoubles = kNoAllocMaxBlocks + 8 + 2 * kNoAllocMaxSlice;
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

template <typename R>
__global__ void slice_to_f64_kernel(const void *state, long long off, int len, double *out) {
    using V = typename C2<R>::T;
    const V *psi = reinterpret_cast<const V *>(state) + off;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
        const V z = psi[i];
        out[2 * i] = (double)z.x;
        out[2 * i + 1] = (double)z.y;
    }
}

// Device address of g_noalloc_scratch on the current device, looked up once per device (the
// array's name in host code is only a host-side stand-in, not a device address).
static double *noalloc_scratch_on_current_device() {
    static std::mutex mu;
    static double *addr[128] = {};
    int dev = 0;
    CUDA_OK(cudaGetDevice(&dev));
    QSIM_REQUIRE(dev >= 0 && dev < 128, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (addr[dev] == nullptr) {
        void *p = nullptr;
        CUDA_OK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        addr[dev] = static_cast<double *>(p);
    }
    return addr[dev];
}

}  // namespace qsim

extern "C" int hhl_readout_noalloc(const void *state, int dtype, const hhl_circuit *h, void *stream,
                                   double *x_out, double *x_state_out, hhl_readout_stats *stats) {
    using namespace qsim;
    return guarded([&] {
        QSIM_REQUIRE(state != nullptr && h != nullptr, "NULL argument");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        const int n = h->n, nb = h->nb;
        const long long slice_len = 1ll << nb;
        if (slice_len > kNoAllocMaxSlice)
            throw Error(QSIM_EINVAL, "hhl_readout_noalloc: the solution slice has 2^" + std::to_string(nb) +
                                         " amplitudes, more than the fixed scratch holds (2^10, i.e. N <= 1024)");
        int lg = std::max(1, std::min(11, n - 12));
        if (n <= 1) lg = 0;
        const int nblk = 1 << lg;
        QSIM_REQUIRE(nblk <= kNoAllocMaxBlocks, "hhl_readout_noalloc: too many partial sums");
        const long long N = 1ll << n;
        const long long chunk = N / nblk;
        const long long off = N / 2;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        double *scratch = noalloc_scratch_on_current_device();
        double *partials = scratch;
        double *out = scratch + kNoAllocMaxBlocks;
        double *slice = scratch + kNoAllocMaxBlocks + 8;
        // every slot read below is written earlier in this same call, so nothing is cleared
        if (dtype == QSIM_C128) {
            norm_partials_kernel<double><<<nblk, 256, 0, st>>>(state, chunk, partials);
            norm_final_kernel<double><<<1, 256, 0, st>>>(partials, nblk, state, off, (int)slice_len, out);
            slice_to_f64_kernel<double><<<(int)((slice_len + 255) / 256), 256, 0, st>>>(state, off, (int)slice_len, slice);
        } else {
            norm_partials_kernel<float><<<nblk, 256, 0, st>>>(state, chunk, partials);
            norm_final_kernel<float><<<1, 256, 0, st>>>(partials, nblk, state, off, (int)slice_len, out);
            slice_to_f64_kernel<float><<<(int)((slice_len + 255) / 256), 256, 0, st>>>(state, off, (int)slice_len, slice);
        }
        check_launch("hhl_readout_noalloc kernels", 3, QSIM_KERNEL_READOUT);
        double sums[3];
        CUDA_OK(cudaMemcpyAsync(sums, out, sizeof(sums), cudaMemcpyDeviceToHost, st));
        // the slice lands straight in the caller's buffer: all 2^nb amplitudes, or the N entries
        // of x (from offset x_off of a dilated system)
        double *dst = x_state_out ? x_state_out : x_out;
        const long long cnt = x_state_out ? slice_len : (long long)h->N;
        const double *src = x_state_out ? slice : slice + 2 * (size_t)h->x_off;
        if (dst) CUDA_OK(cudaMemcpyAsync(dst, src, (size_t)cnt * 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_OK(cudaStreamSynchronize(st));
        const double P = sums[1], P0 = sums[2];
        const double inv = P0 > 0.0 ? 1.0 / std::sqrt(P0) : 0.0;
        const double norm_x = std::sqrt(P) / h->C;
        if (x_state_out) {
            if (x_out)
                for (int i = 0; i < h->N; i++) {
                    x_out[2 * i] = x_state_out[2 * (h->x_off + i)] * inv * norm_x * h->norm_b;
                    x_out[2 * i + 1] = x_state_out[2 * (h->x_off + i) + 1] * inv * norm_x * h->norm_b;
                }
            for (long long i = 0; i < 2 * slice_len; i++) x_state_out[i] *= inv;
        } else if (x_out) {
            for (int i = 0; i < 2 * h->N; i++) x_out[i] *= inv * norm_x * h->norm_b;
        }
        if (stats) {
            stats->p_success = P;
            stats->p_clock0 = P0;
            stats->leakage = P - P0;
            stats->norm2 = sums[0];
            stats->norm_x = norm_x;
            stats->norm_b = h->norm_b;
        }
    });
}

using namespace qsim;

qsim_circuit::~qsim_circuit() {
    for (DeviceBlob &b : blob) {
        if (b.ptr && !b.external) {
            int cur = -1;
            cudaGetDevice(&cur);
            if (cur != b.device) cudaSetDevice(b.device);
            cudaFree(b.ptr);
            if (cur != b.device && cur >= 0) cudaSetDevice(cur);
            b.ptr = nullptr;
        }
    }
}

extern "C" void qsim_circuit_free(qsim_circuit *c) { delete c; }

extern "C" unsigned long long qsim_launch_count(void) { return g_launches.load(); }

extern "C" int qsim_launch_counts(unsigned long long *counts, int n) {
    return guarded([&] {
        QSIM_REQUIRE(counts != nullptr && n >= 0, "NULL argument");
        for (int i = 0; i < n && i < QSIM_KERNEL_FAMILIES; i++) counts[i] = g_family[i].load();
        for (int i = QSIM_KERNEL_FAMILIES; i < n; i++) counts[i] = 0;
    });
}

extern "C" int qsim_apply(void *state, int n_qubits, int dtype, const qsim_circuit *c, void *stream) {
    return guarded([&] {
        QSIM_REQUIRE(state != nullptr && c != nullptr, "NULL argument");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        QSIM_REQUIRE(n_qubits == c->n, "state qubit count does not match the circuit");
        apply_ops(state, n_qubits, dtype, const_cast<qsim_circuit *>(c), stream);
    });
}
