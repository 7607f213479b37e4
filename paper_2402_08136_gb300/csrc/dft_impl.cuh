// Device side of the Fourier-transform passes (sm_103a), included by dft_f32.cu and dft_f64.cu
// (one translation unit per precision, compiled in parallel).
//
// The operation (qsim_circuit_add_dft): for every assignment of the other qubits, a DFT of size
// 2^K over a field of K qubits (y = field value), with the diagonal twiddle
// exp(s 2 pi i w y / 2^(K + ns)) on the input index (before) or on the output index (after),
// w = value of the ns twiddle-source qubits.  The inverse QFT and the QFT of the HHL phase
// estimation (Sec. III-A, Fig. 5) are one to three such passes instead of m Hadamards,
// m (m - 1) / 2 controlled phases and m / 2 swaps.
//
// A CTA owns a tile of 2^K x 2^L amplitudes: the whole field times the L lowest other qubits
// ("lanes"; with the field above them, 2^L amplitudes are contiguous in HBM).  The 2^K-point
// transform is split once more, 2^K = N1 N2 with N2 = 2^ceil(K/2), y = u + N1 v:
//   pass 1  thread (lane l, u) loads its N2 points v < N2 straight from HBM into registers,
//           applies the input twiddle, transforms over v (radix 2, registers), multiplies
//           by exp(s 2 pi i u a / 2^K) (a = output digit) and parks the results in shared
//           memory;
//   pass 2  thread (lane l, group g) reads the N1 points u < N1 of each of its a values back,
//           transforms over u and writes output y' = a + N2 b to HBM with the output twiddle
//           and the 2^(-K/2) normalisation.
// Warp accesses to HBM are runs of 2^L consecutive amplitudes (128 bytes), so the pass streams
// the state once, read and write, whatever K is; the arithmetic is 5 K flops per amplitude
// (radix-2 count) plus the twiddles.
//
// The same kernel with every twiddle equal to 1 and no digit reversal is the Walsh-Hadamard
// transform of the field, H on each of its qubits (qsim_circuit_add_walsh): the Hadamard
// layers of the phase estimation in one pass per field.
//
// Options: the structured phase-estimation diagonal on the inputs or outputs (qmode), the HHL
// inversion rotation on the outputs (KIND 2, writing the unwritten upper half), and an L2
// prefetch of the next tile's lines once a tile's inputs are in registers (pf).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.h"

namespace qsim {
namespace dftk {

#define DFT_CUDA_OK(call)                                                                     \
    do {                                                                                      \
        cudaError_t e__ = (call);                                                             \
        if (e__ != cudaSuccess)                                                               \
            throw ::qsim::Error(QSIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

constexpr int kMaxK = 10;     // field qubits
constexpr int kMaxLane = 8;   // lane qubits
constexpr int kMaxSrc = 30;   // twiddle-source qubits

template <typename R> struct CV;
template <> struct CV<float> { using T = float2; };
template <> struct CV<double> { using T = double2; };

template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

struct DftArgs {
    void *psi;
    const void *W;    // 2^K entries exp(s 2 pi i j / 2^K)
    const void *Tlo;  // 2^hT entries exp(s 2 pi i j / 2^(K+ns))
    const void *Thi;  // 2^(K+ns-hT) entries exp(s 2 pi i j 2^hT / 2^(K+ns))
    long long ntiles;
    double scale;     // 2^(-K/2)
    int L;            // lane qubits
    int twmode;       // 0 no twiddle, 1 before the transform, 2 after
    int hT, ns, nfix;
    int f0;                     // lowest field qubit (contiguous field: bit j on qubit f0 + j)
    int tw_smem;                // 1: the twiddle tables Tlo, Thi are copied to shared memory
    int pf;                     // > 0: the lanes are qubits 0..L-1 and a lane run is one
                                // 128-byte line: each tile prefetches the lines of the tile pf
                                // steps ahead of it (in this CTA's sequence) into L2
    // structured phase-estimation diagonal exp(i s lam_d t c) applied inside the pass (qmode 1:
    // to the inputs, 2: to the outputs): d = qubits 0..qnb-1, c = qubits qnb..qnb+qm-1, tables
    // qlo[(c mod 2^qh) 2^qnb + d], qhi[(c >> qh) 2^qnb + d]
    const void *qlo, *qhi;
    int qmode, qnb, qm, qh;
    int qrec;                   // 1 (complex64): the field lies inside the clock register
                                // (contiguous), so a thread's phases along the field are a
                                // geometric sequence, refreshed from the tables every 8 terms
    // HHL eigenvalue inversion fused into the outputs (contiguous field, upper half unwritten):
    // the ancilla is index bit inv_bit; k = clock value, bits from the index through nseg runs
    // (run s: bits dst[s] .. dst[s]+w[s]-1 of k on qubits src[s] ..), the field's own bits land
    // on bits inv_fdst .. of k; r = clamp(Cs / k) (two's complement if inv_twos), the output z
    // goes to psi[idx] as sqrt((1 - |r|)(1 + |r|)) z and to psi[idx + 2^inv_bit] as r z
    int inv, inv_bit, inv_twos, inv_nc, inv_fdst, inv_nseg;
    double inv_Cs;
    int inv_src[8], inv_w[8], inv_dst[8];
    int fpos[kMaxK];            // qubit of field bit j
    int lpos[kMaxLane];         // qubit of lane bit j
    int spos[kMaxSrc];          // qubit of twiddle-source bit j
    int fix[kMaxK + kMaxLane];  // field and lane qubits ascending (zero insertion)
};

__device__ __forceinline__ unsigned long long insert_zero_bits(unsigned long long x, const int *pos, int cnt) {
    for (int i = 0; i < cnt; i++) {
        const int p = pos[i];
        x = ((x >> p) << (p + 1)) | (x & ((1ull << p) - 1ull));
    }
    return x;
}

// exp(-2 pi i e / 32), e < 32, evaluated at compile time: exact octant reduction (e = 8 q + r,
// angle q pi / 2 + r pi / 16, r folded to at most pi / 8 by cos(pi/2 - x) = sin x), then Taylor
// series, so every entry is within about an ulp.  The in-register transforms of up to 32
// points read their twiddles from this table at compile-time offsets (constant-bank operands).
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int i = 1; i < 14; i++) {
        term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 14; i++) {
        term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        sum += term;
    }
    return sum;
}
struct TwTable {
    double re[32], im[32];
    float fre[32], fim[32];
};
constexpr TwTable make_twiddles() {
    TwTable t{};
    for (int e = 0; e < 32; e++) {
        const int q = e / 8, r = e % 8;
        double c = 0.0, s = 0.0;
        if (r <= 4) {
            c = taylor_cos(kTwoPi * r / 32.0);
            s = taylor_sin(kTwoPi * r / 32.0);
        } else {
            c = taylor_sin(kTwoPi * (8 - r) / 32.0);
            s = taylor_cos(kTwoPi * (8 - r) / 32.0);
        }
        double re = c, im = s;  // exp(+i angle); times i per quadrant
        for (int k = 0; k < q; k++) {
            const double tre = -im;
            im = re;
            re = tre;
        }
        t.re[e] = re;
        t.im[e] = -im;  // exp(-i angle)
        t.fre[e] = (float)re;
        t.fim[e] = (float)-im;
    }
    return t;
}
static __constant__ TwTable kTw32 = make_twiddles();

template <typename V> __device__ __forceinline__ V tw32(int e, int sgn);
template <> __device__ __forceinline__ float2 tw32<float2>(int e, int sgn) {
    return make_float2(kTw32.fre[e], sgn > 0 ? -kTw32.fim[e] : kTw32.fim[e]);
}
template <> __device__ __forceinline__ double2 tw32<double2>(int e, int sgn) {
    return make_double2(kTw32.re[e], sgn > 0 ? -kTw32.im[e] : kTw32.im[e]);
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__host__ __device__ constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; b++) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// Shared-memory load that the compiler may not hoist out of the tile loop (twiddles kept in
// registers across tiles would crowd out the transform's points).
__device__ __forceinline__ float2 lds_fresh(const float2 *p) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}
__device__ __forceinline__ double2 lds_fresh(const double2 *p) {
    double2 v;
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}

// Radix-2 decimation in frequency over R <= 32 points held in registers: on return x[i] holds
// output bitrev(i).  Twiddle exp(s 2 pi i e / R) from the compile-time table; 1 and s i are
// applied exactly.
template <int R, int SGN, bool WALSH, typename V>
__device__ __forceinline__ void dft_regs(V *x) {
    static_assert(R <= 32, "in-register transforms hold at most 32 points");
#pragma unroll
    for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * span) {
#pragma unroll
            for (int j = 0; j < span; j++) {
                const V u = x[b + j], v = x[b + j + span];
                x[b + j].x = u.x + v.x;
                x[b + j].y = u.y + v.y;
                V d;
                d.x = u.x - v.x;
                d.y = u.y - v.y;
                const int e = WALSH ? 0 : j * (R / (2 * span));
                if (4 * e == R) {
                    const auto t = d.x;
                    d.x = SGN > 0 ? -d.y : d.y;
                    d.y = SGN > 0 ? t : -t;
                } else if (e != 0) {
                    d = cmul(d, tw32<V>(e * (32 / R), SGN));
                }
                x[b + j + span] = d;
            }
        }
    }
}

template <typename R> struct MaxThreads { static constexpr int n = sizeof(R) == 4 ? 512 : 256; };

// KIND 0: DFT (output digits reversed by the radix-2 network), 1: Walsh-Hadamard (natural order),
// 2: DFT with the HHL inversion fused into its outputs (inv; contiguous fields only)
template <typename R, int K, int SGN, int KIND, bool CONTIG>
__global__ void __launch_bounds__(MaxThreads<R>::n) dft_kernel(const DftArgs a) {
    constexpr bool WALSH = KIND == 1;
    constexpr bool INV = KIND == 2 && CONTIG;
    using V = typename CV<R>::T;
    constexpr int k1 = K / 2, k2 = K - k1;
    constexpr int N1 = 1 << k1, N2 = 1 << k2, RR = N2 / N1;
    constexpr int KN = 1 << K;
    const int L = a.L, NL = 1 << L;
    const int nthr = N1 << L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [W] [S] [offset tables]
    V *Ws = reinterpret_cast<V *>(smem_raw);
    V *S = Ws + KN;
    // S: block of output digit a at a N1 2^L + (a / RR) 2^L: the 2^L-element gap between the
    // blocks of consecutive thread groups spreads pass 2's reads over the banks
    long long *fo_lo = reinterpret_cast<long long *>(S + (KN << L) + N1 * NL);
    long long *fo_hi = fo_lo + N1;
    long long *lane_off = fo_hi + N2;
    // twiddle tables after the offset tables, padded to a 16-byte boundary
    V *Tsm = reinterpret_cast<V *>(lane_off + NL + ((N1 + N2 + NL) & 1));
    const int ntlo = 1 << a.hT, nthi = 1 << (K + a.ns - a.hT);

    const int tid = threadIdx.x;
    const V *Wg = reinterpret_cast<const V *>(a.W);
    if (!WALSH)
        for (int i = tid; i < KN; i += nthr) Ws[i] = Wg[i];
    for (int i = tid; i < N1; i += nthr) {
        long long o = 0;
        for (int b = 0; b < k1; b++)
            if ((i >> b) & 1) o |= 1ll << a.fpos[b];
        fo_lo[i] = o;
    }
    for (int i = tid; i < N2; i += nthr) {
        long long o = 0;
        for (int b = 0; b < k2; b++)
            if ((i >> b) & 1) o |= 1ll << a.fpos[k1 + b];
        fo_hi[i] = o;
    }
    for (int i = tid; i < NL; i += nthr) {
        long long o = 0;
        for (int b = 0; b < L; b++)
            if ((i >> b) & 1) o |= 1ll << a.lpos[b];
        lane_off[i] = o;
    }
    if (a.tw_smem) {
        const V *tg = reinterpret_cast<const V *>(a.Tlo), *th = reinterpret_cast<const V *>(a.Thi);
        for (int i = tid; i < ntlo; i += nthr) Tsm[i] = tg[i];
        for (int i = tid; i < nthi; i += nthr) Tsm[ntlo + i] = th[i];
    }
    __syncthreads();

    // offsets are re-read from shared memory at every use: kept in registers across the tile
    // loop they would take 2 N2 registers
    const volatile long long *vlo = fo_lo;
    const volatile long long *vhi = fo_hi;
    const int l = tid & (NL - 1);
    const int u = tid >> L;  // pass 1: low field digit; pass 2: group of output digits a
    const int pad2 = u * NL;
    const V *Tlo = a.tw_smem ? Tsm : reinterpret_cast<const V *>(a.Tlo);
    const V *Thi = a.tw_smem ? Tsm + ntlo : reinterpret_cast<const V *>(a.Thi);
    const unsigned tmask = (1u << a.hT) - 1u;
    const R scale = (R)a.scale;
    V *psi = reinterpret_cast<V *>(a.psi);
    const V *qlo = reinterpret_cast<const V *>(a.qlo), *qhi = reinterpret_cast<const V *>(a.qhi);
    const unsigned long long qdm = (1ull << a.qnb) - 1ull, qcm = (1ull << a.qm) - 1ull, qhm = (1ull << a.qh) - 1ull;
    auto qphase_cd = [&](unsigned long long cv, unsigned long long d) -> V {
        return cmul(__ldg(qlo + (((cv & qhm) << a.qnb) + d)), __ldg(qhi + (((cv >> a.qh) << a.qnb) + d)));
    };
    auto qphase = [&](unsigned long long idx) -> V { return qphase_cd((idx >> a.qnb) & qcm, idx & qdm); };
    V x[N2];

    for (long long tix = blockIdx.x; tix < a.ntiles; tix += gridDim.x) {
        const unsigned long long base = insert_zero_bits((unsigned long long)tix, a.fix, a.nfix) + lane_off[l];
        unsigned long long kb = 0;  // clock value bits outside the field (inversion)
        if (INV)
            for (int sg = 0; sg < a.inv_nseg; sg++)
                kb |= ((base >> a.inv_src[sg]) & ((1ull << a.inv_w[sg]) - 1ull)) << a.inv_dst[sg];
        unsigned w = 0;
        for (int j = 0; j < a.ns; j++) w |= (unsigned)((base >> a.spos[j]) & 1ull) << j;
        // pass 1
        if (CONTIG) {
            const V *src = psi + base + ((unsigned long long)u << a.f0);
            const long long step = 1ll << (a.f0 + k1);
#pragma unroll
            for (int v = 0; v < N2; v++) x[v] = src[v * step];
        } else {
            const V *src = psi + base + vlo[u];
#pragma unroll
            for (int v = 0; v < N2; v++) x[v] = src[vhi[v]];
        }
        if (a.qmode == 1) {
            if (CONTIG && a.qrec) {
                // inputs at field values u + N1 v, one data index: the phase is P Q^v with
                // Q = the phase of clock value N1 2^(f0 - qnb)
                const unsigned long long i0 = base + ((unsigned long long)u << a.f0);
                const V Q = qphase_cd((unsigned long long)N1 << (a.f0 - a.qnb), i0 & qdm);
                V P{1, 0};
#pragma unroll
                for (int v = 0; v < N2; v++) {
                    if ((v & 7) == 0) P = qphase(i0 + ((unsigned long long)(N1 * v) << a.f0));
                    x[v] = cmul(x[v], P);
                    P = cmul(P, Q);
                }
            } else {
#pragma unroll
                for (int v = 0; v < N2; v++) {
                    const unsigned long long idx =
                        CONTIG ? base + ((unsigned long long)(u + N1 * v) << a.f0) : base + vlo[u] + vhi[v];
                    x[v] = cmul(x[v], qphase(idx));
                }
            }
        }
        if (a.twmode == 1) {
#pragma unroll
            for (int v = 0; v < N2; v++) {
                const unsigned q = w * (unsigned)(u + N1 * v);
                x[v] = cmul(x[v], cmul(Tlo[q & tmask], Thi[q >> a.hT]));
            }
        }
        dft_regs<N2, SGN, WALSH>(x);
        if (a.pf) {
            // this tile's inputs are in registers: pull a later tile's lines into L2 so that
            // DRAM stays busy through the transform and the stores (thread (u, l) takes the
            // runs of field values u + N1 v, v = l, l + 2^L, ...: each line once)
            const long long nt = tix + (long long)a.pf * gridDim.x;
            if (nt < a.ntiles) {
                const unsigned long long nb = insert_zero_bits((unsigned long long)nt, a.fix, a.nfix);
                for (int v = l; v < N2; v += NL) {
                    const unsigned long long off = CONTIG ? nb + ((unsigned long long)(u + N1 * v) << a.f0)
                                                          : nb + vlo[u] + vhi[v];
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(psi + off));
                }
            }
        }
#pragma unroll
        for (int i = 0; i < N2; i++) {
            const int aa = WALSH ? i : bitrev(i, k2);
            V y = x[i];
            if (!WALSH && aa != 0) y = cmul(y, lds_fresh(Ws + u * aa));  // u aa < 2^K
            S[((aa * N1 + u) << L) + l + (aa / RR) * NL] = y;
        }
        __syncthreads();
        // pass 2
#pragma unroll
        for (int r = 0; r < RR; r++) {
            const int aa = u * RR + r;
#pragma unroll
            for (int uu = 0; uu < N1; uu++) x[r * N1 + uu] = S[((aa * N1 + uu) << L) + l + pad2];
            dft_regs<N1, SGN, WALSH>(x + r * N1);
            // Walsh outputs N1 aa + i in natural order: their phases are P Q^i (see qrec)
            const bool qseq = WALSH && CONTIG && a.qmode == 2 && a.qrec;
            V P{1, 0}, Q{1, 0};
            const unsigned long long q0 = base + ((unsigned long long)(N1 * aa) << a.f0);
            if (qseq) Q = qphase_cd(1ull << (a.f0 - a.qnb), q0 & qdm);
#pragma unroll
            for (int i = 0; i < N1; i++) {
                const int y = WALSH ? i + N1 * aa : aa + N2 * bitrev(i, k1);
                V z = x[r * N1 + i];
                z.x *= scale;
                z.y *= scale;
                if (a.twmode == 2) {
                    const unsigned q = w * (unsigned)y;
                    z = cmul(z, cmul(Tlo[q & tmask], Thi[q >> a.hT]));
                }
                const unsigned long long oi =
                    CONTIG ? base + ((unsigned long long)y << a.f0) : base + vlo[y & (N1 - 1)] + vhi[y >> k1];
                if (qseq) {
                    if ((i & 7) == 0) P = qphase(q0 + ((unsigned long long)i << a.f0));
                    z = cmul(z, P);
                    P = cmul(P, Q);
                } else if (a.qmode == 2) {
                    z = cmul(z, qphase(oi));
                }
                if (INV) {
                    const unsigned long long kk = kb | ((unsigned long long)y << a.inv_fdst);
                    R sr = 0, cr = 1;
                    if (kk) {
                        const long long ks = (a.inv_twos && (kk >> (a.inv_nc - 1))) ? (long long)kk - (1ll << a.inv_nc)
                                                                                   : (long long)kk;
                        sr = (R)a.inv_Cs / (R)ks;
                        if (sr > (R)1) sr = (R)1;
                        if (sr < (R)-1) sr = (R)-1;
                        const R as = sr < 0 ? -sr : sr;
                        cr = sqrt(((R)1 - as) * ((R)1 + as));
                    }
                    psi[oi + (1ull << a.inv_bit)] = V{sr * z.x, sr * z.y};
                    z = V{cr * z.x, cr * z.y};
                }
                psi[oi] = z;
            }
        }
        __syncthreads();  // S is rewritten by the next tile's pass 1
    }
}

inline int num_sms_dft() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return sms;
}

template <typename R, int K, int SGN, int KIND>
void launch_kind(const DftArgs &a, bool contig, int threads, size_t smem, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        DFT_CUDA_OK(cudaFuncSetAttribute(dft_kernel<R, K, SGN, KIND, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        if constexpr (KIND != 2)
            DFT_CUDA_OK(cudaFuncSetAttribute(dft_kernel<R, K, SGN, KIND, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr = true;
    }
    auto kern = dft_kernel<R, K, SGN, KIND, true>;
    if constexpr (KIND != 2) {
        if (!contig) kern = dft_kernel<R, K, SGN, KIND, false>;
    } else {
        QSIM_REQUIRE(contig, "fused inversion needs a contiguous field");
    }
    int per_sm = 0;
    per_sm = occupancy_cached(reinterpret_cast<const void *>(kern), threads, smem);
    QSIM_REQUIRE(per_sm > 0, "Fourier pass does not fit on an SM");
    const long long grid = std::min<long long>(a.ntiles, (long long)num_sms_dft() * per_sm);
    kern<<<(int)grid, threads, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("dft_kernel: ") + cudaGetErrorString(e));
    note_launches(1, QSIM_KERNEL_FOURIER);
}

template <typename R, int K>
void launch_k(const DftArgs &a, int sign, int kind, bool contig, int threads, size_t smem, cudaStream_t st) {
    if (kind == 2) launch_kind<R, K, -1, 2>(a, contig, threads, smem, st);
    else if (kind == 1) launch_kind<R, K, 1, 1>(a, contig, threads, smem, st);
    else if (sign > 0) launch_kind<R, K, 1, 0>(a, contig, threads, smem, st);
    else launch_kind<R, K, -1, 0>(a, contig, threads, smem, st);
}

template <typename R>
void launch_dtype(const DftArgs &a, int K, int sign, int kind, bool contig, int threads, size_t smem,
                  cudaStream_t st) {
    switch (K) {
#define QSIM_DFT_K(k) \
    case k: launch_k<R, k>(a, sign, kind, contig, threads, smem, st); break;
        QSIM_DFT_K(1) QSIM_DFT_K(2) QSIM_DFT_K(3) QSIM_DFT_K(4) QSIM_DFT_K(5)
        QSIM_DFT_K(6) QSIM_DFT_K(7) QSIM_DFT_K(8) QSIM_DFT_K(9) QSIM_DFT_K(10)
#undef QSIM_DFT_K
        default: throw Error(QSIM_EINVAL, "Fourier pass wider than 10 qubits");
    }
}

}  // namespace dftk

// one per precision (dft_f32.cu, dft_f64.cu)
void dft_launch_f32(const dftk::DftArgs &a, int K, int sign, int kind, bool contig, int threads, size_t smem,
                    cudaStream_t st);
void dft_launch_f64(const dftk::DftArgs &a, int K, int sign, int kind, bool contig, int threads, size_t smem,
                    cudaStream_t st);

}  // namespace qsim
