// Tile-resident kernels that do more than one pass's work per visit of the state (complex64,
// sm_103a): two transforms of the same field per tile (the inverse QFT's last pass, the HHL
// inversion and the QFT's first pass; or a QFT pass, the structured phase and the Walsh-Hadamard
// pass), and a pass whose input is generated from the live part of the state instead of read
// (the clock's Hadamard layer on a field still |0>, the structured phase and the inverse QFT's
// first pass).  Same tile layout and transform steps as dft_tma.cu; every mbarrier wait is
// bounded and raises this file's device flag on timeout.
#include "dft_tma.cuh"

namespace qsim {

__device__ unsigned int g_dft_merge_error = 0;

namespace dftt {

// Two transforms of the same field in one tile (rows of 16 lanes, early next-tile load, thread
// stores): T1 (sign SGN1; a1's twiddle before or after) -> MID on its outputs -> T2 (SGN2, or a
// Walsh-Hadamard transform; a2's twiddle) -> outputs.  MID 1: the structured phase (a1's qmode
// tables) on T1's outputs; MID 2 / 3: the HHL inversion's cos / sin factor (a1's inv fields),
// the sin part written to the upper half (index + 2^inv_bit).  Between the transforms T1's
// outputs go back into the tile buffer in natural order [y][lane].
template <int K, int SGN1, int SGN2, bool WALSH2, int MID>
__global__ void __launch_bounds__(Shape<K, 4>::threads, Shape<K, 4>::min_blocks)
    dft2_tma_kernel(const __grid_constant__ CUtensorMap tmap, const DftArgs a1, const DftArgs a2, const TmaExtra x) {
    using S = Shape<K, 4>;
    constexpr int kL = 4, kNL = S::NL;
    constexpr int k1 = S::k1, k2 = S::k2, N1 = S::N1, N2 = S::N2, RR = S::RR, KN = 1 << K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [tile (1024-aligned)] [W1] [W2] [a1's twiddle tables] [mbarrier]
    const unsigned pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw + pad);
    float2 *W1 = buf + S::tile;
    float2 *W2 = W1 + KN;
    float2 *Tsm = W2 + KN;
    const int ntlo = 1 << a1.hT, nthi = 1 << (K + a1.ns - a1.hT);
    uint64_t *bar = reinterpret_cast<uint64_t *>(Tsm + (a1.tw_smem ? ntlo + nthi : 0));
    const unsigned bar_a = smem_u32(bar), buf_a = smem_u32(buf);
    const int tid = threadIdx.x;
    const int l = tid & (kNL - 1);
    const int u = tid >> kL;
    for (int i = tid; i < KN; i += S::threads) {
        W1[i] = reinterpret_cast<const float2 *>(a1.W)[i];
        if (!WALSH2) W2[i] = reinterpret_cast<const float2 *>(a2.W)[i];
    }
    if (a1.tw_smem) {
        const float2 *tg = reinterpret_cast<const float2 *>(a1.Tlo), *th = reinterpret_cast<const float2 *>(a1.Thi);
        for (int i = tid; i < ntlo; i += S::threads) Tsm[i] = tg[i];
        for (int i = tid; i < nthi; i += S::threads) Tsm[ntlo + i] = th[i];
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const float2 *T1lo = a1.tw_smem ? Tsm : reinterpret_cast<const float2 *>(a1.Tlo);
    const float2 *T1hi = a1.tw_smem ? Tsm + ntlo : reinterpret_cast<const float2 *>(a1.Thi);
    const float2 *T2lo = reinterpret_cast<const float2 *>(a2.Tlo), *T2hi = reinterpret_cast<const float2 *>(a2.Thi);
    const unsigned tmask1 = (1u << a1.hT) - 1u, tmask2 = (1u << a2.hT) - 1u;
    const float2 *qlo = reinterpret_cast<const float2 *>(a1.qlo), *qhi = reinterpret_cast<const float2 *>(a1.qhi);
    const unsigned long long qdm = (1ull << a1.qnb) - 1ull, qcm = (1ull << a1.qm) - 1ull, qhm = (1ull << a1.qh) - 1ull;
    auto qphase_cd = [&](unsigned long long cv, unsigned long long d) -> float2 {
        return cmul(__ldg(qlo + (((cv & qhm) << a1.qnb) + d)), __ldg(qhi + (((cv >> a1.qh) << a1.qnb) + d)));
    };
    auto qphase = [&](unsigned long long idx) -> float2 { return qphase_cd((idx >> a1.qnb) & qcm, idx & qdm); };
    const unsigned long long gapm = (1ull << x.gap) - 1ull;
    const unsigned tx_bytes = (unsigned)(S::tile * sizeof(float2));
    auto coords = [&](long long t, int &c1, int &c4) {
        c1 = (int)((unsigned long long)t & gapm);
        c4 = (int)((unsigned long long)t >> x.gap);
    };
    float2 *psi = reinterpret_cast<float2 *>(a1.psi);
    auto issue_load = [&](long long t) {
        int c1, c4;
        coords(t, c1, c4);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar_a), "r"(tx_bytes) : "memory");
        tma_load(buf_a, &tmap, c1, c4, bar_a);
    };
    // step 1 of a transform on the buffer: column u of lane l, optional input twiddle, the
    // N2-point transform, the inner twiddle, then written back transposed (swizzled rows)
    auto step1 = [&](float2(&v)[N2], int sgn_walsh, const float2 *Ws, int twmode, unsigned w, const float2 *Tlo,
                     const float2 *Thi, unsigned tmask, int hT) {
        (void)sgn_walsh;
#pragma unroll
        for (int q = 0; q < N2; q++) v[q] = buf[(u + N1 * q) * kNL + l];
        if (twmode == 1) {
#pragma unroll
            for (int q = 0; q < N2; q++) {
                const unsigned e = w * (unsigned)(u + N1 * q);
                v[q] = cmul(v[q], cmul(Tlo[e & tmask], Thi[e >> hT]));
            }
        }
    };
    bool failed = false;
    float2 v[N2];
    unsigned it = 0;
    if (tid == 0 && (long long)blockIdx.x < x.ntiles) issue_load(blockIdx.x);
    for (long long t = blockIdx.x; t < x.ntiles; t += gridDim.x, it++) {
        int c1, c4;
        coords(t, c1, c4);
        const bool ok = mbar_wait(bar_a, it & 1u);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            const long long tn = t + 2 * (long long)gridDim.x;
            if (tn < x.ntiles) {
                int n1, n4;
                coords(tn, n1, n4);
                tma_prefetch_l2(&tmap, n1, n4);
            }
        }
        const unsigned long long base = (unsigned long long)l | ((unsigned long long)c1 << kL) |
                                        ((unsigned long long)c4 << (a1.f0 + K));
        unsigned long long kb = 0;
        if (MID >= 2)
            for (int sg = 0; sg < a1.inv_nseg; sg++)
                kb |= ((base >> a1.inv_src[sg]) & ((1ull << a1.inv_w[sg]) - 1ull)) << a1.inv_dst[sg];
        unsigned w1 = 0, w2 = 0;
        for (int j = 0; j < a1.ns; j++) w1 |= (unsigned)((base >> a1.spos[j]) & 1ull) << j;
        for (int j = 0; j < a2.ns; j++) w2 |= (unsigned)((base >> a2.spos[j]) & 1ull) << j;
        // ---------------- T1
        step1(v, 0, W1, a1.twmode, w1, T1lo, T1hi, tmask1, a1.hT);
        dft_regs<N2, SGN1, false>(v);
#pragma unroll
        for (int i = 0; i < N2; i++) {
            const int aa = bitrev(i, k2);
            if (aa != 0) v[i] = cmul(v[i], dftk::lds_fresh(W1 + u * aa));
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < N2; i++) {
            const int aa = bitrev(i, k2);
            buf[(aa * N1 + (u ^ ((aa / RR) & 1))) * kNL + l] = v[i];
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RR; r++) {
            const int aa = u * RR + r;
#pragma unroll
            for (int uu = 0; uu < N1; uu++) v[r * N1 + uu] = buf[(aa * N1 + (uu ^ (u & 1))) * kNL + l];
        }
        __syncthreads();  // the buffer takes T1's outputs next
#pragma unroll
        for (int r = 0; r < RR; r++) dft_regs<N1, SGN1, false>(v + r * N1);
        const float scale1 = (float)a1.scale;
#pragma unroll
        for (int r = 0; r < RR; r++) {
            const int aa = u * RR + r;
#pragma unroll
            for (int i = 0; i < N1; i++) {
                const int y = aa + N2 * bitrev(i, k1);
                float2 z = v[r * N1 + i];
                z.x *= scale1;
                z.y *= scale1;
                if (a1.twmode == 2) {
                    const unsigned e = w1 * (unsigned)y;
                    z = cmul(z, cmul(T1lo[e & tmask1], T1hi[e >> a1.hT]));
                }
                if (MID == 1) {
                    z = cmul(z, qphase(base + ((unsigned long long)y << a1.f0)));
                } else {
                    const unsigned long long kk = kb | ((unsigned long long)y << a1.inv_fdst);
                    float f = MID == 2 ? 1.f : 0.f;
                    if (kk) {
                        const long long ks = (a1.inv_twos && (kk >> (a1.inv_nc - 1))) ? (long long)kk - (1ll << a1.inv_nc)
                                                                                     : (long long)kk;
                        const float sr = fminf(fmaxf((float)a1.inv_Cs / (float)ks, -1.f), 1.f);
                        if (MID == 3) f = sr;
                        else {
                            const float as = fabsf(sr);
                            f = sqrtf((1.f - as) * (1.f + as));
                        }
                    }
                    z.x *= f;
                    z.y *= f;
                }
                buf[y * kNL + l] = z;
            }
        }
        __syncthreads();
        // ---------------- T2 on the same buffer
        step1(v, 0, W2, a2.twmode, w2, T2lo, T2hi, tmask2, a2.hT);
        dft_regs<N2, SGN2, WALSH2>(v);
        if (!WALSH2) {
#pragma unroll
            for (int i = 0; i < N2; i++) {
                const int aa = bitrev(i, k2);
                if (aa != 0) v[i] = cmul(v[i], dftk::lds_fresh(W2 + u * aa));
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < N2; i++) {
            const int aa = WALSH2 ? i : bitrev(i, k2);
            buf[(aa * N1 + (u ^ ((aa / RR) & 1))) * kNL + l] = v[i];
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RR; r++) {
            const int aa = u * RR + r;
#pragma unroll
            for (int uu = 0; uu < N1; uu++) v[r * N1 + uu] = buf[(aa * N1 + (uu ^ (u & 1))) * kNL + l];
        }
        __syncthreads();  // the buffer is free: the next tile's load overlaps T2's step 2
        if (tid == 0 && t + gridDim.x < x.ntiles) issue_load(t + gridDim.x);
#pragma unroll
        for (int r = 0; r < RR; r++) dft_regs<N1, SGN2, WALSH2>(v + r * N1);
        const float scale2 = (float)a2.scale;
        const unsigned long long out_off = MID == 3 ? (1ull << a1.inv_bit) : 0ull;
#pragma unroll
        for (int r = 0; r < RR; r++) {
            const int aa = u * RR + r;
#pragma unroll
            for (int i = 0; i < N1; i++) {
                const int y = WALSH2 ? i + N1 * aa : aa + N2 * bitrev(i, k1);
                float2 z = v[r * N1 + i];
                z.x *= scale2;
                z.y *= scale2;
                if (a2.twmode == 2) {
                    const unsigned e = w2 * (unsigned)y;
                    z = cmul(z, cmul(T2lo[e & tmask2], T2hi[e >> a2.hT]));
                }
                psi[base + ((unsigned long long)y << a1.f0) + out_off] = z;
            }
        }
    }
    if (tid == 0 && failed) {
        atomicOr(&g_dft_merge_error, 1u);
        mbar_wait(bar_a, it & 1u);  // the load that did not arrive may still land
    }
}

// A Fourier pass whose input is generated instead of read: the field (qubits f0 .. f0+K-1) is
// still |0> and the state below it is live (w = f0), and the pass is preceded by H on every field
// qubit (the Walsh-Hadamard layer of the phase estimation) and the structured phase.  The input
// of the pass at index i is then 2^(-K/2) psi[i mod 2^f0] exp(i lambda_d t c), so each thread
// reads one live amplitude, steps the phase along the field (as a geometric sequence, refreshed
// from the tables every 8 terms: complex64) and runs the transform; the outputs (with the pass's
// twiddle and scale) fill the 2^(f0+K)-amplitude state.  Rows of 16 lanes; no bulk copy is
// needed (nothing of the field is read).  The output at field value 0 overwrites the live
// amplitude it was generated from, but only after the step-1 barrier, when every thread of the
// tile has read it.
template <int K, int SGN>
__global__ void __launch_bounds__(Shape<K, 4>::threads, Shape<K, 4>::min_blocks) dft_gen_kernel(const DftArgs a, long long ntiles) {
    using S = Shape<K, 4>;
    constexpr int kL = 4, kNL = S::NL;
    constexpr int k1 = S::k1, k2 = S::k2, N1 = S::N1, N2 = S::N2, RR = S::RR, KN = 1 << K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *Ws = buf + S::tile;
    float2 *Tsm = Ws + KN;
    const int ntlo = 1 << a.hT, nthi = 1 << (K + a.ns - a.hT);
    const int tid = threadIdx.x;
    const int l = tid & (kNL - 1);
    const int u = tid >> kL;
    for (int i = tid; i < KN; i += S::threads) Ws[i] = reinterpret_cast<const float2 *>(a.W)[i];
    if (a.tw_smem) {
        const float2 *tg = reinterpret_cast<const float2 *>(a.Tlo), *th = reinterpret_cast<const float2 *>(a.Thi);
        for (int i = tid; i < ntlo; i += S::threads) Tsm[i] = tg[i];
        for (int i = tid; i < nthi; i += S::threads) Tsm[ntlo + i] = th[i];
    }
    __syncthreads();
    const float2 *Tlo = a.tw_smem ? Tsm : reinterpret_cast<const float2 *>(a.Tlo);
    const float2 *Thi = a.tw_smem ? Tsm + ntlo : reinterpret_cast<const float2 *>(a.Thi);
    const unsigned tmask = (1u << a.hT) - 1u;
    const float2 *qlo = reinterpret_cast<const float2 *>(a.qlo), *qhi = reinterpret_cast<const float2 *>(a.qhi);
    const unsigned long long qdm = (1ull << a.qnb) - 1ull, qcm = (1ull << a.qm) - 1ull, qhm = (1ull << a.qh) - 1ull;
    auto qphase_cd = [&](unsigned long long cv, unsigned long long d) -> float2 {
        return cmul(__ldg(qlo + (((cv & qhm) << a.qnb) + d)), __ldg(qhi + (((cv >> a.qh) << a.qnb) + d)));
    };
    auto qphase = [&](unsigned long long idx) -> float2 { return qphase_cd((idx >> a.qnb) & qcm, idx & qdm); };
    float2 *psi = reinterpret_cast<float2 *>(a.psi);
    const float s_in = (float)a.scale;  // the Walsh-Hadamard layer on |0>: 2^(-K/2)
    const float scale = (float)a.scale;
    float2 v[N2];
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const unsigned long long base = (unsigned long long)l | ((unsigned long long)t << kL);  // < 2^f0
        unsigned w = 0;
        for (int j = 0; j < a.ns; j++) w |= (unsigned)((base >> a.spos[j]) & 1ull) << j;
        // step 1: inputs at field values u + N1 q
        {
            const float2 p0 = psi[base];
            const float2 z0 = make_float2(s_in * p0.x, s_in * p0.y);
            const unsigned long long i0 = base + ((unsigned long long)u << a.f0);
            const float2 Q = qphase_cd((unsigned long long)N1 << (a.f0 - a.qnb), i0 & qdm);
            float2 P{1.f, 0.f};
#pragma unroll
            for (int q = 0; q < N2; q++) {
                if ((q & 7) == 0) P = qphase(i0 + ((unsigned long long)(N1 * q) << a.f0));
                v[q] = cmul(z0, P);
                P = cmul(P, Q);
            }
        }
        if (a.twmode == 1) {
#pragma unroll
            for (int q = 0; q < N2; q++) {
                const unsigned e = w * (unsigned)(u + N1 * q);
                v[q] = cmul(v[q], cmul(Tlo[e & tmask], Thi[e >> a.hT]));
            }
        }
        dft_regs<N2, SGN, false>(v);
#pragma unroll
        for (int i = 0; i < N2; i++) {
            const int aa = bitrev(i, k2);
            if (aa != 0) v[i] = cmul(v[i], dftk::lds_fresh(Ws + u * aa));
        }
        __syncthreads();  // the previous tile's step 2 has read the buffer; every thread has read psi[base]
#pragma unroll
        for (int i = 0; i < N2; i++) {
            const int aa = bitrev(i, k2);
            buf[(aa * N1 + (u ^ ((aa / RR) & 1))) * kNL + l] = v[i];
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RR; r++) {
            const int aa = u * RR + r;
#pragma unroll
            for (int uu = 0; uu < N1; uu++) v[r * N1 + uu] = buf[(aa * N1 + (uu ^ (u & 1))) * kNL + l];
            dft_regs<N1, SGN, false>(v + r * N1);
        }
#pragma unroll
        for (int r = 0; r < RR; r++) {
            const int aa = u * RR + r;
#pragma unroll
            for (int i = 0; i < N1; i++) {
                const int y = aa + N2 * bitrev(i, k1);
                float2 z = v[r * N1 + i];
                z.x *= scale;
                z.y *= scale;
                if (a.twmode == 2) {
                    const unsigned e = w * (unsigned)y;
                    z = cmul(z, cmul(Tlo[e & tmask], Thi[e >> a.hT]));
                }
                psi[base + ((unsigned long long)y << a.f0)] = z;
            }
        }
    }
}

template <int K, int SGN1, int SGN2, bool WALSH2, int MID>
void launch2(const CUtensorMap &map, const DftArgs &a1, const DftArgs &a2, const TmaExtra &x, size_t smem,
             cudaStream_t st) {
    using S = Shape<K, 4>;
    auto kern = dft2_tma_kernel<K, SGN1, SGN2, WALSH2, MID>;
    static bool attr = false;
    if (!attr) {
        DFT_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr = true;
    }
    int per_sm = 0;
    per_sm = occupancy_cached(reinterpret_cast<const void *>(kern), S::threads, smem);
    QSIM_REQUIRE(per_sm > 0, "merged Fourier passes do not fit on an SM");
    const long long grid = std::min<long long>(x.ntiles, (long long)num_sms() * per_sm);
    kern<<<(int)grid, S::threads, smem, st>>>(map, a1, a2, x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("dft2_tma_kernel: ") + cudaGetErrorString(e));
    note_launches(1, QSIM_KERNEL_FOURIER_TMA);
}

template <int K, int SGN>
void launch_gen(const DftArgs &a, long long ntiles, size_t smem, cudaStream_t st) {
    using S = Shape<K, 4>;
    auto kern = dft_gen_kernel<K, SGN>;
    static bool attr = false;
    if (!attr) {
        DFT_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr = true;
    }
    int per_sm = 0;
    per_sm = occupancy_cached(reinterpret_cast<const void *>(kern), S::threads, smem);
    QSIM_REQUIRE(per_sm > 0, "generated-input Fourier pass does not fit on an SM");
    const long long grid = std::min<long long>(ntiles, (long long)num_sms() * per_sm);
    kern<<<(int)grid, S::threads, smem, st>>>(a, ntiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("dft_gen_kernel: ") + cudaGetErrorString(e));
    note_launches(1, QSIM_KERNEL_FOURIER_TMA);
}
}  // namespace dftt

unsigned dft_merge_read_error() {
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_dft_merge_error, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}

void dft_merge_clear_error() {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_dft_merge_error, &z, sizeof(z)) != cudaSuccess) cudaGetLastError();
}

// Two passes on one field (run_dft2): T1 = args1's pass, T2 = args2's pass, both with a
// contiguous field of 9 or 10 qubits at qubit 4 or above; rows of 16 lanes.  merge 1: DFT(-1),
// inversion factor (part 0 cos in place, part 1 sin into the upper half), DFT(+1); merge 2:
// DFT(+1), structured phase, Walsh-Hadamard.  False (nothing launched) when the shape does not fit.
bool dft2_tma_launch(const void *args1, const void *args2, int n, int K, int merge, int part, int promo,
                     cudaStream_t st) {
    using namespace dftt;
    const DftArgs &b1 = *static_cast<const DftArgs *>(args1);
    const DftArgs &b2 = *static_cast<const DftArgs *>(args2);
    constexpr int kL = 4;
    if (K < 9 || K > 10) return false;
    const int f0 = b1.f0;
    if (f0 < kL || f0 + K > n || b2.f0 != f0) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (enc == nullptr || (reinterpret_cast<uintptr_t>(b1.psi) & 15) != 0) return false;
    const int klo = (K + 1) / 2, khi = K - klo;
    const int gap = f0 - kL, above = n - f0 - K;
    if (gap > 30 || above > 30) return false;
    cuuint64_t dims[5] = {(cuuint64_t)2 << kL, (cuuint64_t)1 << gap, (cuuint64_t)1 << klo, (cuuint64_t)1 << khi,
                          (cuuint64_t)1 << above};
    const cuuint64_t amp = 8;
    cuuint64_t strides[4] = {amp << kL, amp << f0, amp << (f0 + klo), amp << (f0 + K)};
    cuuint32_t box[5] = {(cuuint32_t)(2 << kL), 1u, (cuuint32_t)1 << klo, (cuuint32_t)1 << khi, 1u};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUtensorMapL2promotion prom[4] = {CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B};
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, b1.psi, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, prom[std::min(std::max(promo, 0), 3)], CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return false;
    DftArgs a1 = b1, a2 = b2;
    a1.L = a2.L = kL;
    a2.tw_smem = 0;
    TmaExtra x;
    x.gap = gap;
    x.above = above;
    x.inv_c4 = 0;
    x.ntiles = 1ll << (n - K - kL);
    x.pf = 1;
    size_t smem = (((size_t)1 << K) << kL) * 8 + 2 * ((size_t)1 << K) * 8;
    const int ntw = a1.ns > 0 ? (1 << a1.hT) + (1 << (K + a1.ns - a1.hT)) : 0;
    a1.tw_smem = 0;
    if (ntw > 0 && smem + (size_t)ntw * 8 + 16 + 1024 <= 220 * 1024) {
        a1.tw_smem = 1;
        smem += (size_t)ntw * 8;
    }
    smem += 16 + 1024;
    if (merge == 1) {
        if (part == 1) K == 10 ? launch2<10, -1, 1, false, 3>(map, a1, a2, x, smem, st) : launch2<9, -1, 1, false, 3>(map, a1, a2, x, smem, st);
        else K == 10 ? launch2<10, -1, 1, false, 2>(map, a1, a2, x, smem, st) : launch2<9, -1, 1, false, 2>(map, a1, a2, x, smem, st);
        return true;
    }
    if (merge == 2) {
        K == 10 ? launch2<10, 1, 1, true, 1>(map, a1, a2, x, smem, st) : launch2<9, 1, 1, true, 1>(map, a1, a2, x, smem, st);
        return true;
    }
    return false;
}

// The generated-input pass (dft_gen_kernel): `args` is the pass (field f0 .. f0+K-1, f0 = the
// live width w, the structured phase in its qmode fields with the recurrence), the state is
// live below f0 and |0> on the field; it becomes live up to f0 + K.  False (nothing launched)
// when the shape does not fit.
bool dft_gen_launch(const void *args, int w, int K, int sign, cudaStream_t st) {
    using namespace dftt;
    const DftArgs &b = *static_cast<const DftArgs *>(args);
    if (K < 9 || K > 10 || b.f0 != w || w < 4 || !b.qrec || b.qmode == 0) return false;
    DftArgs a = b;
    a.L = 4;
    const long long ntiles = 1ll << (w - 4);
    size_t smem = (((size_t)1 << K) << 4) * 8 + ((size_t)1 << K) * 8;
    const int ntw = a.ns > 0 ? (1 << a.hT) + (1 << (K + a.ns - a.hT)) : 0;
    a.tw_smem = 0;
    if (ntw > 0 && smem + (size_t)ntw * 8 <= 200 * 1024) {
        a.tw_smem = 1;
        smem += (size_t)ntw * 8;
    }
    if (sign > 0) K == 10 ? launch_gen<10, 1>(a, ntiles, smem, st) : launch_gen<9, 1>(a, ntiles, smem, st);
    else K == 10 ? launch_gen<10, -1>(a, ntiles, smem, st) : launch_gen<9, -1>(a, ntiles, smem, st);
    return true;
}

}  // namespace qsim
