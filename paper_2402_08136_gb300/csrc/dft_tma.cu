// Fourier and Walsh-Hadamard passes on a complex64 state with the tile staged by the Tensor
// Memory Accelerator (sm_103a): one cp.async.bulk.tensor load of the whole 2^K x 8 tile into
// shared memory, the two-step transform in registers through the same buffer, one bulk tensor
// store back.  The operation is the one of dft_impl.cuh (qsim_circuit_add_dft / _add_walsh: the
// inverse QFT and QFT of the phase estimation as Cooley-Tukey passes, Sec. III-A and Fig. 5,
// and the clock's Hadamard layers), with the same options: the structured phase-estimation
// diagonal on the inputs or outputs, the twiddle before or after, and the HHL inversion
// rotation writing both halves of the state.
//
// Why a second kernel: with the loads issued by the threads, a 2^10 x 16 tile held one 512-thread
// CTA per SM, and every tile went load -> transform -> store behind two CTA-wide barriers with
// nothing else on the SM to cover them.  Here the copy engine moves the tile (no per-thread
// address arithmetic or load instructions), the tile is 2^10 x 8 amplitudes (64 KB, in place,
// no separate exchange buffer), and two or more CTAs share each SM, so one CTA's transform
// overlaps another's copies; the next tile's lines are prefetched into L2 by a bulk tensor
// prefetch as soon as a tile has landed.
//
// Layout.  The field must be contiguous (qubits f0 .. f0+K-1) and above the 3 lowest qubits (the
// lanes: 8 consecutive amplitudes, 64 bytes).  The state is described to the copy engine as a
// 5-dimensional tensor of floats (innermost first): the 8 lanes (16 floats), the qubits between
// the lanes and the field, the low and high halves of the field (box dimensions stay <= 256),
// and the qubits above the field; a tile is the box {16, 1, 2^klo, 2^khi, 1} at coordinates
// (0, c1, 0, 0, c4), landing in shared memory as [field value y][lane].
//
// The transform (2^K = N1 N2, y = u + N1 v, as in dft_impl.cuh):
//   step 1  thread (lane l, u) reads its N2 points v from the tile, transforms them in registers,
//           multiplies by the inner twiddle and, after a barrier, writes them back in place at
//           (a N1 + (u ^ s(a))) x 8 + l for output digit a (s(a) = bit 0 of the thread group of
//           a: a bank swizzle for step 2's reads);
//   step 2  thread (lane l, group g) reads the N1 points of each of its digits a, transforms
//           them, applies the scale, twiddle, phase or inversion, and after a barrier writes
//           output y' into [y'][l], which the bulk store copies back to HBM.
// Every wait on the tile's mbarrier is bounded (1 s of %globaltimer); on timeout the kernel
// raises a device flag (read by qsim_device_status), waits (bounded) for its own copies and
// returns.
#include "dft_tma.cuh"

namespace qsim {

__device__ unsigned int g_dft_tma_error = 0;

namespace dftt {

// KIND 0: DFT, 1: Walsh-Hadamard, 2: DFT with the HHL inversion on its outputs.
// EARLY: the outputs leave by thread stores straight from registers, and the next tile's bulk
// load is issued as soon as step 2 has read the buffer, so that copy overlaps step 2's
// transform and stores; otherwise the outputs go back through the buffer and a bulk store,
// and the next load waits for that store to have read the buffer.
// TW (twiddle mode 0 none, 1 before, 2 after) and QS (structured phase: 0 none, 1 inputs with
// the recurrence, 2 outputs of a Walsh-Hadamard pass with the recurrence) fix the options at
// compile time (3: read from the arguments), so each common pass runs a kernel without the
// code of the options it does not use.
template <int K, int L, int SGN, int KIND, bool EARLY, int TW, int QS>
__global__ void __launch_bounds__(Shape<K, L>::threads, Shape<K, L>::min_blocks)
    dft_tma_kernel(const __grid_constant__ CUtensorMap tmap, const DftArgs a, const TmaExtra x) {
    using S = Shape<K, L>;
    const int twmode = TW == 3 ? a.twmode : TW;
    const int qmode = QS == 3 ? a.qmode : QS;
    const int qrec = QS == 3 ? a.qrec : (QS != 0);
    constexpr int kL = L, kNL = S::NL;
    constexpr bool WALSH = KIND == 1;
    constexpr bool INV = KIND == 2;
    constexpr int k1 = S::k1, k2 = S::k2, N1 = S::N1, N2 = S::N2, RR = S::RR, KN = 1 << K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [tile (1024-aligned)] [W] [twiddle tables] [phase steps] [mbarrier]
    // phase recurrence through a step table: QS 1 along the inputs u + N1 q of a column, QS 2 on a
    // transform along the outputs aa + N2 j of a thread (stride PST, PCNT terms, NR refresh points)
    constexpr bool PT = QS == 1 || (QS == 2 && KIND == 0);
    constexpr int PST = QS == 1 ? S::N1 : S::N2, PCNT = QS == 1 ? S::N2 : S::N1;
    constexpr int NR = (PCNT + 7) / 8;
    const unsigned pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw + pad);
    float2 *Ws = buf + S::tile;
    float2 *Tsm = Ws + KN;
    const int ntlo = 1 << a.hT, nthi = 1 << (K + a.ns - a.hT);
    // for every data index d, the phase of the clock step between consecutive terms ([d][0]) and
    // of the steps to the refresh points ([d][j], j >= 1): the recurrence then needs one table
    // read per sequence instead of one per refresh point
    float2 *Psm = Tsm + (a.tw_smem ? ntlo + nthi : 0);
    uint64_t *bar = reinterpret_cast<uint64_t *>(Psm + (PT ? (NR << a.qnb) : 0));
    const unsigned bar_a = smem_u32(bar), buf_a = smem_u32(buf);
    const int tid = threadIdx.x;
    const int l = tid & (kNL - 1);
    const int u = tid >> kL;  // step 1: low field digit; step 2: group of output digits
    const float2 *Wg = reinterpret_cast<const float2 *>(a.W);
    if (!WALSH)
        for (int i = tid; i < KN; i += S::threads) Ws[i] = Wg[i];
    if (a.tw_smem) {
        const float2 *tg = reinterpret_cast<const float2 *>(a.Tlo), *th = reinterpret_cast<const float2 *>(a.Thi);
        for (int i = tid; i < ntlo; i += S::threads) Tsm[i] = tg[i];
        for (int i = tid; i < nthi; i += S::threads) Tsm[ntlo + i] = th[i];
    }
    if (PT) {
        const float2 *ql = reinterpret_cast<const float2 *>(a.qlo), *qh = reinterpret_cast<const float2 *>(a.qhi);
        const unsigned long long hm = (1ull << a.qh) - 1ull;
        for (int i = tid; i < (NR << a.qnb); i += S::threads) {
            const int d = i / NR, j = i % NR;
            const unsigned long long cv = (unsigned long long)(j == 0 ? PST : PST * 8 * j) << (a.f0 - a.qnb);
            Psm[i] = cmul(ql[((cv & hm) << a.qnb) + d], qh[((cv >> a.qh) << a.qnb) + d]);
        }
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const float2 *Tlo = a.tw_smem ? Tsm : reinterpret_cast<const float2 *>(a.Tlo);
    const float2 *Thi = a.tw_smem ? Tsm + ntlo : reinterpret_cast<const float2 *>(a.Thi);
    const unsigned tmask = (1u << a.hT) - 1u;
    const float scale = (float)a.scale;
    const float2 *qlo = reinterpret_cast<const float2 *>(a.qlo), *qhi = reinterpret_cast<const float2 *>(a.qhi);
    const unsigned long long qdm = (1ull << a.qnb) - 1ull, qcm = (1ull << a.qm) - 1ull, qhm = (1ull << a.qh) - 1ull;
    auto qphase_cd = [&](unsigned long long cv, unsigned long long d) -> float2 {
        return cmul(__ldg(qlo + (((cv & qhm) << a.qnb) + d)), __ldg(qhi + (((cv >> a.qh) << a.qnb) + d)));
    };
    auto qphase = [&](unsigned long long idx) -> float2 { return qphase_cd((idx >> a.qnb) & qcm, idx & qdm); };
    const unsigned long long gapm = (1ull << x.gap) - 1ull;
    const unsigned tx_bytes = (unsigned)(S::tile * sizeof(float2));
    auto coords = [&](long long t, int &c1, int &c4) {
        c1 = (int)((unsigned long long)t & gapm);
        c4 = (int)((unsigned long long)t >> x.gap);
    };
    float2 *psi = reinterpret_cast<float2 *>(a.psi);
    auto issue_load = [&](long long t) {
        int c1, c4;
        coords(t, c1, c4);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar_a), "r"(tx_bytes) : "memory");
        tma_load(buf_a, &tmap, c1, c4, bar_a);
    };
    bool failed = false;
    float2 v[N2];
    unsigned it = 0;
    if (EARLY && tid == 0 && (long long)blockIdx.x < x.ntiles) issue_load(blockIdx.x);
    for (long long t = blockIdx.x; t < x.ntiles; t += gridDim.x, it++) {
        int c1, c4;
        coords(t, c1, c4);
        if (!EARLY && tid == 0) {
            tma_store_wait_read();  // the previous tile's store has read the buffer
            issue_load(t);
        }
        // every thread waits for the tile itself (the copy's completion makes it visible to the
        // thread that observes it); the decision to give up is taken together at the first barrier
        // index of this thread's amplitude at field value 0
        const unsigned long long base = (unsigned long long)l | ((unsigned long long)c1 << kL) |
                                        ((unsigned long long)c4 << (a.f0 + K));
        // the structured phase on the inputs (QS 1): the table reads do not depend on the tile's
        // data, so they are issued before the wait for it and their latency overlaps the copy
        float2 Qp{1.f, 0.f}, P0{1.f, 0.f};
        const float2 *ps = Psm;
        if (QS == 1) {
            const unsigned long long i0 = base + ((unsigned long long)u << a.f0);
            P0 = qphase(i0);
            ps = Psm + (i0 & qdm) * NR;
        }
        const bool ok = mbar_wait(bar_a, it & 1u);
        if (tid == 0 && x.pf > 0) {
            // L2 prefetch of a tile whose load is not issued yet (pf tiles of this CTA ahead)
            const long long tn = t + (EARLY ? x.pf + 1 : x.pf) * (long long)gridDim.x;
            if (tn < x.ntiles) {
                int n1, n4;
                coords(tn, n1, n4);
                tma_prefetch_l2(&tmap, n1, n4);
            }
        }
        unsigned long long kb = 0;  // clock value bits outside the field (inversion)
        if (INV)
            for (int sg = 0; sg < a.inv_nseg; sg++)
                kb |= ((base >> a.inv_src[sg]) & ((1ull << a.inv_w[sg]) - 1ull)) << a.inv_dst[sg];
        unsigned w = 0;
        for (int j = 0; j < a.ns; j++) w |= (unsigned)((base >> a.spos[j]) & 1ull) << j;
        // step 1
#pragma unroll
        for (int q = 0; q < N2; q++) v[q] = buf[(u + N1 * q) * kNL + l];
        if (QS == 1) {
            // inputs at field values u + N1 q: phase P0 Q^q, restarted every 8 terms from P0 times
            // the step to the refresh point (at most 8 FP32 products from an exact table value)
            Qp = ps[0];
            float2 P{1.f, 0.f};
#pragma unroll
            for (int q = 0; q < N2; q++) {
                if ((q & 7) == 0) P = q == 0 ? P0 : cmul(P0, ps[q / 8]);
                v[q] = cmul(v[q], P);
                P = cmul(P, Qp);
            }
        } else if (qmode == 1) {
            const unsigned long long i0 = base + ((unsigned long long)u << a.f0);
            if (qrec) {
                // inputs at field values u + N1 q: the phase is P Q^q, Q = the phase of clock
                // value N1 2^(f0 - qnb) (refreshed from the tables every 8 terms)
                const float2 Q = qphase_cd((unsigned long long)N1 << (a.f0 - a.qnb), i0 & qdm);
                float2 P{1.f, 0.f};
#pragma unroll
                for (int q = 0; q < N2; q++) {
                    if ((q & 7) == 0) P = qphase(i0 + ((unsigned long long)(N1 * q) << a.f0));
                    v[q] = cmul(v[q], P);
                    P = cmul(P, Q);
                }
            } else {
#pragma unroll
                for (int q = 0; q < N2; q++) v[q] = cmul(v[q], qphase(i0 + ((unsigned long long)(N1 * q) << a.f0)));
            }
        }
        if (TW == 1) {
            // the input twiddle exp(s 2 pi i w (u + N1 q) / 2^(K+ns)) is geometric in q: one
            // complex product per input, restarted from the tables every 8 terms
            const unsigned e1 = w * (unsigned)N1;
            const float2 Qt = cmul(Tlo[e1 & tmask], Thi[e1 >> a.hT]);
            float2 P{1.f, 0.f};
#pragma unroll
            for (int q = 0; q < N2; q++) {
                if ((q & 7) == 0) {
                    const unsigned e = w * (unsigned)(u + N1 * q);
                    P = cmul(Tlo[e & tmask], Thi[e >> a.hT]);
                }
                v[q] = cmul(v[q], P);
                P = cmul(P, Qt);
            }
        } else if (twmode == 1) {
#pragma unroll
            for (int q = 0; q < N2; q++) {
                const unsigned e = w * (unsigned)(u + N1 * q);
                v[q] = cmul(v[q], cmul(Tlo[e & tmask], Thi[e >> a.hT]));
            }
        }
        dft_regs<N2, SGN, WALSH>(v);
        if (!WALSH) {
#pragma unroll
            for (int i = 0; i < N2; i++) {
                const int aa = bitrev(i, k2);
                if (aa != 0) v[i] = cmul(v[i], dftk::lds_fresh(Ws + u * aa));  // u aa < 2^K
            }
        }
        if (__syncthreads_or(!ok)) {  // every thread has read its step-1 points (or one gave up)
            failed = true;
            break;
        }
#pragma unroll
        for (int i = 0; i < N2; i++) {
            const int aa = WALSH ? i : bitrev(i, k2);
            const int sw = (aa / RR) & 1;
            buf[(aa * N1 + (u ^ sw)) * kNL + l] = v[i];
        }
        __syncthreads();
        // step 2: thread group u takes output digits aa = u RR + r
#pragma unroll
        for (int r = 0; r < RR; r++) {
            const int aa = u * RR + r;
            const int sw = u & 1;
#pragma unroll
            for (int uu = 0; uu < N1; uu++) v[r * N1 + uu] = buf[(aa * N1 + (uu ^ sw)) * kNL + l];
        }
        __syncthreads();  // every thread has read its step-2 points: the buffer is free
        if (EARLY && tid == 0 && t + gridDim.x < x.ntiles) issue_load(t + gridDim.x);
        // the structured phase on a transform's outputs (QS 2): outputs aa + N2 j of group aa
        // take P(aa) R^j; P(aa) is read from the tables before the transform, whose arithmetic
        // covers the latency
        constexpr bool DSEQ = QS == 2 && KIND == 0;
        float2 Pa[RR];
        if (DSEQ) {
#pragma unroll
            for (int r = 0; r < RR; r++) Pa[r] = qphase(base + ((unsigned long long)(u * RR + r) << a.f0));
        }
#pragma unroll
        for (int r = 0; r < RR; r++) dft_regs<N1, SGN, WALSH>(v + r * N1);
#pragma unroll
        for (int r = 0; r < RR; r++) {
            const int aa = u * RR + r;
            const bool qseq = WALSH && qmode == 2 && qrec;
            float2 P{1.f, 0.f}, Q{1.f, 0.f};
            const unsigned long long q0 = base + ((unsigned long long)(N1 * aa) << a.f0);
            if (qseq) Q = qphase_cd(1ull << (a.f0 - a.qnb), q0 & qdm);
            const float2 *pd = Psm + (base & qdm) * NR;
            if (DSEQ) Q = pd[0];
#pragma unroll
            for (int jj = 0; jj < N1; jj++) {
                // DSEQ visits the outputs in the order of j (output aa + N2 j sits in v[bitrev(j)])
                const int i = DSEQ ? bitrev(jj, k1) : jj;
                const int y = WALSH ? i + N1 * aa : aa + N2 * bitrev(i, k1);
                float2 z = v[r * N1 + i];
                z.x *= scale;
                z.y *= scale;
                if (twmode == 2) {
                    const unsigned e = w * (unsigned)y;
                    z = cmul(z, cmul(Tlo[e & tmask], Thi[e >> a.hT]));
                }
                if (DSEQ) {
                    if ((jj & 7) == 0) P = jj == 0 ? Pa[r] : cmul(Pa[r], pd[jj / 8]);
                    z = cmul(z, P);
                    P = cmul(P, Q);
                } else if (qseq) {
                    if ((i & 7) == 0) P = qphase(q0 + ((unsigned long long)i << a.f0));
                    z = cmul(z, P);
                    P = cmul(P, Q);
                } else if (qmode == 2) {
                    z = cmul(z, qphase(base + ((unsigned long long)y << a.f0)));
                }
                if (EARLY) {
                    const unsigned long long oi = base + ((unsigned long long)y << a.f0);
                    if (INV) {
                        const unsigned long long kk = kb | ((unsigned long long)y << a.inv_fdst);
                        float sr = 0.f, cr = 1.f;
                        if (kk) {
                            const long long ks = (a.inv_twos && (kk >> (a.inv_nc - 1))) ? (long long)kk - (1ll << a.inv_nc)
                                                                                       : (long long)kk;
                            sr = fminf(fmaxf((float)a.inv_Cs / (float)ks, -1.f), 1.f);
                            const float as = fabsf(sr);
                            cr = sqrtf((1.f - as) * (1.f + as));
                        }
                        psi[oi + (1ull << a.inv_bit)] = make_float2(sr * z.x, sr * z.y);
                        z = make_float2(cr * z.x, cr * z.y);
                    }
                    psi[oi] = z;
                    continue;
                }
                if (INV) {
                    // keep z for the upper half; the buffer takes the lower half's cos part first
                    v[r * N1 + i] = z;
                    const unsigned long long kk = kb | ((unsigned long long)y << a.inv_fdst);
                    float cr = 1.f;
                    if (kk) {
                        const long long ks = (a.inv_twos && (kk >> (a.inv_nc - 1))) ? (long long)kk - (1ll << a.inv_nc)
                                                                                   : (long long)kk;
                        float sr = (float)a.inv_Cs / (float)ks;
                        sr = fminf(fmaxf(sr, -1.f), 1.f);
                        const float as = fabsf(sr);
                        cr = sqrtf((1.f - as) * (1.f + as));
                    }
                    z.x *= cr;
                    z.y *= cr;
                }
                buf[y * kNL + l] = z;
            }
        }
        if (EARLY) continue;
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) tma_store(&tmap, c1, c4, buf_a);
        if (INV) {
            // the upper half (ancilla 1) takes r z: wait until the store has read the buffer
            if (tid == 0) tma_store_wait_read();
            __syncthreads();
#pragma unroll
            for (int r = 0; r < RR; r++) {
                const int aa = u * RR + r;
#pragma unroll
                for (int i = 0; i < N1; i++) {
                    const int y = aa + N2 * bitrev(i, k1);
                    const unsigned long long kk = kb | ((unsigned long long)y << a.inv_fdst);
                    float sr = 0.f;
                    if (kk) {
                        const long long ks = (a.inv_twos && (kk >> (a.inv_nc - 1))) ? (long long)kk - (1ll << a.inv_nc)
                                                                                   : (long long)kk;
                        sr = fminf(fmaxf((float)a.inv_Cs / (float)ks, -1.f), 1.f);
                    }
                    const float2 z = v[r * N1 + i];
                    buf[y * kNL + l] = make_float2(sr * z.x, sr * z.y);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            if (tid == 0) tma_store(&tmap, c1, c4 + x.inv_c4, buf_a);
        }
    }
    if (tid == 0) {
        if (failed) {
            atomicOr(&g_dft_tma_error, 1u);
            // the load that did not arrive may still land: give it (bounded) time before exit
            mbar_wait(bar_a, it & 1u);
        }
        tma_store_wait_all();
    }
}

// ------------------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return sms;
}

template <int K, int L, int SGN, int KIND, bool EARLY, int TW = 3, int QS = 3>
void launch(const CUtensorMap &map, const DftArgs &a, const TmaExtra &x, size_t smem, cudaStream_t st) {
    using S = Shape<K, L>;
    auto kern = dft_tma_kernel<K, L, SGN, KIND, EARLY, TW, QS>;
    static bool attr = false;
    if (!attr) {
        DFT_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr = true;
    }
    int per_sm = 0;
    per_sm = occupancy_cached(reinterpret_cast<const void *>(kern), S::threads, smem);
    QSIM_REQUIRE(per_sm > 0, "Fourier pass (bulk-copy tiles) does not fit on an SM");
    const long long grid = std::min<long long>(x.ntiles, (long long)num_sms() * per_sm);
    kern<<<(int)grid, S::threads, smem, st>>>(map, a, x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("dft_tma_kernel: ") + cudaGetErrorString(e));
    note_launches(1, QSIM_KERNEL_FOURIER_TMA);
}

template <int K, int L, bool EARLY>
void launch_k(const CUtensorMap &map, const DftArgs &a, const TmaExtra &x, int sign, int kind, size_t smem,
              cudaStream_t st) {
    if constexpr (EARLY && L == 4) {
        // the passes of the phase estimation, each with a kernel of its own options
        const int qs = a.qmode == 0 ? 0 : (a.qrec && a.qmode == 1 ? 1 : (a.qrec && a.qmode == 2 && kind != 2 ? 2 : 3));
        const int tw = a.twmode;
        if (kind == 2 && tw == 0 && qs == 0) return launch<K, L, -1, 2, EARLY, 0, 0>(map, a, x, smem, st);
        if (kind == 1 && tw == 0 && qs == 0) return launch<K, L, 1, 1, EARLY, 0, 0>(map, a, x, smem, st);
        if (kind == 1 && tw == 0 && qs == 1) return launch<K, L, 1, 1, EARLY, 0, 1>(map, a, x, smem, st);
        if (kind == 1 && tw == 0 && qs == 2) return launch<K, L, 1, 1, EARLY, 0, 2>(map, a, x, smem, st);
        if (kind == 0 && sign < 0 && tw == 2 && qs == 0) return launch<K, L, -1, 0, EARLY, 2, 0>(map, a, x, smem, st);
        if (kind == 0 && sign < 0 && tw == 0 && qs == 0) return launch<K, L, -1, 0, EARLY, 0, 0>(map, a, x, smem, st);
        if (kind == 0 && sign > 0 && tw == 0 && qs == 0) return launch<K, L, 1, 0, EARLY, 0, 0>(map, a, x, smem, st);
        if (kind == 0 && sign > 0 && tw == 1 && qs == 0) return launch<K, L, 1, 0, EARLY, 1, 0>(map, a, x, smem, st);
        if (kind == 0 && sign > 0 && tw == 2 && qs == 0) return launch<K, L, 1, 0, EARLY, 2, 0>(map, a, x, smem, st);
        if (kind == 0 && sign > 0 && tw == 0 && qs == 2) return launch<K, L, 1, 0, EARLY, 0, 2>(map, a, x, smem, st);
    }
    if (kind == 2) launch<K, L, -1, 2, EARLY>(map, a, x, smem, st);
    else if (kind == 1) launch<K, L, 1, 1, EARLY>(map, a, x, smem, st);
    else if (sign > 0) launch<K, L, 1, 0, EARLY>(map, a, x, smem, st);
    else launch<K, L, -1, 0, EARLY>(map, a, x, smem, st);
}


}  // namespace dftt

unsigned dft_tma_read_error() {
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_dft_tma_error, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}

void dft_tma_clear_error() {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_dft_tma_error, &z, sizeof(z)) != cudaSuccess) cudaGetLastError();
}

// The complex64 pass `a` (built by run_dft for a state of n qubits) through the bulk-copy
// kernel (variant 1: bulk load and bulk store; 2: bulk load issued early, thread stores), when
// its shape allows: a contiguous field of 9 or 10 qubits starting at qubit 3 or
// above, the lanes on qubits 0..2.  kind: 0 DFT, 1 Walsh-Hadamard, 2 DFT with the inversion
// (inv_bit = n, the ancilla right above the state).  Returns false when the shape does not
// fit (the caller then runs dft_kernel).
bool dft_tma_launch(const void *args, int n, int K, int sign, int kind, int variant, int promo, int prefetch,
                    cudaStream_t st) {
    using namespace dftt;
    const DftArgs &a0 = *static_cast<const DftArgs *>(args);
    if (K < 9 || K > 10 || variant < 1 || variant > 4) return false;
    const int kL = variant <= 2 ? 3 : 4, kNL = 1 << kL;
    const bool early = variant == 2 || variant == 4;
    const int f0 = a0.f0;
    if (f0 < kL || f0 + K > n) return false;
    for (int j = 0; j < K; j++)
        if (a0.fpos[j] != f0 + j) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (enc == nullptr) return false;
    if ((reinterpret_cast<uintptr_t>(a0.psi) & 15) != 0) return false;
    const int nt = kind == 2 ? n + 1 : n;  // the inversion writes the upper half too
    const int klo = (K + 1) / 2, khi = K - klo;
    const int gap = f0 - kL, above = nt - f0 - K;
    if (gap > 30 || above > 30) return false;
    cuuint64_t dims[5] = {(cuuint64_t)2 * kNL, (cuuint64_t)1 << gap, (cuuint64_t)1 << klo, (cuuint64_t)1 << khi,
                          (cuuint64_t)1 << above};
    const cuuint64_t amp = 8;  // bytes per complex64 amplitude
    cuuint64_t strides[4] = {amp << kL, amp << f0, amp << (f0 + klo), amp << (f0 + K)};
    cuuint32_t box[5] = {(cuuint32_t)(2 * kNL), 1u, (cuuint32_t)1 << klo, (cuuint32_t)1 << khi, 1u};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    const CUtensorMapL2promotion prom[4] = {CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, a0.psi, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, prom[std::min(std::max(promo, 0), 3)],
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    DftArgs a = a0;
    a.L = kL;
    TmaExtra x;
    x.gap = gap;
    x.above = above;
    x.inv_c4 = kind == 2 ? 1 << (n - f0 - K) : 0;
    x.ntiles = 1ll << (n - K - kL);
    x.pf = prefetch;
    const size_t tile_bytes = ((size_t)1 << K) * kNL * 8;
    const int ntw = a.ns > 0 ? (1 << a.hT) + (1 << (K + a.ns - a.hT)) : 0;
    size_t smem = tile_bytes + ((size_t)1 << K) * 8;
    a.tw_smem = 0;
    if (ntw > 0 && smem + (size_t)ntw * 8 + 16 <= (kL == 3 ? 110 : 200) * 1024) {
        a.tw_smem = 1;
        smem += (size_t)ntw * 8;
    }
    if (kL == 4 && early && a.qrec && (a.qmode == 1 || (a.qmode == 2 && kind == 0))) {
        if (a.qnb > 10) return false;
        smem += (size_t)8 * 4 << a.qnb;  // phase steps of the recurrence (at most 32 / 8 = 4 per data index)
    }
    smem += 16 + 1024;  // mbarrier, alignment slack
    if (kL == 3) {
        if (early) K == 10 ? launch_k<10, 3, true>(map, a, x, sign, kind, smem, st) : launch_k<9, 3, true>(map, a, x, sign, kind, smem, st);
        else K == 10 ? launch_k<10, 3, false>(map, a, x, sign, kind, smem, st) : launch_k<9, 3, false>(map, a, x, sign, kind, smem, st);
    } else {
        if (early) K == 10 ? launch_k<10, 4, true>(map, a, x, sign, kind, smem, st) : launch_k<9, 4, true>(map, a, x, sign, kind, smem, st);
        else K == 10 ? launch_k<10, 4, false>(map, a, x, sign, kind, smem, st) : launch_k<9, 4, false>(map, a, x, sign, kind, smem, st);
    }
    return true;
}

}  // namespace qsim
