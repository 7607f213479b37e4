// Host side of the Fourier-transform passes: twiddle tables, tile layout and launch (the
// kernels are in dft_impl.cuh, compiled once per precision by dft_f32.cu and dft_f64.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dft_impl.cuh"

namespace qsim {
namespace {

using dftk::DftArgs;
using dftk::kMaxK;
using dftk::kMaxLane;
using dftk::kMaxSrc;

int lane_bits_default(int dtype, int k1) {
    // 2^L amplitudes = 128 bytes per HBM run; at least 64 threads; at most the thread cap
    const int want = dtype == QSIM_C128 ? 3 : 4;
    const int cap_log = dtype == QSIM_C128 ? 8 : 9;  // log2 of MaxThreads
    return std::min(std::max(want, 6 - k1), cap_log - k1);
}

}  // namespace

int dft_table_split(int K, int ns) { return (K + ns) / 2; }

void dft_tables(const Op &op, std::vector<cd> &W, std::vector<cd> &Tlo, std::vector<cd> &Thi) {
    const int K = (int)op.targets.size(), ns = (int)op.controls.size();
    const int hT = dft_table_split(K, ns);
    const double two_pi = 6.283185307179586476925286766559;
    // angles reduced exactly: j / 2^b is exact in binary, only the final multiply rounds
    auto unit = [&](unsigned long long j, int bits) {
        return std::polar(1.0, op.sign * two_pi * std::ldexp((double)j, -bits));
    };
    W.resize((size_t)1 << K);
    for (size_t j = 0; j < W.size(); j++) W[j] = unit(j, K);
    Tlo.resize((size_t)1 << hT);
    for (size_t j = 0; j < Tlo.size(); j++) Tlo[j] = unit(j, K + ns);
    Thi.resize((size_t)1 << (K + ns - hT));
    for (size_t j = 0; j < Thi.size(); j++) Thi[j] = unit(j << hT, K + ns);
}

// The pass arguments shared by every pass kernel: tables, twiddle mode, the structured phase
// (qop, qmode) and the inversion (inv).  False when the inversion cannot be carried by the pass.
static bool dft_common_args(DftArgs &a, void *state, int n, int dtype, const Op &op, const void *tables,
                            const Op *qop, const void *qlo, const void *qhi, int qmode, const Op *inv) {
    const int K = (int)op.targets.size(), ns = (int)op.controls.size();
    QSIM_REQUIRE(K >= 1 && K <= kMaxK && ns <= kMaxSrc && K + ns <= 30 && K <= n, "Fourier pass shape");
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    const size_t vb = dtype == QSIM_C128 ? 16 : 8;
    const int hT = dft_table_split(K, ns);
    const unsigned char *t = static_cast<const unsigned char *>(tables);
    a.W = t;
    a.Tlo = t + vb * ((size_t)1 << K);
    a.Thi = t + vb * (((size_t)1 << K) + ((size_t)1 << hT));
    a.hT = hT;
    a.ns = ns;
    a.twmode = ns == 0 ? 0 : (op.pre ? 1 : 2);
    if (qop != nullptr && qmode != 0) {
        a.qmode = qmode;
        a.qlo = qlo;
        a.qhi = qhi;
        a.qnb = (int)qop->targets.size();
        a.qm = (int)qop->controls.size();
        a.qh = (a.qm + 1) / 2;  // the split qpe_phase_tables uses
        bool contig_field = true;
        for (int j = 0; j < K; j++) contig_field = contig_field && op.targets[j] == op.targets[0] + j;
        // complex64 only: the recurrence rounds differently from the tables, which complex128's
        // 1e-12 state tolerance at 20+ clock qubits (phase angles near 1e7 rad) does not allow
        a.qrec = dtype == QSIM_C64 && contig_field && op.targets[0] >= a.qnb && op.targets[0] + K <= a.qnb + a.qm
                     ? 1 : 0;
        for (int i = 0; i < a.qnb; i++) QSIM_REQUIRE(qop->targets[i] == i, "phase estimation: data qubits must be 0..nb-1");
        for (int j = 0; j < a.qm; j++)
            QSIM_REQUIRE(qop->controls[j] == a.qnb + j, "phase estimation: clock qubits must follow the data");
    }
    if (inv != nullptr) {
        // the rotation reads the clock value through runs of consecutive qubits; the field must
        // be one contiguous piece of one run (its bits then land on consecutive bits of k)
        bool contig_field = true;
        for (int j = 0; j < K; j++) contig_field = contig_field && op.targets[j] == op.targets[0] + j;
        if (!contig_field || inv->targets[0] != n || op.kind != OP_DFT || op.sign != -1) return false;
        a.inv = 1;
        a.inv_bit = n;
        a.inv_Cs = inv->tq;
        a.inv_nc = (int)inv->controls.size();
        a.inv_twos = inv->sign == -1 ? 1 : 0;
        a.inv_fdst = -1;
        for (int j = 0; j < a.inv_nc;) {
            int wd = 1;
            while (j + wd < a.inv_nc && inv->controls[j + wd] == inv->controls[j] + wd) wd++;
            if (a.inv_nseg == 8) return false;
            a.inv_src[a.inv_nseg] = inv->controls[j];
            a.inv_w[a.inv_nseg] = wd;
            a.inv_dst[a.inv_nseg] = j;
            if (op.targets[0] >= inv->controls[j] && op.targets[0] + K <= inv->controls[j] + wd)
                a.inv_fdst = j + (op.targets[0] - inv->controls[j]);
            a.inv_nseg++;
            j += wd;
        }
        if (a.inv_fdst < 0) return false;
    }
    a.scale = std::ldexp(1.0, -K / 2) * ((K & 1) ? std::sqrt(0.5) : 1.0);
    for (int j = 0; j < K; j++) a.fpos[j] = op.targets[j];
    for (int j = 0; j < ns; j++) a.spos[j] = op.controls[j];
    a.f0 = op.targets[0];
    return true;
}

static bool contiguous_field(const Op &op) {
    for (size_t j = 0; j < op.targets.size(); j++)
        if (op.targets[j] != op.targets[0] + (int)j) return false;
    return true;
}

bool run_dft(void *state, int n, int dtype, const Op &op, const void *tables, cudaStream_t st, const Op *qop,
             const void *qlo, const void *qhi, int qmode, const Op *inv) {
    const int K = (int)op.targets.size(), ns = (int)op.controls.size();
    DftArgs a;
    if (!dft_common_args(a, state, n, dtype, op, tables, qop, qlo, qhi, qmode, inv)) return false;
    const size_t vb = dtype == QSIM_C128 ? 16 : 8;
    const int hT = a.hT;
    const int k1 = K / 2;
    const bool contig = contiguous_field(op);
    const int kind = op.kind == OP_WALSH ? 1 : (a.inv ? 2 : 0);
    // complex64 with a contiguous field: the bulk-copy tile kernel, when the table selects it
    // and the shape fits
    if (const int variant = dtype == QSIM_C64 && contig ? tune_get(QSIM_C64, QSIM_TUNE_DFT_TMA, n) : 0) {
        DftArgs t = a;
        t.hT = hT;
        t.tw_smem = 0;
        if (dft_tma_launch(&t, n, K, op.sign, kind, variant, tune_get(QSIM_C64, QSIM_TUNE_DFT_L2PROMO, n),
                           tune_get(QSIM_C64, QSIM_TUNE_DFT_PREFETCH, n), st))
            return true;
    }
    int L = std::min(lane_bits_default(dtype, k1), n - K);
    if (const int v = tune_get(dtype, QSIM_TUNE_DFT_LANES, n))
        L = std::min({v, n - K, (dtype == QSIM_C128 ? 8 : 9) - k1, kMaxLane});
    L = std::max(L, 0);
    unsigned long long fmask = 0;
    for (int q : op.targets) fmask |= 1ull << q;
    std::vector<int> fix(op.targets.begin(), op.targets.end());
    int cnt = 0;
    for (int q = 0; q < n && cnt < L; q++)
        if (!((fmask >> q) & 1ull)) {
            a.lpos[cnt++] = q;
            fix.push_back(q);
        }
    a.L = L;
    {
        const bool lanes_low = (fmask & ((1ull << L) - 1ull)) == 0;
        const int dist = tune_get(dtype, QSIM_TUNE_DFT_PREFETCH, n);  // tiles ahead
        a.pf = (lanes_low && ((size_t)vb << L) == 128) ? dist : 0;
    }
    std::sort(fix.begin(), fix.end());
    a.nfix = (int)fix.size();
    for (int i = 0; i < a.nfix; i++) a.fix[i] = fix[i];
    a.ntiles = 1ll << (n - K - L);
    const int N1 = 1 << k1, N2 = 1 << (K - k1), NL = 1 << L;
    const int threads = N1 << L;
    size_t smem = vb * (((size_t)1 << K) + ((size_t)1 << (K + L)) + (size_t)N1 * NL) +
                  8 * ((size_t)N1 + N2 + NL + ((N1 + N2 + NL) & 1));
    // twiddle tables in shared memory when they fit (they are read once per amplitude)
    const size_t tw_bytes = vb * (((size_t)1 << hT) + ((size_t)1 << (K + ns - hT)));
    if (ns > 0 && smem + tw_bytes <= 200 * 1024) {
        a.tw_smem = 1;
        smem += tw_bytes;
    }
    if (dtype == QSIM_C128) dft_launch_f64(a, K, op.sign, kind, contig, threads, smem, st);
    else dft_launch_f32(a, K, op.sign, kind, contig, threads, smem, st);
    return true;
}

// Two passes on the same contiguous field in one tile-resident kernel (complex64, bulk-copy
// tiles), when the table selects the 128-byte-row kernel and the shapes fit:
//   merge 1: the inverse QFT's last pass (sign -1), the HHL inversion on the ancilla right above
//            the live state, and the QFT's first pass (sign +1) over the same field: launched
//            twice, first the sin part into the unwritten upper half, then the cos part in place;
//   merge 2: a QFT pass (sign +1), the structured phase (diagonal) and the Walsh-Hadamard pass
//            of the same field.
// Returns false (nothing launched) when the shapes do not fit.
bool run_dft2(void *state, int n, int dtype, int merge, const Op &op1, const void *tab1, const Op &mid,
              const void *qlo, const void *qhi, const Op &op2, const void *tab2, cudaStream_t st) {
    if (dtype != QSIM_C64 || tune_get(QSIM_C64, QSIM_TUNE_DFT_TMA, n) < 3) return false;
    if (!((tune_get(QSIM_C64, QSIM_TUNE_DFT_MERGE, n) >> merge) & 1)) return false;
    if (!contiguous_field(op1) || op1.targets != op2.targets) return false;
    const int K = (int)op1.targets.size();
    if (K < 9 || K > 10) return false;
    DftArgs a1, a2;
    if (merge == 1) {
        if (op1.kind != OP_DFT || op1.sign != -1 || op2.kind != OP_DFT || op2.sign != 1 || mid.kind != OP_HHL_INVERT)
            return false;
        for (int q : op2.controls)
            if (q >= n) return false;
        if (!dft_common_args(a1, state, n, dtype, op1, tab1, nullptr, nullptr, nullptr, 0, &mid)) return false;
        if (!dft_common_args(a2, state, n, dtype, op2, tab2, nullptr, nullptr, nullptr, 0, nullptr)) return false;
        // the sin part reads the lower half and fills the upper one; then the cos part in place
        for (int part = 1; part >= 0; part--)
            if (!dft2_tma_launch(&a1, &a2, n, K, merge, part, tune_get(QSIM_C64, QSIM_TUNE_DFT_L2PROMO, n), st))
                return false;
        return true;
    }
    if (merge == 2) {
        if (op1.kind != OP_DFT || op1.sign != 1 || op2.kind != OP_WALSH || mid.kind != OP_QPE_PHASE) return false;
        if (!dft_common_args(a1, state, n, dtype, op1, tab1, &mid, qlo, qhi, 2, nullptr)) return false;
        if (!dft_common_args(a2, state, n, dtype, op2, tab2, nullptr, nullptr, nullptr, 0, nullptr)) return false;
        return dft2_tma_launch(&a1, &a2, n, K, merge, 0, tune_get(QSIM_C64, QSIM_TUNE_DFT_L2PROMO, n), st);
    }
    return false;
}

// The pass `op` on a field right above the live width w that is still |0>, after H on that
// field and the structured phase qop (complex64, fields of 9-10 qubits): inputs generated from
// the live amplitudes, outputs over 2^(w + K) amplitudes.  False when the shape does not fit.
bool run_dft_generated(void *state, int w, int dtype, const Op &op, const void *tables, const Op &qop,
                       const void *qlo, const void *qhi, cudaStream_t st) {
    if (dtype != QSIM_C64 || op.kind != OP_DFT || !contiguous_field(op) || op.targets[0] != w) return false;
    const int nw = w + (int)op.targets.size();
    if (tune_get(QSIM_C64, QSIM_TUNE_DFT_TMA, nw) < 3 || !(tune_get(QSIM_C64, QSIM_TUNE_DFT_MERGE, nw) & 1)) return false;
    for (int q : op.controls)
        if (q >= w) return false;
    const int K = (int)op.targets.size();
    DftArgs a;
    if (!dft_common_args(a, state, w + K, dtype, op, tables, &qop, qlo, qhi, 1, nullptr)) return false;
    return dft_gen_launch(&a, w, K, op.sign, st);
}

}  // namespace qsim
