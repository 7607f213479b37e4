// HHL circuit construction and solution readout (Sec. III-A "Practical HHL procedures",
// Fig. 5 conceptual circuit, Sec. III-B resource estimate).
#include <algorithm>
#include <cmath>
#include <memory>

#include "common.h"

namespace qsim {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// Sec. III-B: n_QPE = max(n_data + 1, ceil(log2(kappa + 1))).
int qpe_formula(int n_data, double kappa) {
    return std::max(n_data + 1, (int)std::ceil(std::log2(kappa + 1.0)));
}

void add_u(qsim_circuit &c, std::vector<int> targets, std::vector<int> controls, std::vector<cd> U) {
    Gate g;
    g.kind = GATE_U;
    g.targets = std::move(targets);
    g.controls = std::move(controls);
    g.U = std::move(U);
    c.gates.push_back(std::move(g));
}

std::vector<cd> hadamard() {
    const double r = 1.0 / std::sqrt(2.0);
    return {r, r, r, -r};
}

std::vector<cd> cphase(double phi) {
    return {1.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, std::polar(1.0, phi)};
}

std::vector<cd> swap2() {
    return {1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0};
}

std::vector<cd> adjoint(const std::vector<cd> &U) {
    const int d = (int)std::lround(std::sqrt((double)U.size()));
    std::vector<cd> out(U.size());
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) out[(size_t)c * d + r] = std::conj(U[(size_t)r * d + c]);
    return out;
}

// Inverse quantum Fourier transform on `q` (q[j] = bit j of the register value).  The forward
// transform maps |x> to 2^{-m/2} sum_k exp(2 pi i x k / 2^m) |k>; its circuit handles the
// most significant qubit first (H, then controlled phases 2 pi / 2^(d+1) from the qubit d
// places below), followed by the bit-reversal swaps.  The inverse runs that sequence
// backwards with conjugated phases.
void append_iqft(qsim_circuit &c, const std::vector<int> &q) {
    const int m = (int)q.size();
    for (int j = m / 2 - 1; j >= 0; j--) add_u(c, {q[j], q[m - 1 - j]}, {}, swap2());
    for (int j = 0; j < m; j++) {
        for (int l = 0; l < j; l++) add_u(c, {q[l], q[j]}, {}, cphase(-2.0 * kPi / std::ldexp(1.0, j - l + 1)));
        add_u(c, {q[j]}, {}, hadamard());
    }
}

// Inverse of a gate of the phase estimation (dense: adjoint; Fourier pass: opposite sign with
// the twiddle moved to the other side of the transform).
Gate inverse_gate(const Gate &g) {
    Gate r = g;
    if (g.kind == GATE_DFT) {
        r.sign = -g.sign;
        r.pre = 1 - g.pre;
    } else if (g.kind != GATE_WALSH) {  // a Walsh-Hadamard pass is its own inverse
        r.U = adjoint(g.U);
    }
    return r;
}

// Fields of at most 10 clock qubits for the Fourier and Walsh-Hadamard passes, top field first:
// [lo, hi) ranges of register bit positions.
std::vector<std::pair<int, int>> clock_fields(int m) {
    std::vector<std::pair<int, int>> f;
    int rem = m;
    while (rem > 0) {
        const int parts = (rem + 9) / 10;
        const int k = (rem + parts - 1) / parts;
        f.push_back({rem - k, rem});
        rem -= k;
    }
    return f;
}

// H on every clock qubit: m Hadamard gates, or one Walsh-Hadamard pass per field (the passes
// commute; low_first emits the lowest field first, so that on the clock register's |0> each pass
// fills the qubits right above those already filled).
void append_hadamards(qsim_circuit &c, const std::vector<int> &q, bool passes, bool low_first = false) {
    if (!passes) {
        for (int x : q) add_u(c, {x}, {}, hadamard());
        return;
    }
    std::vector<std::pair<int, int>> fields = clock_fields((int)q.size());
    if (low_first) std::reverse(fields.begin(), fields.end());
    for (const auto &f : fields) {
        Gate g;
        g.kind = GATE_WALSH;
        g.targets.assign(q.begin() + f.first, q.begin() + f.second);
        c.gates.push_back(std::move(g));
    }
}

// Inverse QFT on `q` as Cooley-Tukey passes (Cooley & Tukey 1965): the DFT of size 2^m with
// sign -1 factors into a DFT over the top field of the register followed by the twiddle
// exp(-2 pi i u a / 2^m) (u = value of the bits below the field, a = the field's output
// digit), then the same factorisation of the remaining lower bits.  Fields hold at most 10
// qubits.  The result holds the register value v with its digits in field order: the top field
// carries the lowest digits of v.  Returns that order (bit j of v <-> order[j]).
std::vector<int> append_iqft_passes(qsim_circuit &c, const std::vector<int> &q) {
    std::vector<int> order;
    for (const auto &f : clock_fields((int)q.size())) {
        Gate g;
        g.kind = GATE_DFT;
        g.targets.assign(q.begin() + f.first, q.begin() + f.second);
        g.controls.assign(q.begin(), q.begin() + f.first);
        g.sign = -1;
        g.pre = 0;
        c.gates.push_back(g);
        order.insert(order.end(), g.targets.begin(), g.targets.end());
    }
    return order;
}

hhl_circuit *build_from_spectrum(int N, const std::vector<double> &lamA, const std::vector<cd> &VA,
                                 const std::vector<cd> &b, int n_clock, double t, double C, int flags) {
    double amax = 0.0, amin = 1e300;
    for (double l : lamA) {
        amax = std::max(amax, std::fabs(l));
        amin = std::min(amin, std::fabs(l));
    }
    QSIM_REQUIRE(amin > 1e-14 * amax && amin > 0.0, "A is singular");
    // an indefinite A reads the clock register as two's complement: its top bit is the sign
    // qubit n_negval of Sec. III-B
    const bool is_signed = lamA.front() < 0.0;
    std::unique_ptr<hhl_circuit> h(new hhl_circuit());
    h->N = N;
    // step 1: normalize b
    double nb2 = 0.0;
    for (const cd &z : b) nb2 += std::norm(z);
    QSIM_REQUIRE(nb2 > 0.0, "b must be nonzero");
    h->norm_b = std::sqrt(nb2);
    // step 1(b): pad to a power of two with block-diag(A, max|lambda| I)
    int nb = 1;
    while ((1 << nb) < N) nb++;
    const int D = 1 << nb;
    h->nb = nb;
    h->lam_min = lamA.front();
    h->lam_max = lamA.back();
    std::vector<double> lam(D);
    std::vector<cd> V((size_t)D * D, cd(0.0, 0.0));
    for (int i = 0; i < N; i++) {
        lam[i] = lamA[i];
        for (int r = 0; r < N; r++) V[(size_t)r * D + i] = VA[(size_t)r * N + i];
    }
    for (int i = N; i < D; i++) {
        lam[i] = amax;
        V[(size_t)i * D + i] = 1.0;
    }
    h->b_pad.assign(D, cd(0.0, 0.0));
    for (int i = 0; i < N; i++) h->b_pad[i] = b[i] / h->norm_b;
    // Sec. III-B resources
    const double kappa = amax / amin;
    const int n_data = nb, n_neg = is_signed ? 1 : 0;
    h->n_total_formula = n_data + qpe_formula(n_data, kappa) + n_neg + 1;
    const int m = n_clock > 0 ? n_clock : qpe_formula(n_data, kappa) + n_neg;
    QSIM_REQUIRE(m >= 1 && m <= 26, "clock qubit count must be in 1..26");
    QSIM_REQUIRE(!is_signed || m >= 2, "an indefinite A needs at least 2 clock qubits");
    QSIM_REQUIRE(nb + m + 1 <= 34, "more than 34 qubits");
    h->m = m;
    h->n = nb + m + 1;
    const double M = std::ldexp(1.0, m);
    if (!(t > 0.0)) t = 2.0 * kPi * ((is_signed ? M / 2 : M) - 1.0) / (M * amax);
    h->t = t;
    const double step = 2.0 * kPi / (t * M);  // grid value of clock value k is k * step
    if (!(C > 0.0)) {
        C = std::max(1.0, std::floor(amin / step * (1.0 + 1e-9))) * step;
    } else {
        QSIM_REQUIRE(C <= amin * (1.0 + 1e-9), "C above the smallest |eigenvalue|");
    }
    h->C = C;
    QSIM_REQUIRE(std::isfinite(t) && std::isfinite(C), "non-finite t or C");

    // step 2: the circuit
    qsim_circuit &c = h->circ;
    c.n = h->n;
    std::vector<int> data(nb), clock(m);
    for (int i = 0; i < nb; i++) data[i] = i;
    for (int j = 0; j < m; j++) clock[j] = nb + j;
    const int anc = nb + m;
    const bool passes = (flags & QSIM_HHL_FFT_QFT) != 0;
    const bool structured = (flags & QSIM_HHL_STRUCTURED_QPE) != 0;
    const size_t qpe_begin = c.gates.size();
    // structured with passes: V^H comes first (it acts on the data register only and commutes
    // with the clock's Hadamard layer), so the phase operator directly follows the layer's last
    // pass and the executor can apply it inside that pass
    if (!(structured && passes)) append_hadamards(c, clock, passes, true);
    size_t phase_idx = 0;
    if (structured) {
        // prod_j C_j-U^(2^j) = (I (x) V) diag_c(exp(i lam t c)) (I (x) V^H); the V that would
        // follow is cancelled by the V^H of the uncomputation (nothing in between acts on the data)
        std::vector<cd> VH((size_t)D * D);
        for (int r = 0; r < D; r++)
            for (int s2 = 0; s2 < D; s2++) VH[(size_t)r * D + s2] = std::conj(V[(size_t)s2 * D + r]);
        add_u(c, data, {}, std::move(VH));
        if (passes) append_hadamards(c, clock, true, true);
        Gate g;
        g.kind = GATE_QPE_PHASE;
        g.targets = data;
        g.controls = clock;
        g.theta = lam;
        g.tq = t;
        g.sign = 1;
        phase_idx = c.gates.size();
        c.gates.push_back(std::move(g));
    } else {
        for (int j = 0; j < m; j++) {
            // U_j = V diag(exp(i lambda t 2^j)) V^H  (t 2^j scales by a power of two: exact)
            const double tj = std::ldexp(t, j);
            std::vector<cd> ph(D);
            for (int i = 0; i < D; i++) ph[i] = std::polar(1.0, lam[i] * tj);
            std::vector<cd> U((size_t)D * D, cd(0.0, 0.0));
            for (int r = 0; r < D; r++)
                for (int i = 0; i < D; i++) {
                    const cd vr = V[(size_t)r * D + i] * ph[i];
                    for (int s2 = 0; s2 < D; s2++) U[(size_t)r * D + s2] += vr * std::conj(V[(size_t)s2 * D + i]);
                }
            add_u(c, data, {clock[j]}, std::move(U));
        }
    }
    const size_t iqft_begin = c.gates.size();
    // the rotation reads the clock value in the order the inverse QFT leaves it in
    std::vector<int> clock_order = clock;
    if (passes) clock_order = append_iqft_passes(c, clock);
    else append_iqft(c, clock);
    const size_t qpe_end = c.gates.size();
    // eigenvalue inversion: theta_k = 2 asin(min(1, C / (k step))), theta_0 = 0.  Emitted as a
    // uniformly controlled RY whose rotation is computed on the device from C / step (cos and sin
    // of theta_k / 2 are sqrt((1 - r)(1 + r)) and r), instead of a table of 2^m angles.
    {
        Gate g;
        g.kind = GATE_HHL_INVERT;
        g.targets = {anc};
        g.controls = clock_order;
        g.tq = C / step;
        g.sign = is_signed ? -1 : 1;  // -1: two's-complement clock register
        c.gates.push_back(std::move(g));
    }
    // uncompute: inverse of the phase estimation
    if (flags & QSIM_HHL_STRUCTURED_QPE) {
        const size_t qft_begin = c.gates.size();
        for (size_t i = qpe_end; i-- > iqft_begin;) c.gates.push_back(inverse_gate(c.gates[i]));  // QFT
        if (passes && c.gates.size() >= qft_begin + 2) {
            // the twiddle between the QFT's first two passes depends on the first pass's output
            // digit and the second pass's input digit: it moves onto the first pass's outputs (the
            // same diagonal between the same two transforms), so that the second pass, which
            // carries the phase operator on its outputs, has no twiddle of its own
            Gate &p1 = c.gates[qft_begin], &p2 = c.gates[qft_begin + 1];
            if (p1.kind == GATE_DFT && p2.kind == GATE_DFT && p1.controls.empty() && p2.pre == 1 &&
                p2.controls == p1.targets) {
                p1.controls = p2.targets;
                p1.pre = 0;
                p2.controls.clear();
                p2.pre = 0;
            }
        }
        Gate g = c.gates[phase_idx];  // the phase operator, inverted
        g.sign = -1;
        c.gates.push_back(g);
        if (passes) {  // mirror of the opening order: phase, Hadamard layer, then V
            append_hadamards(c, clock, true);
            add_u(c, data, {}, V);
        } else {
            add_u(c, data, {}, V);
            append_hadamards(c, clock, false);
        }
    } else {
        for (size_t i = qpe_end; i-- > qpe_begin;) c.gates.push_back(inverse_gate(c.gates[i]));
    }
    return h.release();
}

std::vector<cd> read_complex(const double *p, size_t n) {
    std::vector<cd> v(n);
    for (size_t i = 0; i < n; i++) {
        QSIM_REQUIRE(std::isfinite(p[2 * i]) && std::isfinite(p[2 * i + 1]), "non-finite input");
        v[i] = cd(p[2 * i], p[2 * i + 1]);
    }
    return v;
}

}  // namespace
}  // namespace qsim

using namespace qsim;

// The host side of a readout: x, |x> and the statistics from the sums and the slice.
static void readout_finish(const hhl_circuit *h, const double sums[3], const std::vector<cd> &slice, double *x_out,
                           double *x_state_out, hhl_readout_stats *stats) {
    const double P = sums[1], P0 = sums[2];  // P(anc = 1), P(anc = 1, clock = 0)
    const double inv = P0 > 0.0 ? 1.0 / std::sqrt(P0) : 0.0;
    const double norm_x = std::sqrt(P) / h->C;
    if (x_state_out)
        for (size_t i = 0; i < slice.size(); i++) {
            x_state_out[2 * i] = slice[i].real() * inv;
            x_state_out[2 * i + 1] = slice[i].imag() * inv;
        }
    if (x_out)
        for (int i = 0; i < h->N; i++) {
            const cd x = slice[h->x_off + i] * (inv * norm_x * h->norm_b);
            x_out[2 * i] = x.real();
            x_out[2 * i + 1] = x.imag();
        }
    if (stats) {
        stats->p_success = P;
        stats->p_clock0 = P0;
        stats->leakage = P - P0;
        stats->norm2 = sums[0];
        stats->norm_x = norm_x;
        stats->norm_b = h->norm_b;
    }
}


extern "C" {

int hhl_build_ex(const double *A, const double *b, int N, int n_clock, double t, double C, int flags,
                 hhl_circuit **out) {
    return guarded([&] {
        QSIM_REQUIRE(A != nullptr && b != nullptr && out != nullptr, "NULL argument");
        QSIM_REQUIRE(N >= 1 && N <= 4096, "N must be in 1..4096");
        QSIM_REQUIRE((flags & ~(QSIM_HHL_STRUCTURED_QPE | QSIM_HHL_FFT_QFT | QSIM_HHL_GAUSS_SEIDEL | QSIM_HHL_DILATE)) == 0,
                     "unknown flags");
        std::vector<cd> Am = read_complex(A, (size_t)N * N), bv = read_complex(b, N);
        // Sec. III-A step 1(a): Gauss-Seidel preconditioning, M = lower triangle of A (with the
        // diagonal); A <- M^-1 A, b <- M^-1 b by forward substitution
        if (flags & QSIM_HHL_GAUSS_SEIDEL) {
            for (int i = 0; i < N; i++) QSIM_REQUIRE(Am[(size_t)i * N + i] != cd(0.0, 0.0), "zero diagonal: no Gauss-Seidel splitting");
            std::vector<cd> X((size_t)N * N), y(N);
            for (int i = 0; i < N; i++) {
                const cd inv = 1.0 / Am[(size_t)i * N + i];
                for (int c = 0; c < N; c++) {
                    cd s2 = Am[(size_t)i * N + c];
                    for (int k = 0; k < i; k++) s2 -= Am[(size_t)i * N + k] * X[(size_t)k * N + c];
                    X[(size_t)i * N + c] = s2 * inv;
                }
                cd sb = bv[i];
                for (int k = 0; k < i; k++) sb -= Am[(size_t)i * N + k] * y[k];
                y[i] = sb * inv;
            }
            Am.swap(X);
            bv.swap(y);
        }
        double amax = 0.0;
        for (const cd &z : Am) amax = std::max(amax, std::abs(z));
        const double tol = 1e-12 * std::max(1.0, amax);
        bool herm = true;
        for (int r = 0; r < N && herm; r++)
            for (int c = 0; c <= r; c++)
                if (std::abs(Am[(size_t)r * N + c] - std::conj(Am[(size_t)c * N + r])) > tol) {
                    herm = false;
                    break;
                }
        // Sec. III-A step 1(c): Hermitian dilation [[0, A], [A^H, 0]] with right-hand side [b; 0]
        int Ne = N, off = 0;
        if (!herm || (flags & QSIM_HHL_DILATE)) {
            QSIM_REQUIRE(flags & (QSIM_HHL_DILATE | QSIM_HHL_GAUSS_SEIDEL),
                         "A is not Hermitian (pass QSIM_HHL_DILATE for the Hermitian dilation)");
            Ne = 2 * N;
            off = N;
            QSIM_REQUIRE(Ne <= 4096, "dilated system larger than 4096");
            std::vector<cd> H((size_t)Ne * Ne, cd(0.0, 0.0));
            for (int r = 0; r < N; r++)
                for (int c = 0; c < N; c++) {
                    H[(size_t)r * Ne + (N + c)] = Am[(size_t)r * N + c];
                    H[(size_t)(N + c) * Ne + r] = std::conj(Am[(size_t)r * N + c]);
                }
            Am.swap(H);
            bv.resize(Ne, cd(0.0, 0.0));
        }
        bool real = true;
        for (const cd &z : Am) real &= z.imag() == 0.0;
        std::vector<double> lam;
        std::vector<cd> V;
        if (real) {  // real symmetric: Householder tridiagonalization + implicit QR
            std::vector<double> Ar((size_t)Ne * Ne), Vr;
            for (int r = 0; r < Ne; r++)
                for (int c = 0; c < Ne; c++)
                    Ar[(size_t)r * Ne + c] = 0.5 * (Am[(size_t)r * Ne + c].real() + Am[(size_t)c * Ne + r].real());
            symmetric_eig_real(Ne, Ar, lam, Vr);
            V.assign(Vr.begin(), Vr.end());
        } else {
            for (int r = 0; r < Ne; r++) Am[(size_t)r * Ne + r] = Am[(size_t)r * Ne + r].real();
            hermitian_eig(Ne, Am, lam, V);
        }
        hhl_circuit *h = build_from_spectrum(Ne, lam, V, bv, n_clock, t, C, flags);
        h->N_eff = Ne;
        h->N = N;
        h->x_off = off;
        h->flags = flags;
        *out = h;
    });
}

int qsim_hermitian_eig(const double *A, int N, int max_iter, double *lambda, double *V) {
    return guarded([&] {
        QSIM_REQUIRE(A != nullptr && lambda != nullptr && V != nullptr, "NULL argument");
        QSIM_REQUIRE(N >= 1 && N <= 4096, "N must be in 1..4096");
        std::vector<cd> Am = read_complex(A, (size_t)N * N);
        double amax = 0.0;
        for (const cd &z : Am) amax = std::max(amax, std::abs(z));
        const double tol = 1e-12 * std::max(1.0, amax);
        for (int r = 0; r < N; r++)
            for (int c = 0; c <= r; c++)
                QSIM_REQUIRE(std::abs(Am[(size_t)r * N + c] - std::conj(Am[(size_t)c * N + r])) <= tol,
                             "A is not Hermitian");
        bool real = true;
        for (const cd &z : Am) real &= z.imag() == 0.0;
        std::vector<double> lam;
        std::vector<cd> Vc;
        if (real) {  // the same solver and symmetrisation as hhl_build
            std::vector<double> Ar((size_t)N * N), Vr;
            for (int r = 0; r < N; r++)
                for (int c = 0; c < N; c++)
                    Ar[(size_t)r * N + c] = 0.5 * (Am[(size_t)r * N + c].real() + Am[(size_t)c * N + r].real());
            symmetric_eig_real(N, Ar, lam, Vr, max_iter);
            Vc.assign(Vr.begin(), Vr.end());
        } else {
            for (int r = 0; r < N; r++) Am[(size_t)r * N + r] = Am[(size_t)r * N + r].real();
            hermitian_eig(N, Am, lam, Vc, max_iter);
        }
        for (int i = 0; i < N; i++) lambda[i] = lam[i];
        for (size_t i = 0; i < (size_t)N * N; i++) {
            V[2 * i] = Vc[i].real();
            V[2 * i + 1] = Vc[i].imag();
        }
    });
}

int hhl_build(const double *A, const double *b, int N, int n_clock, double t, double C, hhl_circuit **out) {
    return hhl_build_ex(A, b, N, n_clock, t, C, 0, out);
}

int hhl_build_spectral_ex(const double *lambda, const double *V, const double *b, int N, int n_clock, double t,
                          double C, int flags, hhl_circuit **out) {
    return guarded([&] {
        QSIM_REQUIRE(lambda != nullptr && V != nullptr && b != nullptr && out != nullptr, "NULL argument");
        QSIM_REQUIRE(N >= 1 && N <= 4096, "N must be in 1..4096");
        QSIM_REQUIRE((flags & ~(QSIM_HHL_STRUCTURED_QPE | QSIM_HHL_FFT_QFT)) == 0,
                     "hhl_build_spectral_ex takes only QSIM_HHL_STRUCTURED_QPE");
        std::vector<double> lam(lambda, lambda + N);
        for (double v : lam) QSIM_REQUIRE(std::isfinite(v), "non-finite eigenvalue");
        std::vector<cd> Vm = read_complex(V, (size_t)N * N), bv = read_complex(b, N);
        std::vector<int> idx(N);
        for (int i = 0; i < N; i++) idx[i] = i;
        std::sort(idx.begin(), idx.end(), [&](int x, int y) { return lam[x] < lam[y]; });
        std::vector<double> ls(N);
        std::vector<cd> Vs((size_t)N * N);
        for (int j = 0; j < N; j++) {
            ls[j] = lam[idx[j]];
            for (int r = 0; r < N; r++) Vs[(size_t)r * N + j] = Vm[(size_t)r * N + idx[j]];
        }
        hhl_circuit *h = build_from_spectrum(N, ls, Vs, bv, n_clock, t, C, flags);
        h->N_eff = N;
        h->flags = flags;
        *out = h;
    });
}

int hhl_build_spectral(const double *lambda, const double *V, const double *b, int N, int n_clock, double t,
                       double C, hhl_circuit **out) {
    return hhl_build_spectral_ex(lambda, V, b, N, n_clock, t, C, 0, out);
}

void hhl_circuit_free(hhl_circuit *h) { delete h; }

const qsim_circuit *hhl_as_circuit(const hhl_circuit *h) { return h ? &h->circ : nullptr; }

int hhl_get_info(const hhl_circuit *h, hhl_info *o) {
    return guarded([&] {
        QSIM_REQUIRE(h != nullptr && o != nullptr, "NULL argument");
        o->N = h->N;
        o->nb = h->nb;
        o->m = h->m;
        o->n = h->n;
        o->t = h->t;
        o->C = h->C;
        o->norm_b = h->norm_b;
        o->lambda_min = h->lam_min;
        o->lambda_max = h->lam_max;
        o->n_total_formula = h->n_total_formula;
        o->n_gates = (int)h->circ.gates.size();
        o->N_eff = h->N_eff;
        o->flags = h->flags;
    });
}

int hhl_prepare_state(void *state, int dtype, const hhl_circuit *h, void *stream) {
    return guarded([&] {
        QSIM_REQUIRE(state != nullptr && h != nullptr, "NULL argument");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        launch_prepare_state(state, h->n, dtype, h->b_pad.data(), h->nb, stream);
    });
}

int hhl_run(void *state, int dtype, const hhl_circuit *h, const qsim_circuit *c, void *stream) {
    return guarded([&] {
        QSIM_REQUIRE(state != nullptr && h != nullptr, "NULL argument");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        const qsim_circuit *g = c ? c : &h->circ;
        QSIM_REQUIRE(g->n == h->n, "circuit and HHL problem disagree on the qubit count");
        // only the data register is populated: every amplitude from 2^nb on is zero
        launch_prepare_state(state, h->n, dtype, h->b_pad.data(), h->nb, stream, h->nb);
        apply_ops(state, h->n, dtype, const_cast<qsim_circuit *>(g), stream, h->nb);
    });
}

int hhl_run_sums(void *state, int dtype, const hhl_circuit *h, const qsim_circuit *c, void *stream,
                 double *sums_device) {
    return guarded([&] {
        QSIM_REQUIRE(state != nullptr && h != nullptr && sums_device != nullptr, "NULL argument");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        const qsim_circuit *g = c ? c : &h->circ;
        QSIM_REQUIRE(g->n == h->n, "circuit and HHL problem disagree on the qubit count");
        launch_prepare_state(state, h->n, dtype, h->b_pad.data(), h->nb, stream, h->nb);
        apply_ops(state, h->n, dtype, const_cast<qsim_circuit *>(g), stream, h->nb, sums_device);
    });
}

int hhl_readout_sums(const void *state, int dtype, const hhl_circuit *h, const double *sums_device, void *stream,
                     double *x_out, double *x_state_out, hhl_readout_stats *stats) {
    return guarded([&] {
        QSIM_REQUIRE(state != nullptr && h != nullptr && sums_device != nullptr, "NULL argument");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        double sums[3];
        std::vector<cd> slice((size_t)1 << h->nb);
        readout_device_sums(state, dtype, h->n, h->nb, stream, sums_device, sums, slice.data());
        readout_finish(h, sums, slice, x_out, x_state_out, stats);
    });
}

int hhl_readout(const void *state, int dtype, const hhl_circuit *h, void *stream, double *x_out,
                double *x_state_out, hhl_readout_stats *stats) {
    return guarded([&] {
        QSIM_REQUIRE(state != nullptr && h != nullptr, "NULL argument");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        double sums[3];  // ||psi||^2, P(anc = 1), P(anc = 1, clock = 0)
        std::vector<cd> slice((size_t)1 << h->nb);
        readout_device(state, dtype, h->n, h->nb, h->m, stream, sums, slice.data());
        readout_finish(h, sums, slice, x_out, x_state_out, stats);
    });
}

}  // extern "C"
