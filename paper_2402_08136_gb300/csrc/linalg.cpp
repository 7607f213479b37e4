// Host linear algebra for hhl_build: cyclic Jacobi eigensolver for complex Hermitian matrices.
//
// Golub & Van Loan, Matrix Computations (4th ed.), Sec. 8.5 (symmetric Schur decomposition and
// the cyclic Jacobi method), extended to Hermitian matrices by first rotating the phase of the
// off-diagonal pivot a_pq onto the real axis with diag(1, e^{-i arg a_pq}).
#include <algorithm>
#include <cmath>

#include "common.h"

namespace qsim {

void hermitian_eig(int N, const std::vector<cd> &Ain, std::vector<double> &lam,
                   std::vector<cd> &V, int max_sweeps) {
    if (max_sweeps <= 0) max_sweeps = 100;
    std::vector<cd> A(Ain);
    V.assign((size_t)N * N, cd(0.0, 0.0));
    for (int i = 0; i < N; i++) V[(size_t)i * N + i] = 1.0;
    auto a = [&](int i, int j) -> cd & { return A[(size_t)i * N + j]; };
    double fro = 0.0;
    for (const cd &z : A) fro += std::norm(z);
    fro = std::sqrt(fro);
    auto off_norm = [&] {
        double off = 0.0;
        for (int p = 0; p < N; p++)
            for (int q = p + 1; q < N; q++) off += std::norm(a(p, q));
        return std::sqrt(2.0 * off);
    };
    for (int sweep = 0; sweep < max_sweeps; sweep++) {
        const double off = off_norm();
        if (off <= 1e-17 * fro || off == 0.0) break;
        for (int p = 0; p < N - 1; p++) {
            for (int q = p + 1; q < N; q++) {
                const double apq_abs = std::abs(a(p, q));
                if (apq_abs == 0.0) continue;
                const cd e = a(p, q) / apq_abs;  // phase of the pivot
                const double app = a(p, p).real(), aqq = a(q, q).real();
                // real symmetric Schur 2x2 on [[app, |apq|], [|apq|, aqq]]
                const double tau = (aqq - app) / (2.0 * apq_abs);
                const double tt = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + tt * tt), s = tt * c;
                // J = diag(1, conj(e)) * [[c, s], [-s, c]]
                const cd jpp = c, jpq = s, jqp = -s * std::conj(e), jqq = c * std::conj(e);
                for (int k = 0; k < N; k++) {  // A <- A J (columns p, q)
                    const cd akp = a(k, p), akq = a(k, q);
                    a(k, p) = akp * jpp + akq * jqp;
                    a(k, q) = akp * jpq + akq * jqq;
                }
                for (int k = 0; k < N; k++) {  // A <- J^H A (rows p, q)
                    const cd apk = a(p, k), aqk = a(q, k);
                    a(p, k) = std::conj(jpp) * apk + std::conj(jqp) * aqk;
                    a(q, k) = std::conj(jpq) * apk + std::conj(jqq) * aqk;
                }
                a(p, q) = 0.0;
                a(q, p) = 0.0;
                a(p, p) = a(p, p).real();
                a(q, q) = a(q, q).real();
                for (int k = 0; k < N; k++) {  // V <- V J
                    const cd vkp = V[(size_t)k * N + p], vkq = V[(size_t)k * N + q];
                    V[(size_t)k * N + p] = vkp * jpp + vkq * jqp;
                    V[(size_t)k * N + q] = vkp * jpq + vkq * jqq;
                }
            }
        }
    }
    // The sweeps aim below rounding level; what remains must at least be rounding noise
    // (a few ulps of ||A||_F per entry), otherwise the diagonal is not the spectrum.
    {
        const double off = off_norm();
        const double accept = std::max(1e-14, 4.0 * N * 2.220446049250313e-16) * fro;
        if (!(off <= accept))
            throw Error(QSIM_EINVAL, "eigensolver did not converge (cyclic Jacobi: off-diagonal norm " +
                                         std::to_string(off) + " after " + std::to_string(max_sweeps) +
                                         " sweeps)");
    }
    // sort ascending
    std::vector<int> idx(N);
    for (int i = 0; i < N; i++) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return a(x, x).real() < a(y, y).real(); });
    lam.resize(N);
    std::vector<cd> Vs((size_t)N * N);
    for (int j = 0; j < N; j++) {
        lam[j] = a(idx[j], idx[j]).real();
        for (int k = 0; k < N; k++) Vs[(size_t)k * N + j] = V[(size_t)k * N + idx[j]];
    }
    V.swap(Vs);
}

}  // namespace qsim

// ---------------------------------------------------------------------------------------
// Real symmetric eigensolver: Householder reduction to tridiagonal form, then the implicit
// symmetric QR iteration with Wilkinson shifts (Golub & Van Loan, Sec. 8.3: Algorithm 8.3.1
// for the reduction, 8.3.2-8.3.3 for the QR step), accumulating every transformation into V.
// O(N^3) with a small constant; used by hhl_build for real symmetric A (the power-flow
// matrices), while the Jacobi solver above handles genuinely complex Hermitian A.
namespace qsim {

void symmetric_eig_real(int N, const std::vector<double> &Ain, std::vector<double> &lam,
                        std::vector<double> &V, int max_iter) {
    if (max_iter <= 0) max_iter = 60 * N;
    std::vector<double> A(Ain);
    auto a = [&](int i, int j) -> double & { return A[(size_t)i * N + j]; };
    V.assign((size_t)N * N, 0.0);
    for (int i = 0; i < N; i++) V[(size_t)i * N + i] = 1.0;
    auto v_ = [&](int i, int j) -> double & { return V[(size_t)i * N + j]; };
    // 1. tridiagonalization: A <- H_k A H_k, V <- V H_k
    std::vector<double> v(N), p(N), w(N);
    for (int k = 0; k + 2 < N; k++) {
        double alpha = 0.0;
        for (int i = k + 1; i < N; i++) alpha += a(i, k) * a(i, k);
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        if (a(k + 1, k) > 0) alpha = -alpha;  // x - alpha e1 without cancellation
        double vnorm2 = 0.0;
        for (int i = k + 1; i < N; i++) {
            v[i] = a(i, k) - (i == k + 1 ? alpha : 0.0);
            vnorm2 += v[i] * v[i];
        }
        if (vnorm2 == 0.0) continue;
        const double beta = 2.0 / vnorm2;
        // p = beta A22 v ; w = p - (beta/2)(p.v) v ; A22 <- A22 - v w^T - w v^T
        double pv = 0.0;
        for (int i = k + 1; i < N; i++) {
            double s = 0.0;
            for (int j = k + 1; j < N; j++) s += a(i, j) * v[j];
            p[i] = beta * s;
            pv += p[i] * v[i];
        }
        for (int i = k + 1; i < N; i++) w[i] = p[i] - 0.5 * beta * pv * v[i];
        for (int i = k + 1; i < N; i++)
            for (int j = k + 1; j < N; j++) a(i, j) -= v[i] * w[j] + w[i] * v[j];
        a(k + 1, k) = a(k, k + 1) = alpha;
        for (int i = k + 2; i < N; i++) a(i, k) = a(k, i) = 0.0;
        // V <- V (I - beta v v^T)
        for (int r = 0; r < N; r++) {
            double s = 0.0;
            for (int j = k + 1; j < N; j++) s += v_(r, j) * v[j];
            s *= beta;
            for (int j = k + 1; j < N; j++) v_(r, j) -= s * v[j];
        }
    }
    std::vector<double> d(N), e(N, 0.0);
    for (int i = 0; i < N; i++) d[i] = a(i, i);
    for (int i = 0; i + 1 < N; i++) e[i] = a(i + 1, i);
    // 2. implicit symmetric QR with Wilkinson shift on unreduced blocks [lo, hi]
    const double eps = 2.220446049250313e-16;
    int hi = N - 1, iter = 0;
    while (hi > 0 && iter < max_iter) {
        // deflate negligible off-diagonals
        for (int i = 0; i < hi; i++)
            if (std::fabs(e[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1]))) e[i] = 0.0;
        while (hi > 0 && e[hi - 1] == 0.0) hi--;
        if (hi == 0) break;
        int lo = hi - 1;
        while (lo > 0 && e[lo - 1] != 0.0) lo--;
        iter++;
        // Wilkinson shift from the trailing 2x2 block
        const double dd = 0.5 * (d[hi - 1] - d[hi]);
        const double eh = e[hi - 1];
        const double den = dd + (dd >= 0 ? 1.0 : -1.0) * std::sqrt(dd * dd + eh * eh);
        const double mu = den != 0.0 ? d[hi] - eh * eh / den : d[hi];
        double x = d[lo] - mu, z = e[lo];
        for (int k = lo; k < hi; k++) {
            // Givens rotation G = [c s; -s c] with G^T [x; z] = [r; 0]
            double c, s;
            if (z == 0.0) {
                c = 1.0;
                s = 0.0;
            } else if (std::fabs(z) > std::fabs(x)) {
                const double t = -x / z;
                s = 1.0 / std::sqrt(1.0 + t * t);
                c = s * t;
            } else {
                const double t = -z / x;
                c = 1.0 / std::sqrt(1.0 + t * t);
                s = c * t;
            }
            // T <- G^T T G on rows/columns k, k+1 (tridiagonal plus one bulge)
            if (k > lo) e[k - 1] = c * e[k - 1] - s * z;
            const double dk = d[k], dk1 = d[k + 1], ek = e[k];
            d[k] = c * c * dk - 2.0 * c * s * ek + s * s * dk1;
            d[k + 1] = s * s * dk + 2.0 * c * s * ek + c * c * dk1;
            e[k] = c * s * (dk - dk1) + (c * c - s * s) * ek;
            if (k + 1 < hi) {
                x = e[k];
                z = -s * e[k + 1];
                e[k + 1] = c * e[k + 1];
            }
            for (int r = 0; r < N; r++) {
                const double vk = v_(r, k), vk1 = v_(r, k + 1);
                v_(r, k) = c * vk - s * vk1;
                v_(r, k + 1) = s * vk + c * vk1;
            }
        }
    }
    // converged = every off-diagonal deflated; otherwise d is not the spectrum
    for (int i = 0; i < hi; i++)
        if (std::fabs(e[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1]))) e[i] = 0.0;
    while (hi > 0 && e[hi - 1] == 0.0) hi--;
    if (hi > 0)
        throw Error(QSIM_EINVAL, "eigensolver did not converge (implicit symmetric QR: " + std::to_string(max_iter) +
                                     " steps, block ending at row " + std::to_string(hi) + " not deflated)");
    std::vector<int> idx(N);
    for (int i = 0; i < N; i++) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int x0, int y0) { return d[x0] < d[y0]; });
    lam.resize(N);
    std::vector<double> Vs((size_t)N * N);
    for (int j = 0; j < N; j++) {
        lam[j] = d[idx[j]];
        for (int r = 0; r < N; r++) Vs[(size_t)r * N + j] = v_(r, idx[j]);
    }
    V.swap(Vs);
}

}  // namespace qsim
