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
                   std::vector<cd> &V) {
    std::vector<cd> A(Ain);
    V.assign((size_t)N * N, cd(0.0, 0.0));
    for (int i = 0; i < N; i++) V[(size_t)i * N + i] = 1.0;
    auto a = [&](int i, int j) -> cd & { return A[(size_t)i * N + j]; };
    double fro = 0.0;
    for (const cd &z : A) fro += std::norm(z);
    fro = std::sqrt(fro);
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int p = 0; p < N; p++)
            for (int q = p + 1; q < N; q++) off += std::norm(a(p, q));
        off = std::sqrt(2.0 * off);
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
