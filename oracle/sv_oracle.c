/*
 * FP64 CPU oracle for state-vector simulation -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously correct reference that the CUDA library is checked
 * against.  Only the tests, the smoke check and the CPU-baseline leg of the benchmark load it;
 * the product path never does.  It shares no code with the CUDA library.
 *
 * State: 2^n complex amplitudes, interleaved (re, im) doubles; qubit q is bit q of the
 * amplitude index (little-endian).  A k-qubit gate matrix U is 2^k x 2^k, row-major,
 * interleaved complex; bit b of its row/column index is the value of qubit targets[b].
 *
 * Gate rule (the textbook definition of applying an operator to a subset of qubits, Sec. II-C
 * of the paper calls this the "unitary evolution of the state"): for every basis index whose
 * target bits are all 0 and whose control bits hold the requested values, gather the 2^k
 * amplitudes obtained by setting the target bits to every pattern r, multiply by U, and
 * scatter them back.  No fusion, no blocking, no reordering.
 *
 * Readout sums (Sec. III-A, step 4) use Neumaier's compensated summation in FP64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_MAXK 12

/* insert a 0 bit at position p of x (bits >= p move up by one) */
static uint64_t insert_zero(uint64_t x, int p) {
    uint64_t low = x & ((1ull << p) - 1ull);
    return ((x >> p) << (p + 1)) | low;
}

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/*
 * Apply U (2^k x 2^k) to targets[0..k-1], conditioned on controls[j] holding ctrl_val[j].
 * Returns 0 on success, -1 on bad arguments (repeated or out-of-range qubits, k too large).
 */
int ora_apply(double *psi, int n, int k, const int *targets, int nc, const int *controls,
              const int *ctrl_val, const double *U) {
    if (k < 1 || k > ORA_MAXK || nc < 0 || k + nc > n || n > 40) return -1;
    int fixed[64];
    int nf = 0;
    uint64_t seen = 0;
    for (int b = 0; b < k; b++) {
        if (targets[b] < 0 || targets[b] >= n || (seen >> targets[b]) & 1ull) return -1;
        seen |= 1ull << targets[b];
        fixed[nf++] = targets[b];
    }
    uint64_t cmask = 0;
    for (int j = 0; j < nc; j++) {
        if (controls[j] < 0 || controls[j] >= n || (seen >> controls[j]) & 1ull) return -1;
        seen |= 1ull << controls[j];
        fixed[nf++] = controls[j];
        if (ctrl_val[j]) cmask |= 1ull << controls[j];
    }
    /* sort fixed qubit positions ascending so zero bits are inserted low to high */
    for (int i = 1; i < nf; i++) {
        int v = fixed[i], j = i - 1;
        while (j >= 0 && fixed[j] > v) { fixed[j + 1] = fixed[j]; j--; }
        fixed[j + 1] = v;
    }
    const int64_t groups = (int64_t)1 << (n - nf);
    const int d = 1 << k;
    uint64_t offs[1 << ORA_MAXK];
    for (int r = 0; r < d; r++) {
        uint64_t o = 0;
        for (int b = 0; b < k; b++)
            if ((r >> b) & 1) o |= 1ull << targets[b];
        offs[r] = o;
    }
#pragma omp parallel if (groups >= 4096)
    {
        double *in = (double *)malloc(sizeof(double) * 2 * d);
#pragma omp for schedule(static)
        for (int64_t g = 0; g < groups; g++) {
            uint64_t base = (uint64_t)g;
            for (int i = 0; i < nf; i++) base = insert_zero(base, fixed[i]);
            base |= cmask;
            for (int r = 0; r < d; r++) {
                in[2 * r] = psi[2 * (base | offs[r])];
                in[2 * r + 1] = psi[2 * (base | offs[r]) + 1];
            }
            for (int r = 0; r < d; r++) {
                double re = 0.0, im = 0.0;
                const double *row = U + 2 * (size_t)r * d;
                for (int c = 0; c < d; c++) {
                    double ur = row[2 * c], ui = row[2 * c + 1];
                    double xr = in[2 * c], xi = in[2 * c + 1];
                    re += ur * xr - ui * xi;
                    im += ur * xi + ui * xr;
                }
                psi[2 * (base | offs[r])] = re;
                psi[2 * (base | offs[r]) + 1] = im;
            }
        }
        free(in);
    }
    return 0;
}

/*
 * Uniformly controlled RY: for every value v of the control register (controls[j] is bit j of
 * v), apply RY(theta[v]) to `target` conditioned on the controls holding v.  This is the
 * eigenvalue-inversion rotation of HHL written out as 2^nc multi-controlled rotations, each by
 * the gate rule above.  RY(a) = [[cos a/2, -sin a/2], [sin a/2, cos a/2]].
 */
int ora_apply_ucry(double *psi, int n, int target, int nc, const int *controls,
                   const double *theta) {
    if (nc < 0 || nc > 30) return -1;
    int vals[32];
    double U[8];
    for (int64_t v = 0; v < ((int64_t)1 << nc); v++) {
        for (int j = 0; j < nc; j++) vals[j] = (int)((v >> j) & 1);
        double c = cos(0.5 * theta[v]), s = sin(0.5 * theta[v]);
        U[0] = c;  U[1] = 0.0; U[2] = -s; U[3] = 0.0;
        U[4] = s;  U[5] = 0.0; U[6] = c;  U[7] = 0.0;
        int rc = ora_apply(psi, n, 1, &target, nc, controls, vals, U);
        if (rc) return rc;
    }
    return 0;
}

/* Neumaier (improved Kahan-Babuska) compensated accumulation of one term. */
static void neumaier_add(double *sum, double *comp, double x) {
    double t = *sum + x;
    if ((*sum >= 0 ? *sum : -*sum) >= (x >= 0 ? x : -x))
        *comp += (*sum - t) + x;
    else
        *comp += (x - t) + *sum;
    *sum = t;
}

/* sum_{i : (i & mask) == want} |psi_i|^2, compensated, sequential (deterministic). */
double ora_masked_norm2(const double *psi, int n, uint64_t mask, uint64_t want) {
    double s = 0.0, c = 0.0;
    const uint64_t N = 1ull << n;
    for (uint64_t i = 0; i < N; i++) {
        if ((i & mask) != want) continue;
        double re = psi[2 * i], im = psi[2 * i + 1];
        neumaier_add(&s, &c, re * re);
        neumaier_add(&s, &c, im * im);
    }
    return s + c;
}

/* Compensated sum of an array (exposed so a test can compare it with an exact sum). */
double ora_sum(const double *x, int64_t len) {
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < len; i++) neumaier_add(&s, &c, x[i]);
    return s + c;
}
