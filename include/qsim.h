/*
 * qsim.h -- C ABI of the GB300 HHL state-vector simulation library (libqsim_gb300.so).
 *
 * Zheng, Chen, Yang & Li, "Early Exploration of a Flexible Framework for Efficient Quantum
 * Linear Solvers in Power Systems" (PESGM 2024).  The library implements the data-parallel
 * core of the paper's method: build the HHL circuit for A x = b (Sec. III-A, Fig. 5), fuse its
 * gates (Sec. II-C, Fig. 4), apply them to a 2^n-amplitude state vector on the GPU (the
 * "unitary evolution of the state", Sec. II-C), and read the solution out of the final state
 * (Sec. III-A, steps 3-4).
 *
 * Conventions used by every call
 *   - Qubit q is bit q of the amplitude index (little-endian).
 *   - A k-qubit gate matrix is 2^k x 2^k, row-major, complex as interleaved (re, im) doubles;
 *     bit b of its row/column index is the value of qubit targets[b].
 *   - State vectors are device buffers of 2^n complex amplitudes, interleaved (re, im):
 *     QSIM_C64 = 2 x float (8 bytes per amplitude), QSIM_C128 = 2 x double (16 bytes).
 *     They are owned by the caller (e.g. a torch tensor); the library never frees them.
 *   - A `stream` argument is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls documented as asynchronous only enqueue work on that stream.
 *   - Host inputs are read only during the call.  Objects returned through `**out` are owned by
 *     the library and released with the matching *_free / *_destroy call.
 *   - Every call returns QSIM_OK (0) or a negative status; it never aborts or exits.  The text
 *     of the last error on the calling thread is returned by qsim_last_error().
 *
 * HHL register layout (used by hhl_* calls): data qubits 0..nb-1, clock qubit j is qubit nb+j
 * (bit j of the clock value), the ancilla is qubit nb+m; n = nb + m + 1.
 */
#ifndef QSIM_GB300_H
#define QSIM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define QSIM_OK 0
#define QSIM_EINVAL (-1)   /* bad argument: shape, range, non-finite, non-Hermitian, ...      */
#define QSIM_ENOMEM (-2)   /* host or device allocation failed                                 */
#define QSIM_EBUSY (-3)    /* pool: request not finished yet / memory budget exhausted         */
#define QSIM_ECUDA (-4)    /* a CUDA runtime call failed (message names it)                   */
#define QSIM_ETIMEOUT (-5) /* a bounded wait ran out                                           */
#define QSIM_ENOTFOUND (-6) /* pool: unknown ticket                                            */

/* ---- state dtypes ---------------------------------------------------------------------- */
#define QSIM_C64 1  /* complex64: FP32 state; gate arithmetic FP32 (dense k>=4 on tensor cores) */
#define QSIM_C128 2 /* complex128: FP64 state and FP64 gate arithmetic                          */

typedef struct qsim_circuit qsim_circuit; /* gate list (unfused or fused)                       */
typedef struct hhl_circuit hhl_circuit;   /* HHL problem + its unfused gate list                */
typedef struct qsim_pool qsim_pool;       /* serving pool (device memory budget + worker)       */

/* Thread-local text of the last error (empty string if none).  Never NULL. */
const char *qsim_last_error(void);

/* Library version string, e.g. "0.1.0 sm_103a". */
const char *qsim_version(void);

/* ======================================================================================= *
 * Circuits                                                                                 *
 * ======================================================================================= */

/* New empty circuit on n_qubits (1..34).  Errors: EINVAL, ENOMEM. */
int qsim_circuit_create(int n_qubits, qsim_circuit **out);

/* Append a k-qubit gate U (1 <= k <= 7), applied only where every controls[j] qubit is 1.
 * targets[0..k-1] and controls[0..n_controls-1] must be distinct and < n_qubits.  U is
 * 2^k x 2^k complex (interleaved doubles, row-major, see conventions); it is copied.
 * A gate that is a unitary product of 1- and 2-qubit gates is the unit of the paper's
 * "gate" (Sec. II-C); unitarity is not checked.  Errors: EINVAL (ranges, repeats, NaN). */
int qsim_circuit_add_gate(qsim_circuit *c, int k, const int *targets, int n_controls,
                          const int *controls, const double *U);

/* Append a uniformly controlled RY: for every value v of the control register (controls[j]
 * is bit j of v, 1 <= n_controls <= 30), rotate `target` by RY(theta[v]) =
 * [[cos theta/2, -sin theta/2], [sin theta/2, cos theta/2]].  This is the HHL eigenvalue-
 * inversion rotation (Sec. III-A, Fig. 5).  theta has 2^n_controls entries (copied).
 * Errors: EINVAL. */
int qsim_circuit_add_ucry(qsim_circuit *c, int target, int n_controls, const int *controls,
                          const double *theta);

/* Append one Cooley-Tukey pass of a quantum Fourier transform (the QFT of the phase
 * estimation, Sec. III-A and Fig. 5, with the DFT of size 2^m factored into passes over fields
 * of the register as in Cooley & Tukey 1965).  With y the value of the field targets[0..k-1]
 * (bit j <-> targets[j], 1 <= k <= 10) and w the value of the twiddle-source register
 * src[0..n_src-1] (bit j <-> src[j]), the 2^k amplitudes of every assignment of the other
 * qubits are mapped by
 *     out[y'] = 2^{-k/2} sum_y exp(sign 2 pi i y y' / 2^k) in[y]          (sign = +1 or -1)
 * and multiplied by the twiddle exp(sign 2 pi i w y' / 2^(k + n_src)) on the output index
 * (twiddle_first = 0), or by exp(sign 2 pi i w y / 2^(k + n_src)) on the input index before
 * the transform (twiddle_first = 1).  k + n_src <= 30; targets and src distinct.  The inverse
 * QFT of an m-qubit register is the passes over its fields from the top field down, each with
 * sign -1, twiddle after, and the register bits below the field as src; its output holds the
 * register value v with the digits of v in field order (the top field holds the lowest digits
 * of v).  The QFT back is the same passes in reverse order with sign +1 and twiddle first.
 * The operation runs as one pass over the state (tile-resident radix-2 transform).
 * Errors: EINVAL. */
int qsim_circuit_add_dft(qsim_circuit *c, int k, const int *targets, int n_src, const int *src, int sign,
                         int twiddle_first);

/* Append H on each of targets[0..k-1] (1 <= k <= 10, distinct): the Walsh-Hadamard transform
 * out[y'] = 2^{-k/2} sum_y (-1)^{popcount(y & y')} in[y] of the field, run as one pass over the
 * state like qsim_circuit_add_dft (the Hadamard layers of the phase estimation, Sec. III-A,
 * Fig. 5).  Errors: EINVAL. */
int qsim_circuit_add_walsh(qsim_circuit *c, int k, const int *targets);

/* Release a circuit and any device copy of its matrices.  NULL is a no-op. */
void qsim_circuit_free(qsim_circuit *c);

/* Counts describing a circuit. */
typedef struct {
    int n_qubits;
    int n_gates;        /* entries in the list (fused: executed operations)                  */
    int n_dense;        /* dense operations (after fusion: 2^k x 2^k products)               */
    int n_diag;         /* diagonal / phase operations                                        */
    int n_perm;         /* permutation operations (swaps)                                     */
    int n_ucry;         /* uniformly controlled rotations                                     */
    int max_k;          /* widest dense operation (targets)                                   */
    int fused;          /* 1 if produced by qsim_fuse                                          */
    double bytes_c64;   /* algorithmic HBM bytes of one application to a complex64 state     */
    double bytes_c128;  /* same for complex128                                                */
    double flops;       /* algorithmic real flops of one application                          */
    int n_dft;          /* Fourier and Walsh-Hadamard passes (qsim_circuit_add_dft / _walsh)  */
} qsim_circuit_info;

int qsim_circuit_get_info(const qsim_circuit *c, qsim_circuit_info *out);

/* ======================================================================================= *
 * Fusion (Sec. II-C, Fig. 4)                                                               *
 * ======================================================================================= */

/* Fuse `in` into a new circuit whose dense operations act on at most max_k qubits
 * (1 <= max_k <= 6; 0 takes the complex64 entry QSIM_TUNE_FUSE_WIDTH of the kernel-choice table,
 * 4 until qsim_autotune has measured it).  Uncontrolled
 * gates are merged greedily in circuit order (a gate joins the latest block that touches any
 * of its qubits when the union stays within max_k, which for max_k = 2 realises the paper's
 * four strategies: 1q+1q, 1q into 2q before and after, 2q+2q); each product is multiplied
 * once on the host in FP64.  Controlled multi-target gates and uniformly controlled rotations
 * are kept as they are.  Fused blocks that are exactly diagonal, single-phase or swaps are
 * tagged so the specialised kernels run them.  The fused circuit is equal to the input up to
 * FP64 rounding.  Errors: EINVAL, ENOMEM. */
int qsim_fuse(const qsim_circuit *in, int max_k, qsim_circuit **out);

/* The paper's gate fusion (Sec. II-C, Fig. 4) on gates of at most two qubits: its four
 * strategies in their priority order, each one pass over the whole circuit: one-qubit gates on
 * the same qubit first; then a one-qubit gate into the two-qubit gate that follows it on its
 * qubit, then into the one that precedes it; finally two-qubit gates on the same pair.  A gate
 * with one control and one target counts as a two-qubit gate; every other gate stays in place
 * and blocks merges across it on its qubits.  Products are formed on the host in FP64; the
 * result equals the input up to rounding.  `in` must be unfused.  Errors: EINVAL, ENOMEM. */
int qsim_fuse_paper(const qsim_circuit *in, qsim_circuit **out);

/* Gate i of a circuit (as built, or as fused): its kind (0 dense gate, 1 uniformly controlled
 * RY, other values: the structured operators), k targets and n_controls controls (each array,
 * when not NULL, must hold that many ints) and, for a dense gate when U is not NULL, its
 * 2^k x 2^k matrix (interleaved doubles, row-major, 2 * 4^k of them).  Errors: EINVAL. */
int qsim_circuit_get_gate(const qsim_circuit *c, int i, int *kind, int *k, int *targets, int *n_controls,
                          int *controls, double *U);

/* ======================================================================================= *
 * Application (the hot loop)                                                               *
 * ======================================================================================= */

/* The paper's hot loop, the "unitary evolution of the state" of Sec. II-C (gate by gate, fused
 * gates as dense 2^k x 2^k products, Fig. 4):
 * apply every operation of `c` in order to `state` (device, 2^n_qubits amplitudes of `dtype`,
 * n_qubits == the circuit's qubit count), asynchronously on `stream`.  The first call for a
 * circuit and dtype uploads its matrices to the device (synchronously) and keeps them until
 * qsim_circuit_free.  Errors: EINVAL (size/dtype mismatch, NULL), ENOMEM, ECUDA. */
int qsim_apply(void *state, int n_qubits, int dtype, const qsim_circuit *c, void *stream);

/* Sticky device-side error flags of this process's kernels (bit 0: a bounded wait inside a
 * tensor-core kernel ran out, its results are invalid).  Synchronizes the device; clear != 0
 * resets the flags.  Errors: EINVAL, ECUDA. */
int qsim_device_status(unsigned *flags, int clear);

/* Number of kernels this library has launched in this process (every launch site counts; the
 * replay of a CUDA graph that captured library calls does not).  Never fails. */
unsigned long long qsim_launch_count(void);

/* The same count split by kernel family (so a caller can tell which kernel ran an operation):
 * counts[i] for family i (QSIM_KERNEL_*), i < n; entries beyond the families are 0. */
#define QSIM_KERNEL_DENSE_SIMT 0   /* dense gates, SIMT (dense_pipe_kernel, dense_tile_kernel)      */
#define QSIM_KERNEL_DENSE_TC 1     /* dense gates on the tensor cores (complex64)                   */
#define QSIM_KERNEL_FOURIER 2      /* Fourier / Walsh-Hadamard passes, thread loads                 */
#define QSIM_KERNEL_FOURIER_TMA 3  /* Fourier / Walsh-Hadamard passes, bulk-copy (TMA) tiles       */
#define QSIM_KERNEL_EXPAND 4       /* write-only broadcast of a pass on an unwritten field          */
#define QSIM_KERNEL_ELEMENTWISE 5  /* phase, diagonal, swap, UCRY, structured phase, inversion     */
#define QSIM_KERNEL_BATCHED 6      /* persistent batched executor                                   */
#define QSIM_KERNEL_READOUT 7      /* readout reductions                                            */
#define QSIM_KERNEL_PREP 8         /* state preparation                                             */
#define QSIM_KERNEL_FAMILIES 9
int qsim_launch_counts(unsigned long long *counts, int n);

/* ======================================================================================= *
 * Kernel-choice table and autotuner                                                        *
 * ======================================================================================= */

/* Every choice the library makes between equivalent kernels or launch shapes reads one table
 * per state dtype (the paper has no counterpart; the benchmark spec asks for fusion width and tile
 * shapes chosen by an autotuner).  Keys: */
#define QSIM_TUNE_DFT_TMA 0      /* Fourier / Walsh-Hadamard passes on complex64 with a contiguous
                                    field of 9-10 qubits above the lane qubits: 0 = thread loads
                                    and stores; tile loaded by the tensor memory accelerator (bulk
                                    tensor copy) with rows of 8 amplitudes (64 B) and 1 = bulk
                                    stores, 2 = thread stores with the next tile's load issued
                                    while the current one is transformed; 3, 4 = the same with
                                    rows of 16 amplitudes (128 B)                                 */
#define QSIM_TUNE_DFT_LANES 1    /* thread-load pass kernel: lane qubits per tile (0 = 128-byte
                                    runs: 4 for complex64, 3 for complex128)                       */
#define QSIM_TUNE_DFT_PREFETCH 2 /* pass kernels: L2 prefetch distance in tiles (0 off; bulk-copy
                                    kernels prefetch with a bulk tensor prefetch)                  */
#define QSIM_TUNE_DENSE_TC 3     /* complex64 dense gates: bit k set = gates of k targets (3..6)
                                    on the tensor cores; bit 7 = real 7-target gates on the
                                    tensor cores.  Gates on qubit 0 or 1 widened with identity
                                    qubits take bit 6 (transposed form) or 7 (real form)          */
#define QSIM_TUNE_FUSE_WIDTH 4   /* width qsim_fuse uses when called with max_k = 0 (the
                                    complex64 entry; 1..6)                                          */
#define QSIM_TUNE_DFT_L2PROMO 5  /* bulk-copy pass kernel: L2 promotion of its tile loads (0 none,
                                    1 64 B, 2 128 B, 3 256 B)                                      */
#define QSIM_TUNE_DFT_MERGE 6    /* complex64 passes of the phase estimation run together (bulk-copy
                                    kernels with 16-lane rows): bit 0 = the clock's H layer on a
                                    field still |0>, the structured phase and the inverse QFT's
                                    first pass with generated inputs; bit 1 = the inverse QFT's
                                    last pass, the inversion and the QFT's first pass (two
                                    transforms per tile, one launch per half); bit 2 = the QFT's
                                    last pass, the structured phase and the Walsh-Hadamard pass    */
#define QSIM_TUNE_TUNED 7        /* 1 once qsim_autotune has written this dtype's entries        */
#define QSIM_TUNE_COUNT 8

/* Each entry is kept per state dtype and per size class (states of up to 24 qubits, 25..28,
 * 29 and more: on a 31-qubit state a pass over the top qubits meets other bounds than on a
 * 27-qubit one).  qsim_tune_get reads the entry that applies to an n_qubits state (1..34);
 * qsim_tune_set writes it for the class of n_qubits, or for every class when n_qubits is 0.
 * Writes take effect for launches enqueued afterwards.  Errors: EINVAL (unknown key, value out
 * of range). */
int qsim_tune_get(int dtype, int key, int n_qubits, int *value);
int qsim_tune_set(int dtype, int key, int n_qubits, int value);
/* Every entry of both dtypes back to its default. */
int qsim_tune_reset(void);

typedef struct {
    int n_qubits;           /* state size the measurements were taken on                       */
    int values[QSIM_TUNE_COUNT]; /* the table after tuning                                      */
    double dft_ms;          /* fastest Fourier-pass variant, ms per pass                        */
    double dense_ms[4];     /* complex64 dense gates of 3, 4, 5, 6 targets: faster kernel, ms/gate */
    double fuse_ms[5];      /* fused gate-level test circuit at widths 2..6, ms per application */
} qsim_tune_report;

/* Time the alternatives on `state` (device, 2^n_qubits amplitudes of `dtype`, 20 <= n <= 34;
 * its contents are overwritten) with CUDA events on `stream` and write the fastest into the
 * table: the Fourier-pass kernel and its lane count and prefetch distance (three 10-qubit
 * passes), tensor cores or SIMT for complex64 dense gates of 4, 5 and 6 targets (three Haar
 * gates each), and the fusion width (a gate-level circuit of 48 random 1- and 2-qubit gates
 * fused at widths 2..6).  Writes the entries of the size class of n_qubits only.  Synchronizes
 * `stream`.  out may be NULL.  Errors: EINVAL, ECUDA. */
int qsim_autotune(void *state, int n_qubits, int dtype, void *stream, qsim_tune_report *out);

/* ======================================================================================= *
 * HHL (Sec. III-A procedure, Fig. 5 circuit, Sec. III-B resources)                         *
 * ======================================================================================= */

/* Build the HHL circuit for A x = b.
 *   A: N x N complex (interleaved, row-major), Hermitian to 1e-12 * max|A_ij|, nonsingular;
 *      b: N complex (not necessarily normalized, nonzero).  An indefinite A (a negative
 *      eigenvalue) reads the clock register as two's complement: its top bit is the sign qubit
 *      n_negval of Sec. III-B.
 *   n_clock: clock qubits m (1..26); <= 0 uses the Sec. III-B formula
 *            max(n_data + 1, ceil(log2(kappa + 1))) (+1 sign qubit for an indefinite A).
 *   t: evolution time; <= 0 picks t = 2 pi (2^m - 1) / (2^m lambda_max), or
 *      2 pi (2^(m-1) - 1) / (2^m max|lambda|) for an indefinite A.
 *   C: inversion constant; <= 0 picks the largest clock grid value 2 pi k / (t 2^m) not above
 *      min|lambda| (at least one grid step); a given C above min|lambda| is EINVAL.
 * Steps: normalize b (record ||b||), pad to 2^nb with block-diag(A, lambda_max I) and zeros in
 * b, eigendecompose on the host in FP64 (real symmetric A: Householder tridiagonalization and
 * implicit QR; complex Hermitian A: cyclic Jacobi), and emit: H on each clock qubit,
 * clock j controls U_j = V diag(exp(i lambda t 2^j)) V^H on the data qubits, the inverse QFT
 * (with bit-reversal swaps) on the clock, the uniformly controlled RY with
 * theta_k = 2 asin(clamp(C / (2 pi k / (t 2^m)), -1, 1)) (theta_0 = 0; k signed for an
 * indefinite A) on the ancilla (evaluated on the device as sin(theta_k/2) = r,
 * cos(theta_k/2) = sqrt((1-|r|)(1+|r|)), r = clamp(C/lt_k, -1, 1)),
 * then the inverse of the phase estimation.  Errors: EINVAL, ENOMEM. */
int hhl_build(const double *A, const double *b, int N, int n_clock, double t, double C,
              hhl_circuit **out);

/* Same as hhl_build from a given spectral decomposition A = V diag(lambda) V^H:
 * lambda: N real eigenvalues (all > 0); V: N x N complex unitary (interleaved, row-major,
 * column i is the eigenvector of lambda[i]).  Used when the spectrum is known exactly. */
int hhl_build_spectral(const double *lambda, const double *V, const double *b, int N,
                       int n_clock, double t, double C, hhl_circuit **out);

/* hhl_build / hhl_build_spectral with options.  flags: any of QSIM_HHL_STRUCTURED_QPE,
 * QSIM_HHL_FFT_QFT, QSIM_HHL_GAUSS_SEIDEL, QSIM_HHL_DILATE (the last two for hhl_build_ex
 * only).
 * QSIM_HHL_STRUCTURED_QPE emits the phase estimation in its diagonalised form (the paper's
 * controlled evolutions, Fig. 5, multiplied out): prod_j C_j-U^(2^j) = (I (x) V)
 * diag_c(exp(i lambda t c)) (I (x) V^H), where c is the clock value.  The V closing the phase
 * estimation cancels against the V^H opening its inverse (nothing in between acts on the data
 * register), so the list becomes H^m, V^H, phase(+), inverse QFT, rotation, QFT, phase(-), V,
 * H^m: two dense nb-qubit gates and two phase passes instead of 2m controlled dense gates, and
 * no U^(2^j) products on the host.  The final state equals the unstructured circuit's up to
 * rounding. */
#define QSIM_HHL_STRUCTURED_QPE 1
/* Sec. III-A step 1(a): precondition with the Gauss-Seidel splitting M = lower triangle of A
 * (with the diagonal): A' = M^-1 A, b' = M^-1 b.  A' is generally not Hermitian, so the
 * dilation below follows automatically. */
#define QSIM_HHL_GAUSS_SEIDEL 2
/* Sec. III-A step 1(c): solve the Hermitian dilation [[0, A], [A^H, 0]] [y; x] = [b; 0]
 * (2N x 2N, eigenvalues +-sigma_i(A), sign qubit) and return x, the lower half; also accepts
 * a non-Hermitian A.  Readouts then return the N entries of x (x_state_out keeps the whole
 * dilated slice). */
#define QSIM_HHL_DILATE 4
/* Emit the inverse QFT and the QFT of the phase estimation as Fourier-transform passes
 * (qsim_circuit_add_dft) over fields of at most 10 clock qubits instead of H, controlled-phase
 * and swap gates: 1 pass for m <= 10, 2 for m <= 20, 3 above; and the two Hadamard layers on
 * the clock as Walsh-Hadamard passes over the same fields (qsim_circuit_add_walsh).  The
 * inverse QFT leaves the clock value with its digits in field order, the rotation reads it in
 * that order and the QFT consumes it, so no relabelling pass is needed; the final state equals
 * the gate-level circuit's up to rounding. */
#define QSIM_HHL_FFT_QFT 8
int hhl_build_ex(const double *A, const double *b, int N, int n_clock, double t, double C, int flags,
                 hhl_circuit **out);
int hhl_build_spectral_ex(const double *lambda, const double *V, const double *b, int N, int n_clock,
                          double t, double C, int flags, hhl_circuit **out);

/* The host eigensolver behind hhl_build (Sec. III-A: U = exp(iAt) of the phase estimation is
 * formed from A = V diag(lambda) V^H), exposed so that callers can check a system before
 * building.  A: N x N complex (interleaved, row-major), Hermitian to 1e-12 * max|A_ij|.
 * A real symmetric A takes Householder tridiagonalisation + implicit symmetric QR with
 * Wilkinson shifts (max_iter = QR steps, <= 0: 60 N); a complex A cyclic Jacobi (max_iter =
 * sweeps, <= 0: 100).  Outputs (caller-owned): lambda[N] ascending, V N x N complex
 * (interleaved, row-major, column i = eigenvector of lambda[i]).  Errors: EINVAL (NULL, N out
 * of 1..4096, not Hermitian, or "eigensolver did not converge" when the iteration cap ends
 * before the matrix is diagonal to rounding; hhl_build reports the same error). */
int qsim_hermitian_eig(const double *A, int N, int max_iter, double *lambda, double *V);

void hhl_circuit_free(hhl_circuit *h);

/* Borrowed view of the HHL gate list as a circuit (valid until hhl_circuit_free). */
const qsim_circuit *hhl_as_circuit(const hhl_circuit *h);

typedef struct {
    int N, nb, m, n;     /* system size, data / clock / total qubits                         */
    double t, C;         /* evolution time and inversion constant used                        */
    double norm_b;       /* ||b||                                                              */
    double lambda_min, lambda_max;
    int n_total_formula; /* Sec. III-B count (data + QPE + sign + ancilla) for this A           */
    int n_gates;         /* unfused gate count                                                */
    int N_eff;           /* size of the system actually solved (2N after the dilation)         */
    int flags;           /* hhl_build_ex flags                                                 */
} hhl_info;

int hhl_get_info(const hhl_circuit *h, hhl_info *out);

/* Write |0>_anc |0>_clock |b/||b||> into `state` (device, 2^n amplitudes of dtype),
 * asynchronously on `stream`.  Errors: EINVAL, ECUDA. */
int hhl_prepare_state(void *state, int dtype, const hhl_circuit *h, void *stream);

/* The device part of one HHL solve, enqueued on `stream`: prepare |0>_anc |0>_clock |b> in
 * `state` and apply circuit `c` (h's gate list, or a qsim_fuse of hhl_as_circuit(h); NULL
 * means h's own list), skipping work on amplitudes that are provably zero.  After the
 * preparation only the 2^nb data amplitudes are populated, and the executor tracks a live width
 * w (every amplitude from index 2^w on is zero and unwritten): an operation on qubits below w
 * runs on the first 2^w amplitudes; a Walsh-Hadamard or Fourier pass on the field right above w
 * (the clock's Hadamard layer of Fig. 5 on |0>) only broadcasts column 0 of the transform (a
 * write-only pass) and widens w; diagonal operations leave the zeros alone; the eigenvalue-
 * inversion rotation of Fig. 5 (Sec. III-A step 2) on the top qubit, the ancilla, writes the
 * upper half without reading it, so everything before it runs on at most half the state; any
 * other operation first zero-fills up to its top qubit.  The final state equals
 * hhl_prepare_state followed by qsim_apply of the same circuit, up to rounding.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int hhl_run(void *state, int dtype, const hhl_circuit *h, const qsim_circuit *c, void *stream);

typedef struct {
    double p_success;  /* P(ancilla = 1)                                                       */
    double p_clock0;   /* P(ancilla = 1 and clock = 0)                                         */
    double leakage;    /* p_success - p_clock0                                                 */
    double norm2;      /* ||psi||^2 (should be 1)                                              */
    double norm_x;     /* ||x|| = sqrt(p_success) / C  (Sec. III-A step 4a, with C = |lambda0|)*/
    double norm_b;     /* ||b||                                                                */
} hhl_readout_stats;

/* Read the solution out of a final HHL state (Sec. III-A steps 3-4), FP64 reductions on the
 * GPU for either dtype, enqueued on `stream`, then a synchronizing copy of 2^nb amplitudes
 * and the sums to the host.  Outputs (each may be NULL):
 *   x_out:       N complex (interleaved): x = ||x|| ||b|| |x>
 *   x_state_out: 2^nb complex: |x> = (ancilla = 1, clock = 0 slice) / sqrt(p_clock0)
 *   stats:       the scalars above.
 * Uses device scratch allocated with cudaMallocAsync on `stream` and freed before return.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int hhl_readout(const void *state, int dtype, const hhl_circuit *h, void *stream, double *x_out,
                double *x_state_out, hhl_readout_stats *stats);

/* Readout sums computed inside the run.  hhl_run_sums is hhl_run that also leaves, in
 * sums_device (device memory of QSIM_READOUT_SUMS_DOUBLES doubles, caller-owned), the FP64
 * partial sums of |psi|^2 over the final state that the readout needs: written by the circuit's
 * last kernel while it stores the state when that is a complex64 tensor-core gate without
 * controls in the transposed 6-target or the real 7-target form (the eigenvector rotation V that
 * ends the structured HHL circuit), else by a reduction pass after it.  Device-only, so it can be captured into a CUDA graph.  hhl_readout_sums is
 * hhl_readout taking those partials instead of reducing the state again; the state must not
 * have changed since the hhl_run_sums that wrote sums_device.  Errors: EINVAL, ENOMEM, ECUDA. */
#define QSIM_READOUT_SUMS_DOUBLES 4096
int hhl_run_sums(void *state, int dtype, const hhl_circuit *h, const qsim_circuit *c, void *stream,
                 double *sums_device);
int hhl_readout_sums(const void *state, int dtype, const hhl_circuit *h, const double *sums_device, void *stream,
                     double *x_out, double *x_state_out, hhl_readout_stats *stats);

/* ======================================================================================= *
 * Batched execution: many small circuits in one persistent launch                          *
 * ======================================================================================= */

typedef struct qsim_batch qsim_batch; /* uploaded op tables of a set of circuits + results   */

/* Upload the op tables of `count` circuits (each applied to states[i], a device buffer of
 * 2^n_i amplitudes of `dtype`, n_i <= 30) into one device allocation (synchronous).  Every
 * operation must be a dense gate of at most 5 targets, a phase, diagonal or swap gate, a
 * uniformly controlled RY over consecutive control qubits, the structured phase or the HHL
 * inversion, or a Fourier / Walsh-Hadamard pass over consecutive ascending qubits (fuse with
 * max_k <= 5); otherwise QSIM_EINVAL.  The state pointers are stored: they must stay valid
 * while the batch is run.  Errors: EINVAL, ENOMEM, ECUDA. */
int qsim_batch_create(const qsim_circuit *const *cs, void *const *states, int count, int dtype,
                      qsim_batch **out);

/* HHL batch: circuit i is hhl i's gate list, or fused[i] when fused != NULL (a qsim_fuse
 * result of hhl_as_circuit(hs[i])).  Each run also prepares |0>|0>|b_i> in states[i] and
 * computes the FP64 readout sums and the solution slice of every circuit on the device. */
int hhl_batch_create(const hhl_circuit *const *hs, const qsim_circuit *const *fused,
                     void *const *states, int count, int dtype, qsim_batch **out);

/* Run the batch: at most two persistent kernels on `stream`, nothing else (no allocation, no
 * copy, no synchronization; each kernel resets its own work counter when it ends), so the call
 * can be captured into a CUDA graph.  Runs of one batch must not overlap (same stream, or
 * ordered).  Circuits whose state exceeds 2^13 (complex128) or 2^14 (complex64) amplitudes
 * run first, each on a team of 4 CTAs (a thread-block cluster) that splits every operation
 * and updates the state in place; then every other circuit runs on one CTA with its state in
 * shared memory.  Within each launch circuits go most expensive first.  A circuit always runs
 * on the same kind of team in a fixed order, so its result is bit-identical whatever else is
 * in the batch; it equals qsim_apply of the same circuit up to rounding (different kernels).
 * Errors: EINVAL, ECUDA. */
int qsim_batch_run(qsim_batch *b, void *stream);

/* After an HHL batch ran on `stream`: wait for `stream` and write, for batch entry i in order,
 * x_i (N_i complex, concatenated into x_out) and stats[i], as hhl_readout would.  The kernel
 * writes its readout sums straight into the batch's pinned host buffer (no copy), so a run
 * overwrites them; the outputs here are the caller's and stay as written.  x_out / stats may
 * be NULL.  Errors: EINVAL, ECUDA. */
int hhl_batch_results(qsim_batch *b, void *stream, double *x_out, hhl_readout_stats *stats);

/* One solve of every circuit of an HHL batch in a single call: qsim_batch_run followed by
 * hhl_batch_results on `stream` (one kernel launch, which writes the readout sums into pinned
 * host memory, one stream synchronization, the host-side scaling of Sec. III-A steps 3-4), for
 * latency-bound use such as one small system at a time.  x_out / stats as in
 * hhl_batch_results (caller-owned, may be NULL).  Errors: EINVAL, ECUDA. */
int hhl_batch_solve(qsim_batch *b, void *stream, double *x_out, hhl_readout_stats *stats);

void qsim_batch_free(qsim_batch *b);

/* Autotuner of the fusion width for an HHL batch: for each candidate width candidates[i]
 * (1..5) fuse every circuit, build the batch on `states`, run it once to warm up and twice
 * timed with CUDA events on `stream`; *best_k receives the fastest width, ms_out[i] (may be
 * NULL) the time per run.  The states are overwritten.  Synchronizes `stream`.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int hhl_batch_autotune(const hhl_circuit *const *hs, void *const *states, int count, int dtype,
                       const int *candidates, int ncand, void *stream, int *best_k, double *ms_out);

/* Convenience: qsim_batch_create + qsim_batch_run + wait + free.  n_qubits[i] must equal the
 * qubit count of cs[i].  Synchronizes `stream`.  Errors: EINVAL, ENOMEM, ECUDA. */
int qsim_apply_batched(void *const *states, const int *n_qubits, const qsim_circuit *const *cs,
                       int count, int dtype, void *stream);

/* ======================================================================================= *
 * State sharding over 2^g ranks with a qubit-swap exchange (Sec. II-C: the simulator's        *
 * state vector spread over several GPUs; Sec. III-B: 42 qubits on several nodes)            *
 * ======================================================================================= */

/* Rank r holds the 2^(n-g) amplitudes whose top g physical qubits equal r.  A plan turns an
 * unfused circuit into steps: a swap exchanges global physical qubit n-g+global_bit with the
 * local physical qubit local_qubit (ranks r and r ^ 2^global_bit trade the halves of their
 * shards whose bit local_qubit differs from bit global_bit of r: qsim_shard_pack the half with
 * that bit = 1 - bit global_bit of r, send it, receive the partner's, qsim_shard_unpack it into
 * the same positions); an apply step runs a local circuit (gates first_gate .. last_gate-1 of the
 * input, their qubits renumbered to physical positions, on n-g qubits) on every shard.  Before a
 * gate that touches a global qubit the planner swaps it with a local position the gate does not
 * touch, the one used again farthest in the future.  The last steps restore the logical order,
 * so the shards in rank order are the state.  The structured phase operator
 * (QSIM_HHL_STRUCTURED_QPE) needs fixed qubit positions and is rejected; a gate may touch at
 * most n-g qubits. */
typedef struct qsim_shard_plan qsim_shard_plan;
typedef struct {
    int kind;          /* 0 swap, 1 apply                                                       */
    int global_bit;    /* swap: global bit b (physical qubit n-g+b)                            */
    int local_qubit;   /* swap: local physical qubit                                           */
    int first_gate, last_gate; /* apply: gates of the input circuit (first == last: the final
                                  local reordering, SWAP gates only)                          */
} qsim_shard_step;

/* Plan the unfused circuit c over 2^n_global ranks (0 <= n_global <= 10, n_global < n).
 * Errors: EINVAL (fused circuit, structured phase operator, a gate wider than a shard), ENOMEM. */
int qsim_shard_plan_create(const qsim_circuit *c, int n_global, qsim_shard_plan **out);
int qsim_shard_plan_num_steps(const qsim_shard_plan *p);
/* Step i; perm (may be NULL) receives the n-entry logical -> physical qubit map that holds
 * during step i (after the swap, for a swap step).  Errors: EINVAL. */
int qsim_shard_plan_get_step(const qsim_shard_plan *p, int i, qsim_shard_step *s, int *perm);
/* The local circuit of apply step i (owned by the plan; NULL for a swap step).  It can be fused
 * (qsim_fuse) and applied with qsim_apply on each n-g qubit shard. */
const qsim_circuit *qsim_shard_plan_local_circuit(const qsim_shard_plan *p, int i);
void qsim_shard_plan_free(qsim_shard_plan *p);

/* Copy the half of a shard (device, 2^n_local amplitudes of dtype) whose bit `qubit` equals
 * `value` into out (device, 2^(n_local-1) amplitudes, in index order), or back (unpack), async
 * on `stream`.  Errors: EINVAL, ECUDA. */
int qsim_shard_pack(const void *shard, int n_local, int dtype, int qubit, int value, void *out, void *stream);
int qsim_shard_unpack(void *shard, int n_local, int dtype, int qubit, int value, const void *in, void *stream);

/* ======================================================================================= *
 * Serving pool: HHL solves admitted as they arrive, states resident in one device arena     *
 * ======================================================================================= */

typedef struct {
    const double *A; /* N x N complex, interleaved, row-major (copied by qsim_submit)          */
    const double *b; /* N complex (copied)                                                     */
    int N;
    int n_clock;     /* as hhl_build                                                           */
    double t, C;     /* as hhl_build                                                           */
    int dtype;       /* QSIM_C64 or QSIM_C128 state                                            */
    int flags;       /* hhl_build_ex flags (QSIM_HHL_STRUCTURED_QPE, ...; the pool adds      */
                     /* QSIM_HHL_FFT_QFT)                                                      */
} hhl_request;

typedef struct {
    size_t bytes_total, bytes_in_use, bytes_peak; /* device arena                           */
    int queued, building, running, done, failed;
    long long batches_launched, singles_launched;
} qsim_pool_info;

/* Create a pool owning one device arena of `bytes` (allocated now, on the current device),
 * n_builders host threads that build and fuse submitted HHL circuits (<= 0: half the host
 * threads) and n_streams CUDA streams (<= 0: 8).  A request is admitted once the arena has
 * room for its state (8 * 2^n bytes for complex64, 16 * 2^n for complex128) and a stream is
 * free.  Requests of at most 16 qubits that the batched executor supports (dense gates of at
 * most 5 targets) and that are ready together run as one batched launch; the others run alone
 * with the full-GPU kernels, preparation and circuit as in hhl_run; launches on different
 * streams overlap.  Every request is built
 * with QSIM_HHL_FFT_QFT added (the QFTs and clock Hadamard layers as passes).
 * Results equal those of the same request run alone (each circuit's arithmetic does not
 * depend on its batch).  Errors: EINVAL, ENOMEM, ECUDA. */
int qsim_pool_create(size_t bytes, int n_builders, int n_streams, qsim_pool **out);

/* Queue a request (inputs copied; returns immediately) and return its ticket.
 * Errors: EINVAL (NULL, N out of 1..4096, bad dtype, pool shutting down). */
int qsim_submit(qsim_pool *p, const hhl_request *req, uint64_t *ticket);

/* Non-blocking: QSIM_EBUSY while the request is pending; QSIM_OK when done (x_out receives N
 * complex values, stats and latency_s = completion - submission in seconds; the ticket is
 * released); the request's own error code if it failed (EINVAL for a bad system, ENOMEM if its
 * state can never fit the arena, ECUDA; ticket released, message in qsim_last_error);
 * QSIM_ENOTFOUND for an unknown or released ticket.  Outputs may be NULL. */
int qsim_poll(qsim_pool *p, uint64_t ticket, double *x_out, hhl_readout_stats *stats,
              double *latency_s);

/* Block until the request is no longer pending or `timeout_s` seconds pass (QSIM_ETIMEOUT).
 * Does not release the ticket.  Errors: ETIMEOUT, ENOTFOUND, EINVAL. */
int qsim_pool_wait(qsim_pool *p, uint64_t ticket, double timeout_s);

/* Completion queue: wait up to timeout_s for at least one finished request, then move up to
 * `capacity` tickets of finished (done or failed) requests, oldest first, into `tickets` and
 * set *count (0 on timeout).  Each finished ticket is handed out once; read it with
 * qsim_poll.  Errors: EINVAL. */
int qsim_pool_take_completed(qsim_pool *p, uint64_t *tickets, int capacity, int *count,
                             double timeout_s);

int qsim_pool_get_info(qsim_pool *p, qsim_pool_info *out);

/* One retired launch of the pool: the stream slot, whether it was a batched launch (1) or one
 * large request with the full-GPU kernels (0), the requests it carried (tickets first..last in
 * submission order), and its device-time interval [t_start, t_end] in seconds since the pool was
 * created (CUDA events recorded on the slot's stream around the launch's work; -1 if the work
 * failed).  Intervals of launches on different slots that intersect ran concurrently. */
typedef struct {
    int slot;
    int batched;
    int n_requests;
    uint64_t first_ticket, last_ticket;
    double t_start, t_end;
} qsim_pool_launch;

/* The most recent retired launches (at most 4096 are kept), oldest first: up to `capacity`
 * entries into out, *count set.  Errors: EINVAL. */
int qsim_pool_launch_log(qsim_pool *p, qsim_pool_launch *out, int capacity, int *count);

/* Finish admitted work, drop requests not yet built, release everything.  NULL is a no-op. */
void qsim_pool_destroy(qsim_pool *p);

/* hhl_readout for callers that cannot allocate device memory.  The paper has no counterpart;
 * this is a library convenience.  Such callers include an application whose own pool
 * allocator already owns all device memory, and code that must not call cudaMalloc or
 * cudaMallocAsync while it reads results.  Arguments, outputs, reductions and results are
 * those of hhl_readout.  The scratch (per-block partial sums, the totals and an FP64 copy of
 * the solution slice) is one fixed array inside the library, about 33 KB, which every GPU
 * that loads the library holds until the process exits; no device or host memory is
 * allocated per call.  Limit: 2^nb <= 1024 amplitudes (N <= 1024), otherwise QSIM_EINVAL.
 * The first call on a device looks up the array's device address (once per device).  The
 * call copies its results into host memory and synchronizes `stream`, so it cannot be
 * captured into a CUDA graph.  All calls share the one array: calls that overlap on the GPU
 * (other streams, other host threads) race on it and must be serialized by the caller.
 * Errors: EINVAL (including nb > 10, before any device access), ECUDA. */
int hhl_readout_noalloc(const void *state, int dtype, const hhl_circuit *h, void *stream,
                        double *x_out, double *x_state_out, hhl_readout_stats *stats);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_GB300_H */
