// Internal types of the GB300 HHL simulation library (not part of the C ABI).
#pragma once

#include <complex>
#include <cstdint>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/qsim.h"

namespace qsim {

using cd = std::complex<double>;

// Error carrying a status code; converted to a return value at the C boundary.
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string &msg);
void clear_last_error();

#define QSIM_REQUIRE(cond, msg)                                                  \
    do {                                                                         \
        if (!(cond)) throw ::qsim::Error(QSIM_EINVAL, std::string(msg));         \
    } while (0)

// Wrap a C entry point body: exceptions become status codes + thread-local message.
template <class F>
int guarded(F &&f) {
    try {
        clear_last_error();
        f();
        return QSIM_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return QSIM_ENOMEM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return QSIM_EINVAL;
    }
}

// ---------------------------------------------------------------------------------------
// Gate list entries (what the user or hhl_build appends).
enum GateKind { GATE_U = 0, GATE_UCRY = 1, GATE_QPE_PHASE = 2, GATE_HHL_INVERT = 3, GATE_DFT = 4, GATE_WALSH = 5 };

struct Gate {
    GateKind kind = GATE_U;
    std::vector<int> targets;   // GATE_U: matrix bit b <-> targets[b]; GATE_UCRY: {target}
    std::vector<int> controls;  // must be 1 (GATE_U); register bits (GATE_UCRY)
    std::vector<cd> U;          // GATE_U: 2^k x 2^k row-major
    std::vector<double> theta;  // GATE_UCRY: 2^|controls|; GATE_QPE_PHASE: eigenvalues (2^|targets|)
    double tq = 0.0;            // GATE_QPE_PHASE: evolution time; GATE_HHL_INVERT: C / grid step
    int sign = 1;               // GATE_QPE_PHASE: +1 phase estimation, -1 its inverse;
                                // GATE_HHL_INVERT: 1 unsigned, -1 two's-complement clock;
                                // GATE_DFT: sign of the exponent
    int pre = 0;                // GATE_DFT: twiddle before (1) or after (0) the transform;
                                // GATE_DFT uses `controls` as the twiddle-source register
};

// Executable operation kinds (one device pass each, or a pass group for the tile kernel).
enum OpKind {
    OP_DENSE = 0,  // dense 2^k x 2^k on targets, applied where outer controls are 1
    OP_PHASE = 1,  // multiply amplitudes whose `targets` bits are all 1 by `phase`
    OP_DIAG = 2,   // multiply by diag entry selected by the targets' bits
    OP_SWAP = 3,   // swap qubits targets[0], targets[1] (where controls are 1)
    OP_UCRY = 4,   // uniformly controlled RY
    OP_QPE_PHASE = 5,  // psi[i] *= exp(i sign lam[d] t c), d = data bits (targets), c = clock bits
    OP_HHL_INVERT = 6, // HHL inversion rotation: RY(2 asin(clamp(tq / k, -1, 1))) on the target,
                       // k = clock value (two's complement when sign == -1)
    OP_DFT = 7,        // DFT of size 2^k on the targets with a twiddle from the controls
    OP_WALSH = 8,      // H on every target (Walsh-Hadamard transform of the field), one pass
};

struct Op {
    OpKind kind = OP_DENSE;
    std::vector<int> targets;
    std::vector<int> controls;
    std::vector<cd> U;          // OP_DENSE: 2^k x 2^k; OP_DIAG: 2^k diagonal
    cd phase = 1.0;             // OP_PHASE
    std::vector<double> theta;  // OP_UCRY angles; OP_QPE_PHASE eigenvalues
    double tq = 0.0;            // OP_QPE_PHASE
    int sign = 1;               // OP_QPE_PHASE, OP_HHL_INVERT, OP_DFT
    int pre = 0;                // OP_DFT
    // device offsets (bytes) into the circuit's device blob, per dtype
    size_t dev_off[2] = {0, 0};
    // second table, per dtype: complex64 dense ops with 4..7 targets, the TF32 hi/lo split of
    // the real form (tensor cores); OP_QPE_PHASE, the high half of its two-table split
    size_t dev_off_tc[2] = {0, 0};
    bool has_tc = false;
    // complex64 dense op of 1..5 targets on qubit 0 or 1 widened with identity qubits to the
    // transposed 6-target tensor-core form, whose loads and stores run along the low qubits.
    // tc_pads: the added qubits (empty: not widened), qubits 0 and 1 among them when not targets;
    // dev_off_tcw: the widened form's blob (complex64 device data)
    std::vector<int> tc_pads;
    size_t dev_off_tcw = 0;
    bool real_u = false;        // OP_DENSE: every entry of U is real (SIMT kernels use 2 FMAs per entry)
};

struct DeviceBlob {
    void *ptr = nullptr;
    size_t bytes = 0;
    int device = -1;
    bool external = false;  // memory owned by someone else (the serving pool's arena)
};

}  // namespace qsim

struct qsim_circuit {
    int n = 0;
    bool fused = false;
    std::vector<qsim::Gate> gates;  // source list
    std::vector<qsim::Op> ops;      // executable list (built lazily for unfused circuits)
    bool ops_ready = false;
    qsim::DeviceBlob blob[2];       // [0] complex64 matrices, [1] complex128 matrices
    std::mutex mu;                  // guards ops/blob lazy construction
    ~qsim_circuit();                // releases the device copies (kernels.cu)
};

struct hhl_circuit {
    int N = 0, nb = 0, m = 0, n = 0;
    int N_eff = 0, x_off = 0, flags = 0;  // system actually solved (dilated: 2N, x at offset N)
    double t = 0, C = 0, norm_b = 0, lam_min = 0, lam_max = 0;
    int n_total_formula = 0;
    std::vector<qsim::cd> b_pad;  // normalized, padded to 2^nb
    qsim_circuit circ;
};

namespace qsim {
// circuit.cpp
void build_ops(qsim_circuit *c);                 // classify gates -> ops (no fusion)
Op classify_dense(const std::vector<int> &targets, const std::vector<int> &controls,
                  const std::vector<cd> &U);
void circuit_info(const qsim_circuit *c, qsim_circuit_info *out);
// kernels.cu
// live < n: the caller guarantees that the input is zero at every index >= 2^live and that only
// the first 2^live amplitudes have been written (see hhl_run); the result is the full state.
// sums (optional, QSIM_READOUT_SUMS_DOUBLES doubles of device memory): the readout partial sums
// of the final state (buf[0] = P, then P partials, the first half over the lower half of the
// state): written by the last operation's kernel when it can, else by a reduction after it
void apply_ops(void *state, int n, int dtype, qsim_circuit *c, void *stream, int live = -1, double *sums = nullptr);
// final readout from such a buffer: sums[3] and the (ancilla = 1, clock = 0) slice on the host
void readout_device_sums(const void *state, int dtype, int n, int nb, void *stream, const double *buf,
                         double sums[3], cd *slice);
// every kernel launch site reports its launches (qsim_launch_count)
void note_launches(int k, int family);
// resident blocks per SM of `kernel` (a __global__ function) for this launch shape on the current
// device, queried once per (kernel, threads, smem, device) and then served from a cache (the
// query runs on every launch otherwise, and the host time adds up for short solves)
int occupancy_cached(const void *kernel, int threads, size_t smem);
void ensure_device_blob(qsim_circuit *c, int dtype);
std::vector<unsigned char> pack_device_blob(qsim_circuit *c, int dtype);   // sets op offsets
void attach_external_blob(qsim_circuit *c, int dtype, void *dev, size_t bytes);
// launches the readout reductions and async copies of the sums (3 doubles) and of the raw
// 2^nb-amplitude slice into pinned host memory; scratch holds >= readout_scratch_doubles(n),
// its first QSIM_READOUT_SUMS_DOUBLES entries a readout-sums buffer (already written by
// apply_ops when sums_ready)
size_t readout_scratch_doubles(int n);
void readout_launch_async(const void *state, int dtype, int n, int nb, cudaStream_t st, double *scratch,
                          double *pinned_sums, void *pinned_slice, bool sums_ready = false);
// live in [nb, n): zero and write only the first 2^live amplitudes (apply_ops with the same
// live width treats the rest as zero)
void launch_prepare_state(void *state, int n, int dtype, const cd *b_pad, int nb, void *stream,
                          int live = -1);
void readout_device(const void *state, int dtype, int n, int nb, int m, void *stream,
                    double sums[3], cd *slice);
// dense_tc.cu
bool dense_tc_supported(int k);
size_t dense_tc_blob_bytes(int k);
void dense_tc_pack(int k, const std::vector<cd> &U, unsigned char *out);
// sums (may be NULL): readout partial sums of the result, written by the transposed form only
// (6 targets with qubits 0 and 1, no controls); *sums_written says whether they were
bool launch_dense_tc(void *state, int n, const std::vector<int> &targets, const std::vector<int> &controls,
                     const void *Bdev, int sms, cudaStream_t st, double *sums = nullptr, int hi_bit = 0,
                     bool *sums_written = nullptr);
// complex64, real U on 7 targets including qubits 0 and 1 (ascending)
bool dense_tc_real7_applies(const Op &op);
size_t dense_tc_real7_blob_bytes();
void dense_tc_pack_real7(const std::vector<cd> &U, unsigned char *out);
// sums (optional): readout partial sums of the result, split by bit hi_bit of the index (see
// tc::Args); only for a gate without controls
bool launch_dense_tc_real7(void *state, int n, const std::vector<int> &targets, const std::vector<int> &controls,
                           const void *Bdev, int sms, cudaStream_t st, double *sums = nullptr, int hi_bit = 0,
                           bool *sums_written = nullptr);
// batched.cu: plan (host image) / instantiate (device tables) / launch / results, for the pool
struct BatchImage;
bool batch_supported(const qsim_circuit *c);  // every op runs in the batched executor
BatchImage *batch_plan(const std::vector<const qsim_circuit *> &cs, const std::vector<const hhl_circuit *> &hs,
                       void *const *states, int dtype);
size_t batch_plan_device_bytes(const BatchImage *im);
size_t batch_plan_result_doubles(const BatchImage *im);
void batch_plan_free(BatchImage *im);
// tables uploaded asynchronously on `st` into `dev` (external memory); results go to `pinned`
qsim_batch *batch_instantiate(BatchImage *im, void *dev, double *pinned, cudaStream_t st);
void batch_launch(qsim_batch *b, cudaStream_t st);
void batch_enqueue_results(qsim_batch *b, cudaStream_t st);
void batch_host_result(const qsim_batch *b, int i, double *x_out, hhl_readout_stats *stats);
// dft.cu: Fourier-transform pass; tables packed into the circuit blob as W, Tlo, Thi
void dft_tables(const Op &op, std::vector<cd> &W, std::vector<cd> &Tlo, std::vector<cd> &Thi);
// qop (OP_QPE_PHASE, optional): its diagonal applied to the pass's inputs (qmode 1) or outputs
// (qmode 2), tables qlo / qhi as packed for that op
// inv (OP_HHL_INVERT on qubit n, optional): applied to the outputs, which then also fill the
// unwritten upper half 2^n .. 2^(n+1); returns false (nothing launched) if the field is not one
// contiguous run of the rotation's clock order
bool run_dft(void *state, int n, int dtype, const Op &op, const void *tables, cudaStream_t st,
             const Op *qop = nullptr, const void *qlo = nullptr, const void *qhi = nullptr, int qmode = 0,
             const Op *inv = nullptr);
// tuning.cpp: the kernel-choice table (QSIM_TUNE_* keys of qsim.h)
int tune_get(int dtype, int key, int n_qubits);  // entry of the size class of n_qubits
// dft_tma.cu: complex64 pass with bulk-copy (TMA) tiles; false when the shape does not fit
bool dft_tma_launch(const void *dft_args, int n, int K, int sign, int kind, int variant, int l2promo, int prefetch,
                    cudaStream_t st);
// two passes on one field in one kernel (see run_dft2); part (merge 1): 1 sin part into the upper
// half, 0 cos part in place
bool dft2_tma_launch(const void *args1, const void *args2, int n, int K, int merge, int part, int l2promo,
                     cudaStream_t st);
bool run_dft2(void *state, int n, int dtype, int merge, const Op &op1, const void *tab1, const Op &mid,
              const void *qlo, const void *qhi, const Op &op2, const void *tab2, cudaStream_t st);
// a pass on a field that is still |0> right above the live width, preceded by H on the field and
// the structured phase: inputs generated, not read (dft_gen_kernel)
bool dft_gen_launch(const void *args, int w, int K, int sign, cudaStream_t st);
bool run_dft_generated(void *state, int w, int dtype, const Op &op, const void *tables, const Op &qop,
                       const void *qlo, const void *qhi, cudaStream_t st);
unsigned dft_tma_read_error();
unsigned dft_merge_read_error();
void dft_merge_clear_error();
void dft_tma_clear_error();
// linalg.cpp
// Both throw Error(QSIM_EINVAL, "eigensolver did not converge ...") when the iteration cap
// (<= 0: 100 Jacobi sweeps / 60 N implicit QR steps) ends before the matrix is diagonal.
void hermitian_eig(int N, const std::vector<cd> &A, std::vector<double> &lam, std::vector<cd> &V,
                   int max_sweeps = 0);
void symmetric_eig_real(int N, const std::vector<double> &A, std::vector<double> &lam, std::vector<double> &V,
                        int max_iter = 0);
// host tables of the structured phase-estimation operator: lo[c * D + d] = exp(i s lam_d t c)
// for c < 2^h, hi[c * D + d] = exp(i s lam_d t c 2^h) for c < 2^(m-h), h = (m + 1) / 2
void qpe_phase_tables(const Op &op, std::vector<cd> &lo, std::vector<cd> &hi, int &h);
}  // namespace qsim
