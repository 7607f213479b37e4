// Gate lists, operation classification and gate fusion (Sec. II-C, Fig. 4 of the paper).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "common.h"

namespace qsim {

static thread_local std::string g_last_error;
void set_last_error(const std::string &msg) { g_last_error = msg; }
void clear_last_error() { g_last_error.clear(); }

static void check_qubits(int n, const int *q, int cnt, uint64_t &seen, const char *what) {
    for (int i = 0; i < cnt; i++) {
        QSIM_REQUIRE(q[i] >= 0 && q[i] < n, std::string(what) + " qubit out of range");
        QSIM_REQUIRE(!((seen >> q[i]) & 1ull), std::string(what) + " qubits must be distinct");
        seen |= 1ull << q[i];
    }
}

// ---------------------------------------------------------------------------------------
// Classification: a dense gate becomes the cheapest exact operation kind.
Op classify_dense(const std::vector<int> &targets, const std::vector<int> &controls,
                  const std::vector<cd> &U) {
    const int k = (int)targets.size();
    const int d = 1 << k;
    Op op;
    op.targets = targets;
    op.controls = controls;
    bool diag = true;
    for (int r = 0; r < d && diag; r++)
        for (int c = 0; c < d; c++)
            if (r != c && U[(size_t)r * d + c] != cd(0.0, 0.0)) { diag = false; break; }
    if (diag) {
        // phase on the all-ones pattern only?
        bool single = true;
        for (int r = 0; r < d - 1; r++)
            if (U[(size_t)r * d + r] != cd(1.0, 0.0)) { single = false; break; }
        if (single) {
            op.kind = OP_PHASE;
            op.phase = U[(size_t)(d - 1) * d + (d - 1)];
            // all gate qubits must be 1: merge targets into the condition set
            op.targets.insert(op.targets.end(), controls.begin(), controls.end());
            op.controls.clear();
            return op;
        }
        op.kind = OP_DIAG;
        op.U.resize(d);
        for (int r = 0; r < d; r++) op.U[r] = U[(size_t)r * d + r];
        return op;
    }
    if (k == 2) {  // exact SWAP matrix
        static const double sw[16] = {1, 0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 0, 0, 0, 1};
        bool is_swap = true;
        for (int i = 0; i < 16; i++)
            if (U[i] != cd(sw[i], 0.0)) { is_swap = false; break; }
        if (is_swap) {
            op.kind = OP_SWAP;
            return op;
        }
    }
    op.kind = OP_DENSE;
    op.real_u = true;
    for (const cd &z : U) op.real_u = op.real_u && z.imag() == 0.0;
    // canonical order: targets ascending (rows and columns of U relabelled to match), so that
    // the kernels see contiguous amplitude runs whenever the lowest qubits are targets
    std::vector<int> perm(k);  // perm[b'] = original matrix bit of sorted position b'
    for (int b = 0; b < k; b++) perm[b] = b;
    std::sort(perm.begin(), perm.end(), [&](int x, int y) { return targets[x] < targets[y]; });
    bool sorted = true;
    for (int b = 0; b < k; b++) sorted = sorted && perm[b] == b;
    if (sorted) {
        op.U = U;
        return op;
    }
    std::vector<int> idx(d);  // sorted-basis index -> original index
    for (int r = 0; r < d; r++) {
        int o = 0;
        for (int b = 0; b < k; b++)
            if ((r >> b) & 1) o |= 1 << perm[b];
        idx[r] = o;
    }
    for (int b = 0; b < k; b++) op.targets[b] = targets[perm[b]];
    op.U.resize((size_t)d * d);
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) op.U[(size_t)r * d + c] = U[(size_t)idx[r] * d + idx[c]];
    return op;
}

void build_ops(qsim_circuit *c) {
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->ops_ready) return;
    c->ops.clear();
    for (const Gate &g : c->gates) {
        if (g.kind != GATE_U) {
            Op op;
            op.kind = g.kind == GATE_UCRY        ? OP_UCRY
                      : g.kind == GATE_QPE_PHASE ? OP_QPE_PHASE
                      : g.kind == GATE_DFT       ? OP_DFT
                      : g.kind == GATE_WALSH     ? OP_WALSH
                                                 : OP_HHL_INVERT;
            op.targets = g.targets;
            op.controls = g.controls;
            op.theta = g.theta;
            op.tq = g.tq;
            op.sign = g.sign;
            op.pre = g.pre;
            c->ops.push_back(std::move(op));
        } else {
            c->ops.push_back(classify_dense(g.targets, g.controls, g.U));
        }
    }
    c->ops_ready = true;
}

// ---------------------------------------------------------------------------------------
// Fusion.
//
// A block holds a dense unitary on an ordered qubit list.  Gate g (uncontrolled, qubit set Q)
// may be appended to block B when no block after B touches Q (then g commutes with every later
// block and can move back to B), and |B.qubits u Q| <= max_k.  The candidate is the latest
// block touching Q; a gate touching no open qubit joins the latest block with room.  Any other
// entry (controlled multi-target gate, uniformly controlled rotation) closes the blocks that
// touch its qubits by acting as a barrier on them.
namespace {

struct Block {
    std::vector<int> qubits;  // bit b of the block matrix index <-> qubits[b]
    std::vector<cd> M;        // 2^|qubits| square, row-major
    bool barrier = false;     // a kept-as-is gate (index into gates via src)
    int src = -1;
};

// Expand gate matrix U (on `tq`) to the block basis `bq` (tq subset of bq): returns E with
// E[r][c] = U[rt][ct] if the non-target bits of r and c agree, else 0.
std::vector<cd> expand_to(const std::vector<int> &bq, const std::vector<int> &tq,
                          const std::vector<cd> &U) {
    const int K = (int)bq.size(), k = (int)tq.size();
    const int D = 1 << K, d = 1 << k;
    std::vector<int> pos(k);
    uint64_t tmask = 0;
    for (int b = 0; b < k; b++) {
        pos[b] = (int)(std::find(bq.begin(), bq.end(), tq[b]) - bq.begin());
        tmask |= 1ull << pos[b];
    }
    auto sub = [&](int r) {
        int v = 0;
        for (int b = 0; b < k; b++) v |= ((r >> pos[b]) & 1) << b;
        return v;
    };
    std::vector<cd> E((size_t)D * D, cd(0.0, 0.0));
    for (int r = 0; r < D; r++)
        for (int c = 0; c < D; c++)
            if ((r & ~tmask) == (c & ~tmask)) E[(size_t)r * D + c] = U[(size_t)sub(r) * d + sub(c)];
    return E;
}

void matmul_into(std::vector<cd> &out, const std::vector<cd> &A, const std::vector<cd> &B, int D) {
    out.assign((size_t)D * D, cd(0.0, 0.0));
    for (int i = 0; i < D; i++)
        for (int l = 0; l < D; l++) {
            const cd a = A[(size_t)i * D + l];
            if (a == cd(0.0, 0.0)) continue;
            for (int j = 0; j < D; j++) out[(size_t)i * D + j] += a * B[(size_t)l * D + j];
        }
}

// B.M <- G_expanded * B.M after widening B to include the gate's new qubits.
void absorb(Block &B, const std::vector<int> &tq, const std::vector<cd> &U) {
    std::vector<int> nq = B.qubits;
    for (int q : tq)
        if (std::find(nq.begin(), nq.end(), q) == nq.end()) nq.push_back(q);
    if (nq.size() != B.qubits.size()) {
        // widen: M' = I (x) M, the new qubits being the high bits of the block index
        const int Ko = (int)B.qubits.size(), K = (int)nq.size();
        const int Do = 1 << Ko, D = 1 << K;
        std::vector<cd> W((size_t)D * D, cd(0.0, 0.0));
        for (int r = 0; r < D; r++)
            for (int c = 0; c < D; c++)
                if ((r >> Ko) == (c >> Ko))
                    W[(size_t)r * D + c] = Ko == 0 ? cd(1.0, 0.0)
                                                   : B.M[(size_t)(r & (Do - 1)) * Do + (c & (Do - 1))];
        B.qubits = nq;
        B.M.swap(W);
    }
    const int D = 1 << (int)B.qubits.size();
    std::vector<cd> E = expand_to(B.qubits, tq, U), out;
    matmul_into(out, E, B.M, D);
    B.M.swap(out);
}

}  // namespace

static qsim_circuit *fuse_impl(const qsim_circuit *in, int max_k) {
    std::unique_ptr<qsim_circuit> out(new qsim_circuit());
    out->n = in->n;
    out->fused = true;
    std::vector<Block> blocks;
    std::vector<int> last(in->n, -1);  // latest block index touching each qubit
    for (size_t gi = 0; gi < in->gates.size(); gi++) {
        const Gate &g = in->gates[gi];
        std::vector<int> Q = g.targets;
        Q.insert(Q.end(), g.controls.begin(), g.controls.end());
        const bool fusable = g.kind == GATE_U && g.controls.empty() && (int)g.targets.size() <= max_k;
        if (!fusable) {
            Block b;
            b.barrier = true;
            b.src = (int)gi;
            b.qubits = Q;
            blocks.push_back(std::move(b));
            for (int q : Q) last[q] = (int)blocks.size() - 1;
            continue;
        }
        int cand = -1;
        for (int q : Q) cand = std::max(cand, last[q]);
        auto fits = [&](int bi) {
            if (bi < 0 || blocks[bi].barrier) return false;
            int cnt = (int)blocks[bi].qubits.size();
            for (int q : Q)
                if (std::find(blocks[bi].qubits.begin(), blocks[bi].qubits.end(), q) ==
                    blocks[bi].qubits.end())
                    cnt++;
            return cnt <= max_k;
        };
        // join the latest block touching Q, else the newest block (every block after the
        // candidate shares no qubit with the gate, so the gate commutes back to it)
        int target = -1;
        const int newest = (int)blocks.size() - 1;
        if (cand >= 0 && fits(cand)) target = cand;
        else if (newest >= 0 && newest != cand && fits(newest)) target = newest;
        if (target < 0) {
            blocks.emplace_back();
            target = (int)blocks.size() - 1;
        }
        absorb(blocks[target], g.targets, g.U);
        for (int q : blocks[target].qubits) last[q] = std::max(last[q], target);
        for (int q : Q) last[q] = target;
    }
    for (const Block &b : blocks) {
        if (b.barrier) {
            out->gates.push_back(in->gates[b.src]);
        } else {
            Gate g;
            g.kind = GATE_U;
            g.targets = b.qubits;
            g.U = b.M;
            out->gates.push_back(std::move(g));
        }
    }
    return out.release();
}

// The paper's gate fusion (Sec. II-C, Fig. 4) on gates of at most two qubits, its four
// strategies applied in their priority order, each as one pass over the whole circuit:
//   1. consecutive one-qubit gates on the same qubit are multiplied together;
//   2. a one-qubit gate is multiplied into the two-qubit gate that follows it on its qubit;
//   3. a one-qubit gate is multiplied into the two-qubit gate that precedes it on its qubit;
//   4. consecutive two-qubit gates on the same pair of qubits are multiplied together.
// "Consecutive on a qubit" means that no gate in between touches that qubit (strategy 4: either
// qubit), so every merge moves a gate past gates it commutes with.  A gate with one control and
// one target is a two-qubit gate here (its dense 4 x 4 form once it takes part in a merge);
// every other gate stays where it is and is never merged across on its qubits.
namespace {
struct FGate {
    Gate g;
    bool alive = true;
    int nq = 0;  // 1 or 2: mergeable one- or two-qubit gate; 0: anything else
    std::vector<int> q;
};

// the dense two-qubit form (targets {t, c}) of a gate with one control c and one target t
void densify(FGate &f) {
    if (f.g.controls.empty()) return;
    const int t = f.g.targets[0], c = f.g.controls[0];
    std::vector<cd> U(16, cd(0.0, 0.0));
    for (int r = 0; r < 4; r++)
        for (int k = 0; k < 4; k++) {
            if ((r >> 1) != (k >> 1)) continue;  // bit 1 <-> c (untouched)
            if ((r >> 1) == 0) U[(size_t)r * 4 + k] = (r & 1) == (k & 1) ? cd(1.0, 0.0) : cd(0.0, 0.0);
            else U[(size_t)r * 4 + k] = f.g.U[(size_t)(r & 1) * 2 + (k & 1)];
        }
    f.g.targets = {t, c};
    f.g.controls.clear();
    f.g.U.swap(U);
}
}  // namespace

static qsim_circuit *fuse_paper_impl(const qsim_circuit *in) {
    std::vector<FGate> fs(in->gates.size());
    for (size_t i = 0; i < fs.size(); i++) {
        FGate &f = fs[i];
        f.g = in->gates[i];
        f.q = f.g.targets;
        f.q.insert(f.q.end(), f.g.controls.begin(), f.g.controls.end());
        if (f.g.kind == GATE_U && f.g.targets.size() == 1 && f.g.controls.empty()) f.nq = 1;
        else if (f.g.kind == GATE_U && f.q.size() == 2 && f.g.controls.size() <= 1) f.nq = 2;
    }
    auto touches = [&](size_t j, int q) { return std::find(fs[j].q.begin(), fs[j].q.end(), q) != fs[j].q.end(); };
    auto next_on = [&](size_t i, int q) -> long {
        for (size_t j = i + 1; j < fs.size(); j++)
            if (fs[j].alive && touches(j, q)) return (long)j;
        return -1;
    };
    auto prev_on = [&](size_t i, int q) -> long {
        for (size_t j = i; j-- > 0;)
            if (fs[j].alive && touches(j, q)) return (long)j;
        return -1;
    };
    // merge A into B (A's qubits are among B's): A acts before B (a_first: U_B U_A) or after it
    // (U_A U_B); B keeps its place in the list
    auto merge = [&](FGate &A, FGate &B, bool a_first) {
        densify(A);
        densify(B);
        const int K = (int)B.g.targets.size(), D = 1 << K;
        std::vector<cd> E = expand_to(B.g.targets, A.g.targets, A.g.U), out;
        if (a_first) matmul_into(out, B.g.U, E, D);  // A acts first: U_B U_A
        else matmul_into(out, E, B.g.U, D);          // A acts after: U_A U_B
        B.g.U.swap(out);
        B.q = B.g.targets;
        A.alive = false;
    };
    // 1. one-qubit + one-qubit
    for (size_t i = 0; i < fs.size(); i++) {
        if (!fs[i].alive || fs[i].nq != 1) continue;
        const long j = next_on(i, fs[i].q[0]);
        if (j >= 0 && fs[j].nq == 1) merge(fs[i], fs[j], true);
    }
    // 2. one-qubit into the following two-qubit gate
    for (size_t i = 0; i < fs.size(); i++) {
        if (!fs[i].alive || fs[i].nq != 1) continue;
        const long j = next_on(i, fs[i].q[0]);
        if (j >= 0 && fs[j].nq == 2) merge(fs[i], fs[j], true);
    }
    // 3. one-qubit into the preceding two-qubit gate
    for (size_t i = 0; i < fs.size(); i++) {
        if (!fs[i].alive || fs[i].nq != 1) continue;
        const long j = prev_on(i, fs[i].q[0]);
        if (j >= 0 && fs[j].nq == 2) merge(fs[i], fs[j], false);
    }
    // 4. two-qubit + two-qubit on the same pair
    for (size_t i = 0; i < fs.size(); i++) {
        if (!fs[i].alive || fs[i].nq != 2) continue;
        const long j = next_on(i, fs[i].q[0]);
        if (j < 0 || fs[j].nq != 2 || j != next_on(i, fs[i].q[1])) continue;
        if (!touches((size_t)j, fs[i].q[0]) || !touches((size_t)j, fs[i].q[1])) continue;
        merge(fs[i], fs[j], true);
    }
    std::unique_ptr<qsim_circuit> out(new qsim_circuit());
    out->n = in->n;
    out->fused = true;
    for (FGate &f : fs)
        if (f.alive) out->gates.push_back(std::move(f.g));
    return out.release();
}

namespace {
// exp(i x c) for a double x and an integer c, |c| < 2^27, to a few ulps however large x c is.
// The product is formed exactly as p + e (e = fma(x, c, -p)), reduced by 2 pi split into three
// 26-bit heads and a double tail (Cody & Waite 1980: k P1, k P2, k P3 are exact for k < 2^27 and
// p - k P1 is exact, so the reduced argument carries the rounding of a few additions near pi),
// then cos and sin of the reduced argument.  At 20+ clock qubits the phase estimation's angles
// lambda t c reach ~1e7 rad, where rounding the product x c to a double alone would move the
// phase by ~1e-9.
cd exp_i_times(double x, double c) {
    constexpr double P1 = 0x1.921fb58p+2, P2 = -0x1.dde974p-25, P3 = 0x1.1a62630p-52,
                     P4 = 0x1.8a2e03707344ap-79;  // P1 + P2 + P3 + P4 = 2 pi to ~1e-40
    const double p = x * c;
    const double e = std::fma(x, c, -p);
    const double k = std::nearbyint(p * 0.15915494309189533577);  // p / (2 pi), to the nearest integer
    if (!(std::fabs(k) < 134217728.0)) throw Error(QSIM_EINVAL, "phase argument out of range");
    double r = (p - k * P1) - k * P2;
    r = ((r - k * P3) - k * P4) + e;
    return cd(std::cos(r), std::sin(r));
}
}  // namespace

// Tables of the structured phase exp(i s x_d c), x_d = lambda_d t (one rounding, as
// lambda_d * t), c = the clock value split as c_lo + 2^h c_hi: lo[c_lo][d] and hi[c_hi][d],
// each the exponential of the exact product x_d c_lo or x_d (c_hi 2^h).
void qpe_phase_tables(const Op &op, std::vector<cd> &lo, std::vector<cd> &hi, int &h) {
    const int nb = (int)op.targets.size(), m = (int)op.controls.size();
    const int D = 1 << nb;
    h = (m + 1) / 2;
    const size_t nlo = (size_t)1 << h, nhi = (size_t)1 << (m - h);
    lo.resize(nlo * D);
    hi.resize(nhi * D);
    std::vector<double> x(D);
    for (int d = 0; d < D; d++) x[d] = op.sign * (op.theta[d] * op.tq);
    for (size_t c = 0; c < nlo; c++)
        for (int d = 0; d < D; d++) lo[c * D + d] = exp_i_times(x[d], (double)c);
    for (size_t c = 0; c < nhi; c++)
        for (int d = 0; d < D; d++) hi[c * D + d] = exp_i_times(x[d], std::ldexp((double)c, h));
}

void circuit_info(const qsim_circuit *c, qsim_circuit_info *o) {
    std::memset(o, 0, sizeof(*o));
    o->n_qubits = c->n;
    o->fused = c->fused ? 1 : 0;
    const double N = std::ldexp(1.0, c->n);
    for (const Op &op : c->ops) {
        const int k = (int)op.targets.size();
        const double frac_ctrl = std::ldexp(1.0, -(int)op.controls.size());
        double amps = 0.0, flops = 0.0;  // amplitudes read+written once, real flops
        switch (op.kind) {
            case OP_DENSE:
                o->n_dense++;
                o->max_k = std::max(o->max_k, k);
                amps = N * frac_ctrl;
                flops = amps * 8.0 * std::ldexp(1.0, k);
                break;
            case OP_PHASE:
                o->n_diag++;
                amps = N * std::ldexp(1.0, -k);
                flops = amps * 6.0;
                break;
            case OP_DIAG:
                o->n_diag++;
                amps = N * frac_ctrl;
                flops = amps * 6.0;
                break;
            case OP_SWAP:
                o->n_perm++;
                amps = N * frac_ctrl * 0.5;
                break;
            case OP_UCRY:
            case OP_HHL_INVERT:
                o->n_ucry++;
                amps = N;
                flops = amps * 6.0;
                break;
            case OP_QPE_PHASE:
                o->n_diag++;
                amps = N;
                flops = amps * 12.0;
                break;
            case OP_DFT:  // radix-2 count 5 k per amplitude, plus the twiddle and the scaling
                o->n_dft++;
                amps = N;
                flops = amps * (5.0 * k + (op.controls.empty() ? 2.0 : 8.0));
                break;
            case OP_WALSH:  // one complex add or subtract per amplitude and qubit, the scaling
                o->n_dft++;
                amps = N;
                flops = amps * (2.0 * k + 2.0);
                break;
        }
        o->bytes_c64 += 2.0 * 8.0 * amps;
        o->bytes_c128 += 2.0 * 16.0 * amps;
        o->flops += flops;
    }
    o->n_gates = (int)c->ops.size();
}

}  // namespace qsim

using namespace qsim;

extern "C" {

const char *qsim_last_error(void) { return g_last_error.c_str(); }

const char *qsim_version(void) { return "0.1.0 sm_103a"; }

int qsim_circuit_create(int n_qubits, qsim_circuit **out) {
    return guarded([&] {
        QSIM_REQUIRE(out != nullptr, "out is NULL");
        QSIM_REQUIRE(n_qubits >= 1 && n_qubits <= 34, "n_qubits must be in 1..34");
        qsim_circuit *c = new qsim_circuit();
        c->n = n_qubits;
        *out = c;
    });
}

int qsim_circuit_add_gate(qsim_circuit *c, int k, const int *targets, int n_controls,
                          const int *controls, const double *U) {
    return guarded([&] {
        QSIM_REQUIRE(c != nullptr && targets != nullptr && U != nullptr, "NULL argument");
        QSIM_REQUIRE(k >= 1 && k <= 7, "k must be in 1..7");
        QSIM_REQUIRE(n_controls >= 0 && (n_controls == 0 || controls != nullptr), "bad controls");
        QSIM_REQUIRE(k + n_controls <= c->n, "more gate qubits than circuit qubits");
        uint64_t seen = 0;
        check_qubits(c->n, targets, k, seen, "target");
        check_qubits(c->n, controls, n_controls, seen, "control");
        const size_t d = (size_t)1 << k;
        Gate g;
        g.kind = GATE_U;
        g.targets.assign(targets, targets + k);
        if (n_controls) g.controls.assign(controls, controls + n_controls);
        g.U.resize(d * d);
        for (size_t i = 0; i < d * d; i++) {
            QSIM_REQUIRE(std::isfinite(U[2 * i]) && std::isfinite(U[2 * i + 1]), "non-finite matrix entry");
            g.U[i] = cd(U[2 * i], U[2 * i + 1]);
        }
        std::lock_guard<std::mutex> lk(c->mu);
        QSIM_REQUIRE(!c->fused, "cannot append to a fused circuit");
        c->gates.push_back(std::move(g));
        c->ops_ready = false;
    });
}

int qsim_circuit_add_ucry(qsim_circuit *c, int target, int n_controls, const int *controls,
                          const double *theta) {
    return guarded([&] {
        QSIM_REQUIRE(c != nullptr && controls != nullptr && theta != nullptr, "NULL argument");
        QSIM_REQUIRE(n_controls >= 1 && n_controls <= 30, "n_controls must be in 1..30");
        QSIM_REQUIRE(n_controls + 1 <= c->n, "more gate qubits than circuit qubits");
        uint64_t seen = 0;
        check_qubits(c->n, &target, 1, seen, "target");
        check_qubits(c->n, controls, n_controls, seen, "control");
        Gate g;
        g.kind = GATE_UCRY;
        g.targets = {target};
        g.controls.assign(controls, controls + n_controls);
        const size_t cnt = (size_t)1 << n_controls;
        g.theta.assign(theta, theta + cnt);
        for (double v : g.theta) QSIM_REQUIRE(std::isfinite(v), "non-finite angle");
        std::lock_guard<std::mutex> lk(c->mu);
        QSIM_REQUIRE(!c->fused, "cannot append to a fused circuit");
        c->gates.push_back(std::move(g));
        c->ops_ready = false;
    });
}

int qsim_circuit_add_dft(qsim_circuit *c, int k, const int *targets, int n_src, const int *src, int sign,
                         int twiddle_first) {
    return guarded([&] {
        QSIM_REQUIRE(c != nullptr && targets != nullptr, "NULL argument");
        QSIM_REQUIRE(k >= 1 && k <= 10, "k must be in 1..10");
        QSIM_REQUIRE(n_src >= 0 && (n_src == 0 || src != nullptr), "bad twiddle-source register");
        QSIM_REQUIRE(k + n_src <= 30 && k + n_src <= c->n, "k + n_src must be at most 30 and the qubit count");
        QSIM_REQUIRE(sign == 1 || sign == -1, "sign must be +1 or -1");
        QSIM_REQUIRE(twiddle_first == 0 || twiddle_first == 1, "twiddle_first must be 0 or 1");
        uint64_t seen = 0;
        check_qubits(c->n, targets, k, seen, "target");
        check_qubits(c->n, src, n_src, seen, "twiddle-source");
        Gate g;
        g.kind = GATE_DFT;
        g.targets.assign(targets, targets + k);
        if (n_src) g.controls.assign(src, src + n_src);
        g.sign = sign;
        g.pre = twiddle_first;
        std::lock_guard<std::mutex> lk(c->mu);
        QSIM_REQUIRE(!c->fused, "cannot append to a fused circuit");
        c->gates.push_back(std::move(g));
        c->ops_ready = false;
    });
}

int qsim_circuit_add_walsh(qsim_circuit *c, int k, const int *targets) {
    return guarded([&] {
        QSIM_REQUIRE(c != nullptr && targets != nullptr, "NULL argument");
        QSIM_REQUIRE(k >= 1 && k <= 10 && k <= c->n, "k must be in 1..10");
        uint64_t seen = 0;
        check_qubits(c->n, targets, k, seen, "target");
        Gate g;
        g.kind = GATE_WALSH;
        g.targets.assign(targets, targets + k);
        std::lock_guard<std::mutex> lk(c->mu);
        QSIM_REQUIRE(!c->fused, "cannot append to a fused circuit");
        c->gates.push_back(std::move(g));
        c->ops_ready = false;
    });
}

int qsim_circuit_get_info(const qsim_circuit *c, qsim_circuit_info *out) {
    return guarded([&] {
        QSIM_REQUIRE(c != nullptr && out != nullptr, "NULL argument");
        qsim_circuit *cc = const_cast<qsim_circuit *>(c);
        build_ops(cc);
        circuit_info(cc, out);
    });
}

int qsim_fuse_paper(const qsim_circuit *in, qsim_circuit **out) {
    return guarded([&] {
        QSIM_REQUIRE(in != nullptr && out != nullptr, "NULL argument");
        QSIM_REQUIRE(!in->fused, "fuse the unfused gate list");
        qsim_circuit *f = fuse_paper_impl(in);
        build_ops(f);
        *out = f;
    });
}

int qsim_circuit_get_gate(const qsim_circuit *c, int i, int *kind, int *k, int *targets, int *n_controls,
                          int *controls, double *U) {
    return guarded([&] {
        QSIM_REQUIRE(c != nullptr && kind != nullptr && k != nullptr && n_controls != nullptr, "NULL argument");
        QSIM_REQUIRE(i >= 0 && i < (int)c->gates.size(), "gate index out of range");
        const Gate &g = c->gates[i];
        *kind = (int)g.kind;
        *k = (int)g.targets.size();
        *n_controls = (int)g.controls.size();
        if (targets)
            for (size_t b = 0; b < g.targets.size(); b++) targets[b] = g.targets[b];
        if (controls)
            for (size_t b = 0; b < g.controls.size(); b++) controls[b] = g.controls[b];
        if (U && g.kind == GATE_U)
            for (size_t e = 0; e < g.U.size(); e++) {
                U[2 * e] = g.U[e].real();
                U[2 * e + 1] = g.U[e].imag();
            }
    });
}

int qsim_fuse(const qsim_circuit *in, int max_k, qsim_circuit **out) {
    return guarded([&] {
        QSIM_REQUIRE(in != nullptr && out != nullptr, "NULL argument");
        QSIM_REQUIRE(max_k >= 0 && max_k <= 6, "max_k must be in 0..6");
        if (max_k == 0) max_k = tune_get(QSIM_C64, QSIM_TUNE_FUSE_WIDTH, in->n);
        qsim_circuit *f = fuse_impl(in, max_k);
        build_ops(f);
        *out = f;
    });
}

}  // extern "C"
