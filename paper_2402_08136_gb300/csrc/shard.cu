// State sharding over G = 2^g ranks with a qubit-swap exchange (the paper's simulator scales one
// state vector over several GPUs, Sec. II-C, and reaches 42 qubits that way, Sec. III-B).
//
// Layout: rank r holds the 2^(n-g) amplitudes whose top g physical qubits equal r (physical
// qubits n-g .. n-1 are "global", the others "local").  A logical-to-physical qubit map starts
// as the identity.  A gate can run on a shard only when every qubit it touches (targets,
// controls, twiddle sources, the rotation's clock register) sits on a local position.  The
// planner walks the gate list and, before a gate that touches a global qubit, swaps that
// qubit with a local position the gate does not touch, choosing the one whose logical qubit is
// used again farthest in the future (so a run of gates on the same qubits needs one swap).
// A swap of global bit b with local position p is a pairwise exchange between ranks r and
// r ^ 2^b of half of each shard: rank r sends its amplitudes whose bit p differs from bit b of
// r and receives the partner's into the same positions (pack, send/receive, unpack; remote data
// always lands in local memory before use).  Consecutive gates that need no swap form one
// local circuit (the gates with their qubits renumbered to physical positions).  At the end,
// global positions get their own logical qubits back by swaps and the local positions by SWAP
// gates, so the gathered shards are the state in logical order.
//
// The structured phase-estimation operator needs its qubits at fixed positions and is not
// accepted; every other gate kind is.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <type_traits>
#include <vector>

#include "common.h"

struct qsim_shard_plan {
    int n = 0, g = 0;
    std::vector<qsim_shard_step> steps;
    std::vector<std::vector<int>> perms;      // logical -> physical, as of each step
    std::vector<qsim_circuit *> locals;       // local circuit of each apply step (nullptr: swap)
    ~qsim_shard_plan() {
        for (qsim_circuit *c : locals)
            if (c) qsim_circuit_free(c);
    }
};

namespace qsim {
namespace {

std::vector<int> touched(const Gate &g) {
    std::vector<int> q(g.targets);
    q.insert(q.end(), g.controls.begin(), g.controls.end());
    return q;
}

Gate remap(const Gate &g, const std::vector<int> &perm) {
    Gate r = g;
    for (int &q : r.targets) q = perm[q];
    for (int &q : r.controls) q = perm[q];
    return r;
}

template <typename R>
__global__ void shard_pack_kernel(const typename std::conditional<sizeof(R) == 4, float2, double2>::type *in,
                                  typename std::conditional<sizeof(R) == 4, float2, double2>::type *out,
                                  long long half, int q, int v, int unpack) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < half; i += (long long)gridDim.x * blockDim.x) {
        const long long lo = i & ((1ll << q) - 1);
        const long long j = ((i >> q) << (q + 1)) | ((long long)v << q) | lo;
        if (unpack) out[j] = in[i];
        else out[i] = in[j];
    }
}

void pack_launch(const void *src, void *dst, int n_local, int dtype, int q, int v, bool unpack, cudaStream_t st) {
    const long long half = 1ll << (n_local - 1);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = std::min<long long>((half + 255) / 256, (long long)sms * 8);
    if (dtype == QSIM_C128)
        shard_pack_kernel<double><<<(int)blocks, 256, 0, st>>>(static_cast<const double2 *>(src),
                                                               static_cast<double2 *>(dst), half, q, v, unpack);
    else
        shard_pack_kernel<float><<<(int)blocks, 256, 0, st>>>(static_cast<const float2 *>(src),
                                                              static_cast<float2 *>(dst), half, q, v, unpack);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("shard_pack_kernel: ") + cudaGetErrorString(e));
    note_launches(1, QSIM_KERNEL_ELEMENTWISE);
}

}  // namespace
}  // namespace qsim

using namespace qsim;

extern "C" {

int qsim_shard_plan_create(const qsim_circuit *c, int n_global, qsim_shard_plan **out) {
    return guarded([&] {
        QSIM_REQUIRE(c != nullptr && out != nullptr, "NULL argument");
        QSIM_REQUIRE(!c->fused, "plan the unfused circuit (fuse the local circuits afterwards)");
        const int n = c->n, nl = n - n_global;
        QSIM_REQUIRE(n_global >= 0 && n_global <= 10 && nl >= 1, "n_global must leave at least one local qubit");
        std::unique_ptr<qsim_shard_plan> p(new qsim_shard_plan());
        p->n = n;
        p->g = n_global;
        const std::vector<Gate> &gs = c->gates;
        std::vector<int> perm(n), who(n);  // logical -> physical, physical -> logical
        for (int q = 0; q < n; q++) perm[q] = who[q] = q;
        // next use of each logical qubit after gate i (for the choice of the swapped-out qubit)
        std::vector<std::vector<int>> uses(n);
        for (size_t i = 0; i < gs.size(); i++) {
            QSIM_REQUIRE(gs[i].kind != GATE_QPE_PHASE,
                         "the structured phase-estimation operator needs fixed qubit positions: shard the "
                         "circuit built without QSIM_HHL_STRUCTURED_QPE");
            for (int q : touched(gs[i])) {
                QSIM_REQUIRE((int)touched(gs[i]).size() <= nl, "a gate touches more qubits than a shard holds");
                uses[q].push_back((int)i);
            }
        }
        std::vector<size_t> ucur(n, 0);
        auto next_use = [&](int q, int i) {
            while (ucur[q] < uses[q].size() && uses[q][ucur[q]] < i) ucur[q]++;
            return ucur[q] < uses[q].size() ? uses[q][ucur[q]] : (int)gs.size() + 1;
        };
        auto push_swap = [&](int b, int loc) {
            qsim_shard_step s{};
            s.kind = 0;
            s.global_bit = b;
            s.local_qubit = loc;
            p->steps.push_back(s);
            const int lg = who[nl + b], ll = who[loc];
            std::swap(who[nl + b], who[loc]);
            perm[lg] = loc;
            perm[ll] = nl + b;
            p->perms.push_back(perm);
            p->locals.push_back(nullptr);
        };
        size_t first = 0;
        auto close_run = [&](size_t end) {
            if (end <= first) return;
            qsim_circuit *lc = nullptr;
            if (qsim_circuit_create(nl, &lc) != QSIM_OK) throw Error(QSIM_ENOMEM, "local circuit");
            for (size_t k = first; k < end; k++) lc->gates.push_back(remap(gs[k], perm));
            qsim_shard_step s{};
            s.kind = 1;
            s.first_gate = (int)first;
            s.last_gate = (int)end;
            p->steps.push_back(s);
            p->perms.push_back(perm);
            p->locals.push_back(lc);
        };
        for (size_t i = 0; i < gs.size(); i++) {
            const std::vector<int> tq = touched(gs[i]);
            bool need = false;
            for (int q : tq) need = need || perm[q] >= nl;
            if (!need) continue;
            close_run(i);
            first = i;
            std::vector<char> busy(nl, 0);
            for (int q : tq)
                if (perm[q] < nl) busy[perm[q]] = 1;
            for (int q : tq) {
                if (perm[q] < nl) continue;
                int best = -1, best_use = -1;
                for (int loc = 0; loc < nl; loc++) {
                    if (busy[loc]) continue;
                    const int u = next_use(who[loc], (int)i);
                    if (u > best_use) best_use = u, best = loc;
                }
                QSIM_REQUIRE(best >= 0, "no free local qubit to swap with");
                push_swap(perm[q] - nl, best);
                busy[best] = 1;
            }
        }
        close_run(gs.size());
        // back to the logical order: global positions first (swaps), then local ones (SWAP gates)
        for (int b = 0; b < n_global; b++) {
            const int want = nl + b;
            if (who[want] == want) continue;
            QSIM_REQUIRE(perm[want] < nl, "planner: logical qubit of a global position is not local");
            push_swap(b, perm[want]);
        }
        std::vector<cd> sw = {1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0};
        qsim_circuit *fix = nullptr;
        for (int q = 0; q < nl; q++) {
            if (who[q] == q) continue;
            const int at = perm[q];  // logical q sits at physical `at`, which is local
            if (!fix && qsim_circuit_create(nl, &fix) != QSIM_OK) throw Error(QSIM_ENOMEM, "local circuit");
            Gate g;
            g.kind = GATE_U;
            g.targets = {q, at};
            g.U = sw;
            fix->gates.push_back(g);
            const int lq = who[q];
            std::swap(who[q], who[at]);
            perm[q] = q;
            perm[lq] = at;
        }
        if (fix) {
            qsim_shard_step s{};
            s.kind = 1;
            s.first_gate = s.last_gate = (int)gs.size();
            p->steps.push_back(s);
            p->perms.push_back(perm);
            p->locals.push_back(fix);
        }
        *out = p.release();
    });
}

int qsim_shard_plan_num_steps(const qsim_shard_plan *p) { return p ? (int)p->steps.size() : 0; }

int qsim_shard_plan_get_step(const qsim_shard_plan *p, int i, qsim_shard_step *s, int *perm) {
    return guarded([&] {
        QSIM_REQUIRE(p != nullptr && s != nullptr, "NULL argument");
        QSIM_REQUIRE(i >= 0 && i < (int)p->steps.size(), "step index out of range");
        *s = p->steps[i];
        if (perm) std::memcpy(perm, p->perms[i].data(), sizeof(int) * p->n);
    });
}

const qsim_circuit *qsim_shard_plan_local_circuit(const qsim_shard_plan *p, int i) {
    if (!p || i < 0 || i >= (int)p->steps.size()) return nullptr;
    return p->locals[i];
}

void qsim_shard_plan_free(qsim_shard_plan *p) { delete p; }

int qsim_shard_pack(const void *shard, int n_local, int dtype, int qubit, int value, void *out, void *stream) {
    return guarded([&] {
        QSIM_REQUIRE(shard != nullptr && out != nullptr, "NULL argument");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        QSIM_REQUIRE(n_local >= 1 && n_local <= 34 && qubit >= 0 && qubit < n_local && (value == 0 || value == 1),
                     "bad shard shape");
        pack_launch(shard, out, n_local, dtype, qubit, value, false, static_cast<cudaStream_t>(stream));
    });
}

int qsim_shard_unpack(void *shard, int n_local, int dtype, int qubit, int value, const void *in, void *stream) {
    return guarded([&] {
        QSIM_REQUIRE(shard != nullptr && in != nullptr, "NULL argument");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        QSIM_REQUIRE(n_local >= 1 && n_local <= 34 && qubit >= 0 && qubit < n_local && (value == 0 || value == 1),
                     "bad shard shape");
        pack_launch(in, shard, n_local, dtype, qubit, value, true, static_cast<cudaStream_t>(stream));
    });
}

}  // extern "C"
