// Batched execution of many small circuits in one persistent launch (the batching pattern of the
// HHL solver: many N-1 contingency solves of uneven size at once).
//
// Each CTA repeatedly takes the next circuit from a work counter (circuits ordered by
// decreasing cost on the host) and runs the whole circuit by itself: optional HHL state
// preparation, every operation of the (fused) gate list with a CTA barrier between operations,
// and the optional FP64 readout sums.  A state of up to `smem_amps` amplitudes lives in shared
// memory for the whole circuit (loaded once, written back once); a larger state is updated in
// place in global memory, where it stays L2-resident.  Because one CTA executes one circuit
// with a fixed instruction and reduction order, a circuit's result does not depend on what
// else is in the batch.
//
// Supported operations: dense gates with up to 5 targets and any controls, phase, diagonal,
// swap, uniformly controlled RY over a contiguous control register, the structured phase, the HHL
// inversion, and Fourier / Walsh-Hadamard passes over contiguous fields; qubit masks are 32-bit
// (states of at most 30 qubits).  The running circuit's op list and data are staged in shared
// memory when they fit; the work counter is reset by the last CTA of a launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>

#include "common.h"

namespace qsim {
namespace batch {

// threads per CTA: 512 for complex64 (more independent loads in flight for states updated in
// global memory), 256 for complex128 (register budget of the 5-target dense gate)
template <typename V> struct Threads { static constexpr int n = sizeof(V) == 8 ? 512 : 256; };

enum BKind : unsigned char {
    B_DENSE = 0, B_PHASE = 1, B_DIAG = 2, B_SWAP = 3, B_UCRY = 4, B_QPE = 5, B_INVERT = 6,
    B_DFT = 7,    // DFT over the contiguous field c0 .. c0+k-1; t[0] twiddle-source start, nreg its
                  // width, t[1] twiddle mode (0 none, 1 before, 2 after), t[2] sign, t[3] table split
    B_WALSH = 8,  // H on every qubit of the contiguous field c0 .. c0+k-1
};

struct BOp {
    unsigned char kind, k, c0, nreg;  // c0 / nreg: UCRY control register (contiguous);
                                      // B_INVERT: t[1] = rotation of that register;
                                      // B_DENSE: c0 = 1 if U is real
    signed char t[8];                 // targets in matrix-bit order (UCRY: t[0] = target)
    unsigned fixmask;                 // targets | controls (zero bits inserted when enumerating)
    unsigned cmask;                   // controls that must be 1 (PHASE: all its qubits)
    unsigned data;                    // element offset into the circuit's data
    unsigned data2;                   // B_QPE: offset of the second phase table
    unsigned pad;                     // 32-byte records (copied to shared memory in 16-byte units)
};
static_assert(sizeof(BOp) == 32, "BOp is copied in 16-byte units");

struct BCirc {
    void *state;
    const BOp *ops;
    const void *data;
    double *result;  // readout: [norm2, P, P0, pad] then 2^nb complex (re, im) doubles
    int n, nops, nb, flags;  // flags: 1 = prepare |0>|0>|b>, 2 = readout sums and slice
    unsigned b_off;       // element offset of b (HHL preparation) in the data
    unsigned data_bytes;  // size of the circuit's data (a multiple of 8)
};

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

__device__ __forceinline__ unsigned expand(unsigned g, unsigned fixmask) {
    for (unsigned m = fixmask; m; m &= m - 1) {
        const int p = __ffs(m) - 1;
        g = ((g >> p) << (p + 1)) | (g & ((1u << p) - 1u));
    }
    return g;
}

// A circuit runs on a team: one CTA (CS = 1), or the CS CTAs of a thread-block cluster for a
// state too large for one CTA's shared memory (it stays in global memory, L2-resident).  vt is
// the thread's index in the team, team_sync<CS> the barrier between steps of an operation.
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}

template <int CS>
__device__ __forceinline__ void team_sync() {
    if (CS == 1) {
        __syncthreads();
    } else {
        // every thread of every CTA of the cluster; release / acquire order the global-memory
        // updates of one step before the next step's reads in the other CTAs
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
    }
}

// store a 32-bit / 64-bit value into the shared memory of CTA `rank` of the cluster, at the
// address that `local` has in this CTA
__device__ __forceinline__ void st_cluster(const void *local, unsigned rank, unsigned v) {
    unsigned a = (unsigned)__cvta_generic_to_shared(local), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.u32 [%0], %1;\n" ::"r"(ra), "r"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(const void *local, unsigned rank, double v) {
    unsigned a = (unsigned)__cvta_generic_to_shared(local), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.f64 [%0], %1;\n" ::"r"(ra), "d"(v) : "memory");
}

template <typename V, int K, bool REAL, int CS>
__device__ void op_dense(V *psi, int n, const BOp &op, const V *U, unsigned vt) {
    constexpr int D = 1 << K;
    constexpr int NT = CS * Threads<V>::n;
    // independent groups per iteration (their loads overlap); complex128 keeps the register
    // count of the 3..5-target gates in check with one group
    constexpr int ILP = (K <= 2 || (K <= 4 && sizeof(V) == 8)) ? 2 : 1;
    const unsigned ngroups = 1u << (n - __popc(op.fixmask));  // fixmask = targets | controls
    unsigned offs[D];
#pragma unroll
    for (int r = 0; r < D; r++) {
        unsigned o = 0;
#pragma unroll
        for (int b = 0; b < K; b++)
            if ((r >> b) & 1) o |= 1u << op.t[b];
        offs[r] = o;
    }
    if (sizeof(V) == 16 && ngroups < (unsigned)(ILP * NT)) {
        // complex128 with fewer groups than the loop below has slots (small states): S =
        // min(D, NT / ngroups) threads share a group, each computing D / S of its rows, so that
        // the FP64 work, whose pipe is narrow, spreads over every warp instead of the first
        // (and no dead second group issues arithmetic); a barrier separates the group's loads
        // from its stores.  ngroups and NT are powers of two.  complex64 keeps the loop: its
        // arithmetic is cheap and the loop's two interleaved groups pay more than the split.
        const int S = min(D, NT / (int)ngroups);
        const unsigned gi = vt / (unsigned)S;
        const int s = (int)(vt & (unsigned)(S - 1));
        const bool live = gi < ngroups;
        const unsigned base = live ? (expand(gi, op.fixmask) | op.cmask) : 0u;
        V x[D];
#pragma unroll
        for (int c = 0; c < D; c++) x[c] = live ? psi[base + offs[c]] : V{0, 0};
        team_sync<CS>();
        if (!live) return;
#pragma unroll 1
        for (int r = s; r < D; r += S) {
            const V *u = U + r * D;
            V acc{0, 0};
#pragma unroll
            for (int c = 0; c < D; c++) {
                const V w = u[c];
                acc.x = fma(w.x, x[c].x, acc.x);
                acc.y = fma(w.x, x[c].y, acc.y);
                if (!REAL) {
                    acc.x = fma(-w.y, x[c].y, acc.x);
                    acc.y = fma(w.y, x[c].x, acc.y);
                }
            }
            unsigned o = 0;  // offs[r] without a dynamic register-array index
#pragma unroll
            for (int b = 0; b < K; b++)
                if ((r >> b) & 1) o |= 1u << op.t[b];
            psi[base + o] = acc;
        }
        return;
    }
    for (unsigned g0 = vt; g0 < ngroups; g0 += ILP * NT) {
        unsigned base[ILP];
        bool live[ILP];
        V x[ILP][D];
#pragma unroll
        for (int j = 0; j < ILP; j++) {
            live[j] = g0 + j * NT < ngroups;
            base[j] = live[j] ? (expand(g0 + j * NT, op.fixmask) | op.cmask) : 0u;
#pragma unroll
            for (int c = 0; c < D; c++) x[j][c] = live[j] ? psi[base[j] + offs[c]] : V{0, 0};
        }
#pragma unroll 1
        for (int r = 0; r < D; r++) {
            const V *u = U + r * D;
#pragma unroll
            for (int j = 0; j < ILP; j++) {
                V acc{0, 0};
#pragma unroll
                for (int c = 0; c < D; c++) {
                    const V w = u[c];
                    acc.x = fma(w.x, x[j][c].x, acc.x);
                    acc.y = fma(w.x, x[j][c].y, acc.y);
                    if (!REAL) {  // real U: the imaginary parts are zero
                        acc.x = fma(-w.y, x[j][c].y, acc.x);
                        acc.y = fma(w.y, x[j][c].x, acc.y);
                    }
                }
                if (live[j]) psi[base[j] + offs[r]] = acc;
            }
        }
    }
}

template <typename V>
__device__ __forceinline__ V cmulb(V a, V b) {
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// Fourier (DFT) or Walsh-Hadamard transform of the contiguous field f0 .. f0+K-1 inside one
// circuit: K radix-2 decimation-in-frequency stages (stage j pairs the amplitudes that differ
// in field bit j; the DFT multiplies the difference by exp(s 2 pi i r / 2^(j+1)), r = the field
// bits below j, from the table W[e] = exp(s 2 pi i e / 2^K), e = r 2^(K-1-j)), a barrier after
// each, then one pass that undoes the digit reversal of the DFT, scales by 2^(-K/2) and
// applies the output twiddle.  The input twiddle, if any, is a pass of its own first.
template <typename V, int CS>
__device__ void op_fourier(V *psi, int n, const BOp &op, const V *data, unsigned vt, bool walsh) {
    constexpr int NT = CS * Threads<V>::n;
    using Rr = decltype(V{}.x);
    const int K = op.k, f0 = op.c0;
    const unsigned N = 1u << n, fmask = ((1u << K) - 1u) << f0;
    const V *W = data + op.data;
    const int twmode = walsh ? 0 : op.t[1];
    const int ns = op.nreg, s0 = op.t[0], hT = op.t[3];
    const V *Tlo = data + op.data2, *Thi = Tlo + (1u << hT);
    const unsigned smask = (1u << ns) - 1u, tmask = (1u << hT) - 1u;
    auto tw = [&](unsigned i, unsigned y) -> V {  // exp(s 2 pi i w y / 2^(K+ns))
        const unsigned q = ((i >> s0) & smask) * y;
        return cmulb(Tlo[q & tmask], Thi[q >> hT]);
    };
    if (twmode == 1) {
        for (unsigned i = vt; i < N; i += NT) psi[i] = cmulb(psi[i], tw(i, (i & fmask) >> f0));
        team_sync<CS>();
    }
    for (int j = K - 1; j >= 0; j--) {
        const int p = f0 + j;
        const unsigned bit = 1u << p, rmask = (1u << j) - 1u;
        // two independent pairs per iteration: their loads are in flight together (states
        // updated in place in L2 would otherwise wait for one round trip per pair)
        constexpr int U4 = 2;
        for (unsigned g0 = vt; g0 < N / 2; g0 += U4 * NT) {
            V a[U4], b[U4];
            unsigned i0[U4];
#pragma unroll
            for (int e = 0; e < U4; e++) {
                const unsigned g = g0 + e * NT;
                i0[e] = ((g >> p) << (p + 1)) | (g & (bit - 1u));
                if (g < N / 2) {
                    a[e] = psi[i0[e]];
                    b[e] = psi[i0[e] | bit];
                }
            }
#pragma unroll
            for (int e = 0; e < U4; e++) {
                if (g0 + e * NT >= N / 2) break;
                V d;
                d.x = a[e].x - b[e].x;
                d.y = a[e].y - b[e].y;
                psi[i0[e]] = V{a[e].x + b[e].x, a[e].y + b[e].y};
                if (!walsh) {
                    const unsigned r = (i0[e] >> f0) & rmask;
                    if (r) d = cmulb(d, W[r << (K - 1 - j)]);
                }
                psi[i0[e] | bit] = d;
            }
        }
        team_sync<CS>();
    }
    const Rr scale = (K & 1) ? (Rr)(0.70710678118654752440 / (double)(1u << (K / 2))) : (Rr)(1.0 / (double)(1u << (K / 2)));
    for (unsigned i = vt; i < N; i += NT) {
        const unsigned y = (i & fmask) >> f0;
        const unsigned yr = walsh ? y : (__brev(y) >> (32 - K));
        if (yr < y) continue;  // the pair (y, yr) belongs to the thread that holds the smaller one
        const unsigned rest = i & ~fmask, ir = rest | (yr << f0);
        V u = psi[i], v = psi[ir];  // position p holds output bitrev(p)
        V out_y = walsh ? u : v, out_r = walsh ? v : u;
        out_y.x *= scale; out_y.y *= scale;
        out_r.x *= scale; out_r.y *= scale;
        if (twmode == 2) {
            out_y = cmulb(out_y, tw(i, y));
            if (ir != i) out_r = cmulb(out_r, tw(ir, yr));
        }
        psi[i] = out_y;
        if (ir != i) psi[ir] = out_r;
    }
}

// The same transform for a state updated in place in global memory (L2): tile by tile through
// the CTA's shared memory.  A tile is the whole field times the L lowest qubits (lanes, below
// the field); it is read once, all K stages run on it in shared memory, and the write-back
// undoes the digit reversal and applies the scaling and the output twiddle.  One L2 read and
// write per amplitude instead of one per stage.
template <typename V, int CS>
__device__ void op_fourier_tiled(V *g, int n, const BOp &op, const V *data, int tid, unsigned rank, bool walsh, V *sm,
                                 int L) {
    constexpr int NT = Threads<V>::n;  // the CTA's threads: a tile belongs to one CTA of the team
    using Rr = decltype(V{}.x);
    const int K = op.k, f0 = op.c0;
    const unsigned TN = 1u << (K + L), lmask = (1u << L) - 1u;
    const int mid = f0 - L;  // qubits between the lanes and the field
    const unsigned ntile = 1u << (n - K - L);
    const V *W = data + op.data;
    const int twmode = walsh ? 0 : op.t[1];
    const int ns = op.nreg, s0 = op.t[0], hT = op.t[3];
    const V *Tlo = data + op.data2, *Thi = Tlo + (1u << hT);
    const unsigned smask = (1u << ns) - 1u, tmask = (1u << hT) - 1u;
    auto tw = [&](unsigned i, unsigned y) -> V {
        const unsigned q = ((i >> s0) & smask) * y;
        return cmulb(Tlo[q & tmask], Thi[q >> hT]);
    };
    auto gidx = [&](unsigned o, unsigned j) -> unsigned {  // tile o, local index j = lane + (y << L)
        const unsigned olo = o & ((1u << mid) - 1u), ohi = o >> mid;
        return (j & lmask) | (olo << L) | ((j >> L) << f0) | (ohi << (f0 + K));
    };
    const Rr scale = (K & 1) ? (Rr)(0.70710678118654752440 / (double)(1u << (K / 2))) : (Rr)(1.0 / (double)(1u << (K / 2)));
    for (unsigned o = rank; o < ntile; o += CS) {
        for (unsigned j = tid; j < TN; j += NT) {
            const unsigned gi = gidx(o, j);
            V x = g[gi];
            if (twmode == 1) x = cmulb(x, tw(gi, j >> L));
            sm[j] = x;
        }
        __syncthreads();
        for (int jj = K - 1; jj >= 0; jj--) {
            const int p = L + jj;
            const unsigned bit = 1u << p, rmask = (1u << jj) - 1u;
            for (unsigned q = tid; q < TN / 2; q += NT) {
                const unsigned i0 = ((q >> p) << (p + 1)) | (q & (bit - 1u));
                const V a = sm[i0], b = sm[i0 | bit];
                V d;
                d.x = a.x - b.x;
                d.y = a.y - b.y;
                sm[i0] = V{a.x + b.x, a.y + b.y};
                if (!walsh) {
                    const unsigned r = (i0 >> L) & rmask;
                    if (r) d = cmulb(d, W[r << (K - 1 - jj)]);
                }
                sm[i0 | bit] = d;
            }
            __syncthreads();
        }
        for (unsigned j = tid; j < TN; j += NT) {
            const unsigned y = j >> L;
            const unsigned yr = walsh ? y : (__brev(y) >> (32 - K));
            V v = sm[(j & lmask) | (yr << L)];  // position yr holds output y
            v.x *= scale;
            v.y *= scale;
            const unsigned gi = gidx(o, j);
            if (twmode == 2) v = cmulb(v, tw(gi, y));
            g[gi] = v;
        }
        __syncthreads();  // the next tile reuses the buffer
    }
}

template <typename R, int CS>
__device__ void run_op(typename C2<R>::T *psi, int n, const BOp &op, const typename C2<R>::T *data, unsigned vt,
                       int tid, unsigned rank, typename C2<R>::T *sm, int smem_log) {
    using V = typename C2<R>::T;
    constexpr int kThreads = CS * Threads<V>::n;  // the team's threads
    const V *d = data + op.data;
    switch (op.kind) {
        case B_DENSE:
            if (op.c0)  // real U (flag set by the encoder)
                switch (op.k) {
                    case 1: op_dense<V, 1, true, CS>(psi, n, op, d, vt); break;
                    case 2: op_dense<V, 2, true, CS>(psi, n, op, d, vt); break;
                    case 3: op_dense<V, 3, true, CS>(psi, n, op, d, vt); break;
                    case 4: op_dense<V, 4, true, CS>(psi, n, op, d, vt); break;
                    case 5: op_dense<V, 5, true, CS>(psi, n, op, d, vt); break;
                    default: break;
                }
            else
                switch (op.k) {
                    case 1: op_dense<V, 1, false, CS>(psi, n, op, d, vt); break;
                    case 2: op_dense<V, 2, false, CS>(psi, n, op, d, vt); break;
                    case 3: op_dense<V, 3, false, CS>(psi, n, op, d, vt); break;
                    case 4: op_dense<V, 4, false, CS>(psi, n, op, d, vt); break;
                    case 5: op_dense<V, 5, false, CS>(psi, n, op, d, vt); break;
                    default: break;
                }
            break;
        case B_PHASE: {
            const unsigned cnt = 1u << (n - __popc(op.fixmask));
            const V ph = d[0];
            for (unsigned g = vt; g < cnt; g += kThreads) {
                const unsigned i = expand(g, op.fixmask) | op.cmask;
                psi[i] = cmulb(psi[i], ph);
            }
            break;
        }
        case B_DIAG: {
            const unsigned cnt = 1u << (n - __popc(op.cmask));  // every index with the controls set
            for (unsigned g = vt; g < cnt; g += kThreads) {
                const unsigned i = expand(g, op.cmask) | op.cmask;  // enumerate all but controls
                unsigned p = 0;
                for (int b = 0; b < op.k; b++) p |= ((i >> op.t[b]) & 1u) << b;
                psi[i] = cmulb(psi[i], d[p]);
            }
            break;
        }
        case B_SWAP: {
            const unsigned cnt = 1u << (n - __popc(op.fixmask));
            const unsigned ma = 1u << op.t[0], mb = 1u << op.t[1];
            for (unsigned g = vt; g < cnt; g += kThreads) {
                const unsigned i = expand(g, op.fixmask) | op.cmask;
                const V x = psi[i | ma], y = psi[i | mb];
                psi[i | ma] = y;
                psi[i | mb] = x;
            }
            break;
        }
        case B_UCRY: {
            const unsigned cnt = 1u << (n - 1);
            const int tq = op.t[0];
            const unsigned tb = 1u << tq, vmask = (1u << op.nreg) - 1u;
            for (unsigned g = vt; g < cnt; g += kThreads) {
                const unsigned i0 = ((g >> tq) << (tq + 1)) | (g & (tb - 1u));
                const V cs = d[(i0 >> op.c0) & vmask];
                const V x0 = psi[i0], x1 = psi[i0 | tb];
                V y0, y1;
                y0.x = cs.x * x0.x - cs.y * x1.x;
                y0.y = cs.x * x0.y - cs.y * x1.y;
                y1.x = cs.y * x0.x + cs.x * x1.x;
                y1.y = cs.y * x0.y + cs.x * x1.y;
                psi[i0] = y0;
                psi[i0 | tb] = y1;
            }
            break;
        }
        case B_INVERT: {  // HHL inversion: rotation from Cs / k (data holds (Cs, 0); op.k = 1:
                          // two's-complement clock register; t[1] = rot: the register's low rot
                          // qubits hold the top digits of k, as Fourier passes leave it)
            const unsigned cnt = 1u << (n - 1);
            const int tq = op.t[0], rot = op.t[1];
            const unsigned tb = 1u << tq, vmask = (1u << op.nreg) - 1u;
            using Rr = decltype(V{}.x);
            const Rr Cs = d[0].x;
            for (unsigned g = vt; g < cnt; g += kThreads) {
                const unsigned i0 = ((g >> tq) << (tq + 1)) | (g & (tb - 1u));
                const unsigned raw = (i0 >> op.c0) & vmask;
                const unsigned k = rot ? ((raw >> rot) | ((raw & ((1u << rot) - 1u)) << (op.nreg - rot))) : raw;
                Rr s = 0, c = 1;
                if (k) {
                    const int ks = (op.k && (k >> (op.nreg - 1))) ? (int)k - (1 << op.nreg) : (int)k;
                    s = Cs / (Rr)ks;
                    if (s > (Rr)1) s = (Rr)1;
                    if (s < (Rr)-1) s = (Rr)-1;
                    const Rr as = s < 0 ? -s : s;
                    c = sqrt(((Rr)1 - as) * ((Rr)1 + as));
                }
                const V x0 = psi[i0], x1 = psi[i0 | tb];
                V y0, y1;
                y0.x = c * x0.x - s * x1.x;
                y0.y = c * x0.y - s * x1.y;
                y1.x = s * x0.x + c * x1.x;
                y1.y = s * x0.y + c * x1.y;
                psi[i0] = y0;
                psi[i0 | tb] = y1;
            }
            break;
        }
        case B_DFT:
        case B_WALSH: {
            const bool walsh = op.kind == B_WALSH;
            const int L = min((int)op.c0, smem_log - (int)op.k);  // lanes below the field
            if (psi != sm && L >= 0) op_fourier_tiled<V, CS>(psi, n, op, data, tid, rank, walsh, sm, L);
            else op_fourier<V, CS>(psi, n, op, data, vt, walsh);
            break;
        }
        case B_QPE: {  // data qubits 0..k-1, clock register k..k+nreg-1, split at c0 bits
            const V *hi = data + op.data2;
            const unsigned N = 1u << n, dmask = (1u << op.k) - 1u, cm = (1u << op.nreg) - 1u;
            const unsigned hm = (1u << op.c0) - 1u;
            constexpr int U4 = 2;  // independent amplitudes per iteration (loads in flight together)
            for (unsigned i0 = vt; i0 < N; i0 += U4 * kThreads) {
                V x[U4], ph[U4];
#pragma unroll
                for (int e = 0; e < U4; e++) {
                    const unsigned i = i0 + e * kThreads;
                    if (i < N) {
                        const unsigned dd = i & dmask, c = (i >> op.k) & cm;
                        x[e] = psi[i];
                        ph[e] = cmulb(d[((c & hm) << op.k) + dd], hi[((c >> op.c0) << op.k) + dd]);
                    }
                }
#pragma unroll
                for (int e = 0; e < U4; e++)
                    if (i0 + e * kThreads < N) psi[i0 + e * kThreads] = cmulb(x[e], ph[e]);
            }
            break;
        }
        default: break;
    }
}

// Three CTA-wide FP64 sums at once (one pair of barriers instead of three), each in a fixed
// order: warp shuffles, then the warp totals in warp order; thread 0 receives the totals.
template <int kThreads>
__device__ __forceinline__ void block_sum3(double &a, double &b, double &c, double *sh) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    constexpr int W = kThreads >> 5;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[w] = a;
        sh[W + w] = b;
        sh[2 * W + w] = c;
    }
    __syncthreads();
    if (w == 0) {
        a = l < W ? sh[l] : 0.0;
        b = l < W ? sh[W + l] : 0.0;
        c = l < W ? sh[2 * W + l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
            c += __shfl_down_sync(0xffffffffu, c, o);
        }
    }
    __syncthreads();
}

// CS = 1: each CTA runs whole circuits by itself.  CS > 1 (launched as clusters of CS CTAs):
// the cluster is one team that runs each of its circuits together, the state in global memory,
// every operation's work split over the team's threads (a Fourier pass: its tiles over the
// team's CTAs) and a cluster barrier between steps; readout partial sums are added in rank
// order, so results do not depend on the rest of the batch either.
template <typename R, int CS>
__global__ void __launch_bounds__(Threads<typename C2<R>::T>::n) batched_kernel(const BCirc *circs, const int *order,
                                                                              int count, unsigned *counter,
                                                                              int smem_amps, int stage_bytes) {
    using V = typename C2<R>::T;
    constexpr int kThreads = Threads<V>::n;  // per CTA
    constexpr int kTeam = CS * kThreads;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    // after the state area: the running circuit's data (matrices, tables) and op list when they
    // fit, so that each op reads its descriptor and operands from shared memory rather than
    // through two dependent L2 round trips
    unsigned char *stage = smraw + (((size_t)smem_amps * sizeof(V) + 15) & ~(size_t)15);
    __shared__ int cur;
    __shared__ double red[3 * (Threads<V>::n >> 5)];
    __shared__ double part[3 * CS];  // team: each CTA's readout sums, gathered in rank 0
    const int tid = threadIdx.x;
    const unsigned rank = CS == 1 ? 0u : cluster_rank();
    const unsigned vt = rank * (unsigned)kThreads + (unsigned)tid;
    const int nteams = (int)gridDim.x / CS;
    const int smem_log = 31 - __clz(smem_amps);
    team_sync<CS>();  // a cluster's CTAs have all started before one writes another's shared memory
    for (;;) {
        if (rank == 0 && tid == 0) {
            const int v = (int)atomicAdd(counter, 1u);
            if (CS == 1) cur = v;
            else
                for (unsigned r = 0; r < (unsigned)CS; r++) st_cluster(&cur, r, (unsigned)v);
        }
        team_sync<CS>();
        const int ci = cur;
        team_sync<CS>();
        if (ci >= count) {
            // Every team ends with one increment that returns count or more; the one that
            // returns count + nteams - 1 is the launch's last, so it puts the counter back to
            // zero for the next launch (no separate reset before each run).
            if (rank == 0 && tid == 0 && ci == count + nteams - 1) *counter = 0u;
            break;
        }
        const BCirc c = circs[order[ci]];
        const unsigned N = 1u << c.n;
        V *g = reinterpret_cast<V *>(c.state);
        // a state that fits stays in shared memory for the whole circuit (one CTA); larger ones
        // stay in global memory (L2), where the passes tile through shared memory
        V *psi = (CS == 1 && (int)N <= smem_amps) ? sm : g;
        const V *gdata = reinterpret_cast<const V *>(c.data);
        const V *data = gdata;
        const BOp *ops = c.ops;
        {
            // data (8-byte units: its size is a multiple of 8 and it starts 256-byte aligned)
            // first, then the ops (32-byte records, 16-byte units); every CTA of a team keeps
            // its own copy
            const unsigned ob = (unsigned)c.nops * (unsigned)sizeof(BOp);
            const unsigned db = (c.data_bytes + 15u) & ~15u;
            const bool with_data = db + ob <= (unsigned)stage_bytes;
            if (with_data) {
                const uint2 *src = reinterpret_cast<const uint2 *>(c.data);
                uint2 *dst = reinterpret_cast<uint2 *>(stage);
                for (unsigned i = tid; i < c.data_bytes / 8u; i += kThreads) dst[i] = src[i];
                data = reinterpret_cast<const V *>(stage);
            }
            if (ob <= (unsigned)stage_bytes) {
                const unsigned o0 = with_data ? db : 0u;
                const uint4 *src = reinterpret_cast<const uint4 *>(c.ops);
                uint4 *dst = reinterpret_cast<uint4 *>(stage + o0);
                for (unsigned i = tid; i < ob / 16u; i += kThreads) dst[i] = src[i];
                ops = reinterpret_cast<const BOp *>(stage + o0);
            }
        }
        if (c.flags & 1) {
            const unsigned Db = 1u << c.nb;
            for (unsigned i = vt; i < N; i += kTeam) psi[i] = i < Db ? gdata[c.b_off + i] : V{0, 0};
        } else if (psi == sm) {
            for (unsigned i = tid; i < N; i += kThreads) psi[i] = g[i];
        }
        team_sync<CS>();
        for (int o = 0; o < c.nops; o++) {
            run_op<R, CS>(psi, c.n, ops[o], data, vt, tid, rank, sm, smem_log);
            team_sync<CS>();
        }
        if (c.flags & 2) {
            // FP64 sums in a fixed order: ||psi||^2, P(top qubit = 1), P(slice)
            double s_all = 0.0, s_hi = 0.0;
            for (unsigned i = vt; i < N; i += kTeam) {
                const V z = psi[i];
                const double q = (double)z.x * (double)z.x + (double)z.y * (double)z.y;
                s_all += q;
                if (i >= N / 2) s_hi += q;
            }
            const unsigned Db = 1u << c.nb;
            double s_sl = 0.0;
            for (unsigned i = vt; i < Db; i += kTeam) {
                const V z = psi[N / 2 + i];
                s_sl += (double)z.x * (double)z.x + (double)z.y * (double)z.y;
                c.result[4 + 2 * i] = (double)z.x;
                c.result[4 + 2 * i + 1] = (double)z.y;
            }
            block_sum3<kThreads>(s_all, s_hi, s_sl, red);
            if (CS == 1) {
                if (tid == 0) {
                    c.result[0] = s_all;
                    c.result[1] = s_hi;
                    c.result[2] = s_sl;
                }
            } else {
                if (tid == 0) {
                    st_cluster(&part[3 * rank], 0u, s_all);
                    st_cluster(&part[3 * rank + 1], 0u, s_hi);
                    st_cluster(&part[3 * rank + 2], 0u, s_sl);
                }
                team_sync<CS>();
                if (rank == 0 && tid == 0) {
                    double a = 0.0, b = 0.0, d = 0.0;
                    for (int r = 0; r < CS; r++) {
                        a += part[3 * r];
                        b += part[3 * r + 1];
                        d += part[3 * r + 2];
                    }
                    c.result[0] = a;
                    c.result[1] = b;
                    c.result[2] = d;
                }
            }
        }
        if (psi == sm)
            for (unsigned i = tid; i < N; i += kThreads) g[i] = psi[i];
        team_sync<CS>();
    }
}

}  // namespace batch
}  // namespace qsim

// ------------------------------------------------------------------------------- host side
struct qsim_batch {
    int count = 0, dtype = 0, smem_amps = 0, stage_bytes = 0, grid = 1;
    int nbig = 0, grid_big = 0;  // circuits run by cluster teams (the first nbig of the order)
    size_t smem_bytes = 0;
    bool hhl = false;
    void *dev = nullptr;  // one allocation: circs | order | counter | ops | data | results
    size_t dev_bytes = 0;
    qsim::batch::BCirc *d_circs = nullptr;
    int *d_order = nullptr;
    unsigned *d_counter = nullptr;
    double *d_results = nullptr;
    size_t results_doubles = 0;
    double *h_results = nullptr;  // pinned mirror
    struct Meta {
        int N = 0, nb = 0, x_off = 0;
        double C = 1, norm_b = 1;
        size_t roff = 0;
    };
    std::vector<Meta> meta;
    bool external = false;  // device tables and pinned results owned by the serving pool
    bool results_on_host = false;  // the kernel writes the readout into h_results directly
    ~qsim_batch() {
        if (external) return;
        if (dev) cudaFree(dev);
        if (h_results) cudaFreeHost(h_results);
    }
};

namespace qsim {
namespace {

using batch::BOp;

template <typename R>
void configure_batch(qsim_batch *B);

void put_v(std::vector<unsigned char> &blob, int dtype, const cd &z) {
    if (dtype == QSIM_C128) {
        double v[2] = {z.real(), z.imag()};
        blob.insert(blob.end(), (unsigned char *)v, (unsigned char *)v + 16);
    } else {
        float v[2] = {(float)z.real(), (float)z.imag()};
        blob.insert(blob.end(), (unsigned char *)v, (unsigned char *)v + 8);
    }
}

size_t vbytes(int dtype) { return dtype == QSIM_C128 ? 16 : 8; }

// Rotation r of a register given bit by bit: controls[j] = c0 + ((j + r) mod nc) with c0 the
// lowest qubit; -1 if the list is not a rotated contiguous register.
int register_rotation(const std::vector<int> &controls) {
    const int nc = (int)controls.size();
    if (nc == 0) return -1;
    const int c0 = *std::min_element(controls.begin(), controls.end());
    for (int r = 0; r < nc; r++) {
        bool ok = true;
        for (int j = 0; j < nc && ok; j++) ok = controls[j] == c0 + (j + r) % nc;
        if (ok) return r;
    }
    return -1;
}

bool contiguous_ascending(const std::vector<int> &q) {
    for (size_t j = 1; j < q.size(); j++)
        if (q[j] != q[0] + (int)j) return false;
    return true;
}

unsigned maskq(const std::vector<int> &q) {
    unsigned m = 0;
    for (int x : q) m |= 1u << x;
    return m;
}

// Translate one executable op; returns false if the batched kernel does not support it.
bool encode(const Op &op, int dtype, std::vector<unsigned char> &data, BOp &b) {
    std::memset(&b, 0, sizeof(b));
    const size_t el = data.size() / vbytes(dtype);
    b.data = (unsigned)el;
    switch (op.kind) {
        case OP_DENSE: {
            const int k = (int)op.targets.size();
            if (k > 5) return false;
            b.kind = batch::B_DENSE;
            b.k = (unsigned char)k;
            b.c0 = op.real_u ? 1 : 0;  // B_DENSE: real U flag
            for (int i = 0; i < k; i++) b.t[i] = (signed char)op.targets[i];
            b.cmask = maskq(op.controls);
            b.fixmask = maskq(op.targets) | b.cmask;
            for (const cd &z : op.U) put_v(data, dtype, z);  // row-major
            return true;
        }
        case OP_PHASE:
            b.kind = batch::B_PHASE;
            b.cmask = b.fixmask = maskq(op.targets);
            put_v(data, dtype, op.phase);
            return true;
        case OP_DIAG: {
            const int k = (int)op.targets.size();
            if (k > 8) return false;
            b.kind = batch::B_DIAG;
            b.k = (unsigned char)k;
            for (int i = 0; i < k; i++) b.t[i] = (signed char)op.targets[i];
            b.cmask = maskq(op.controls);
            b.fixmask = b.cmask;  // (k counted separately in the enumeration)
            for (const cd &z : op.U) put_v(data, dtype, z);
            return true;
        }
        case OP_SWAP:
            b.kind = batch::B_SWAP;
            b.t[0] = (signed char)op.targets[0];
            b.t[1] = (signed char)op.targets[1];
            b.cmask = maskq(op.controls);
            b.fixmask = maskq(op.targets) | b.cmask;
            return true;
        case OP_UCRY: {
            const int nc = (int)op.controls.size();
            for (int j = 1; j < nc; j++)
                if (op.controls[j] != op.controls[0] + j) return false;
            b.kind = batch::B_UCRY;
            b.t[0] = (signed char)op.targets[0];
            b.c0 = (unsigned char)op.controls[0];
            b.nreg = (unsigned char)nc;
            for (double th : op.theta) put_v(data, dtype, cd(std::cos(0.5 * th), std::sin(0.5 * th)));
            return true;
        }
        case OP_HHL_INVERT: {
            const int nc = (int)op.controls.size();
            const int rot = register_rotation(op.controls);
            if (rot < 0) return false;
            b.kind = batch::B_INVERT;
            b.k = op.sign == -1 ? 1 : 0;
            b.t[0] = (signed char)op.targets[0];
            b.t[1] = (signed char)rot;
            b.c0 = (unsigned char)*std::min_element(op.controls.begin(), op.controls.end());
            b.nreg = (unsigned char)nc;
            put_v(data, dtype, cd(op.tq, 0.0));
            return true;
        }
        case OP_QPE_PHASE: {
            const int nb = (int)op.targets.size(), m = (int)op.controls.size();
            for (int i = 0; i < nb; i++)
                if (op.targets[i] != i) return false;
            for (int j = 0; j < m; j++)
                if (op.controls[j] != nb + j) return false;
            std::vector<cd> lo, hi;
            int h = 0;
            qpe_phase_tables(op, lo, hi, h);
            b.kind = batch::B_QPE;
            b.k = (unsigned char)nb;
            b.nreg = (unsigned char)m;
            b.c0 = (unsigned char)h;
            for (const cd &z : lo) put_v(data, dtype, z);
            b.data2 = (unsigned)(data.size() / vbytes(dtype));
            for (const cd &z : hi) put_v(data, dtype, z);
            return true;
        }
        case OP_DFT: {
            const int K = (int)op.targets.size(), ns = (int)op.controls.size();
            if (K > 10 || K + ns > 20 || !contiguous_ascending(op.targets) || !contiguous_ascending(op.controls))
                return false;
            std::vector<cd> W, Tlo, Thi;
            dft_tables(op, W, Tlo, Thi);
            b.kind = batch::B_DFT;
            b.k = (unsigned char)K;
            b.c0 = (unsigned char)op.targets[0];
            b.nreg = (unsigned char)ns;
            b.t[0] = (signed char)(ns ? op.controls[0] : 0);
            b.t[1] = (signed char)(ns == 0 ? 0 : (op.pre ? 1 : 2));
            b.t[2] = (signed char)op.sign;
            b.t[3] = (signed char)((K + ns) / 2);  // the split dft_tables uses
            for (const cd &z : W) put_v(data, dtype, z);
            b.data2 = (unsigned)(data.size() / vbytes(dtype));
            for (const cd &z : Tlo) put_v(data, dtype, z);
            for (const cd &z : Thi) put_v(data, dtype, z);
            return true;
        }
        case OP_WALSH: {
            std::vector<int> q = op.targets;
            std::sort(q.begin(), q.end());
            if (q.size() > 10 || !contiguous_ascending(q)) return false;
            b.kind = batch::B_WALSH;
            b.k = (unsigned char)q.size();
            b.c0 = (unsigned char)q[0];
            return true;
        }
    }
    return false;
}

// log2 of the amplitudes a CTA keeps in shared memory
int batch_smem_log(int dtype) { return dtype == QSIM_C128 ? 13 : 14; }

double circuit_cost(const qsim_circuit *c) {
    double s = 0;
    for (const Op &op : c->ops) s += (op.kind == OP_DENSE ? (double)(1 << op.targets.size()) : 1.0);
    return s * std::ldexp(1.0, c->n);
}

}  // namespace

// Host image of a batch: every table the kernel reads, laid out as one device allocation.
// Device pointers inside the circuit descriptors are patched once the base address is known.
struct BatchImage {
    std::vector<unsigned char> host;
    size_t o_circs = 0, o_order = 0, o_counter = 0, o_ops = 0, o_data = 0, o_res = 0, total = 0;
    std::vector<size_t> op_first, data_first;
    size_t results = 0;
    std::vector<qsim_batch::Meta> meta;
    int count = 0, dtype = 0, max_n = 0;
    int nbig = 0;  // circuits whose state exceeds one CTA's shared memory (first in the order)
    size_t stage_bytes = 0;  // shared memory for the largest circuit's data and op list (capped)
    bool hhl = false;
};

// Shared memory set aside per CTA for a circuit's data and op list (larger ones stay in global
// memory; an op list alone is staged when it fits).
constexpr size_t kStageCap = 32768;

BatchImage batch_image(const std::vector<const qsim_circuit *> &cs, const std::vector<const hhl_circuit *> &hs,
                       void *const *states, int dtype) {
    BatchImage im;
    const int count = (int)cs.size();
    im.count = count;
    im.dtype = dtype;
    im.hhl = !hs.empty();
    std::vector<BOp> ops;
    std::vector<unsigned char> data;
    std::vector<batch::BCirc> circs(count);
    im.op_first.resize(count);
    im.data_first.resize(count);
    im.meta.resize(count);
    for (int i = 0; i < count; i++) {
        const qsim_circuit *c = cs[i];
        build_ops(const_cast<qsim_circuit *>(c));
        QSIM_REQUIRE(c->n <= 30, "batched states are limited to 30 qubits");
        QSIM_REQUIRE(states[i] != nullptr, "NULL state");
        im.max_n = std::max(im.max_n, c->n);
        while (data.size() % 256) data.push_back(0);
        im.data_first[i] = data.size();
        im.op_first[i] = ops.size();
        std::vector<unsigned char> local;
        for (const Op &op : c->ops) {
            BOp b;
            QSIM_REQUIRE(encode(op, dtype, local, b), "operation not supported by the batched executor "
                                                      "(dense gates wider than 5 qubits or a scattered "
                                                      "rotation register): fuse with max_k <= 5");
            ops.push_back(b);
        }
        batch::BCirc &bc = circs[i];
        std::memset(&bc, 0, sizeof(bc));
        bc.n = c->n;
        bc.nops = (int)c->ops.size();
        bc.state = states[i];
        if (im.hhl) {
            const hhl_circuit *h = hs[i];
            QSIM_REQUIRE(h->n == c->n, "HHL circuit and gate list disagree on the qubit count");
            bc.flags = 3;
            bc.nb = h->nb;
            bc.b_off = (unsigned)(local.size() / vbytes(dtype));
            for (const cd &z : h->b_pad) put_v(local, dtype, z);
            im.meta[i].N = h->N;
            im.meta[i].x_off = h->x_off;
            im.meta[i].nb = h->nb;
            im.meta[i].C = h->C;
            im.meta[i].norm_b = h->norm_b;
            im.meta[i].roff = im.results;
            im.results += 4 + 2 * ((size_t)1 << h->nb);
        }
        bc.data_bytes = (unsigned)local.size();
        im.stage_bytes = std::max(im.stage_bytes, ((local.size() + 15) & ~(size_t)15) + sizeof(BOp) * c->ops.size());
        data.insert(data.end(), local.begin(), local.end());
    }
    im.stage_bytes = std::min(im.stage_bytes, kStageCap);
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> cost(count);
    for (int i = 0; i < count; i++) cost[i] = circuit_cost(cs[i]);
    // states larger than one CTA's shared memory go to the cluster teams (a launch of their
    // own): they come first; each part in order of decreasing cost
    const int cap_log = batch_smem_log(dtype);
    auto big = [&](int i) { return cs[i]->n > cap_log; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (big(a) != big(b)) return big(a);
        return cost[a] > cost[b];
    });
    for (int i = 0; i < count; i++) im.nbig += big(i) ? 1 : 0;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    im.o_circs = 0;
    im.o_order = al(im.o_circs + sizeof(batch::BCirc) * count);
    im.o_counter = al(im.o_order + sizeof(int) * count);
    im.o_ops = al(im.o_counter + 256);
    im.o_data = al(im.o_ops + sizeof(BOp) * std::max<size_t>(1, ops.size()));
    im.o_res = al(im.o_data + std::max<size_t>(1, data.size()));
    im.total = al(im.o_res + sizeof(double) * std::max<size_t>(1, im.results));
    im.host.assign(im.o_res, 0);  // results are written by the kernel, not uploaded
    std::memcpy(im.host.data() + im.o_circs, circs.data(), sizeof(batch::BCirc) * count);
    std::memcpy(im.host.data() + im.o_order, order.data(), sizeof(int) * count);
    if (!ops.empty()) std::memcpy(im.host.data() + im.o_ops, ops.data(), sizeof(BOp) * ops.size());
    if (!data.empty()) std::memcpy(im.host.data() + im.o_data, data.data(), data.size());
    return im;
}

// Patch the device pointers of `im` for base address `dev` and build the batch object.
// external: `dev` (im.total bytes) and `pinned_results` belong to the caller and the tables
// are uploaded asynchronously on `st`; otherwise the batch allocates and uploads synchronously.
qsim_batch *batch_from_image(BatchImage &im, void *dev, double *pinned_results, cudaStream_t st) {
    std::unique_ptr<qsim_batch> B(new qsim_batch());
    B->count = im.count;
    B->dtype = im.dtype;
    B->hhl = im.hhl;
    B->meta = im.meta;
    const bool external = dev != nullptr;
    B->external = external;
    if (!external) {
        cudaError_t e = cudaMalloc(&dev, im.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error(QSIM_ENOMEM, std::string("cudaMalloc for batch tables: ") + cudaGetErrorString(e));
        }
    }
    B->dev = dev;
    B->dev_bytes = im.total;
    cudaError_t e;
    if (im.results && !external) {
        // pinned host memory is device-accessible under unified addressing: the kernel writes
        // the readout there itself, so reading the results needs no copy, only the stream's end
        e = cudaMallocHost(&B->h_results, sizeof(double) * im.results);
        if (e != cudaSuccess) throw Error(QSIM_ENOMEM, "pinned host buffer for batch results");
        B->results_on_host = true;
    }
    unsigned char *base = static_cast<unsigned char *>(dev);
    double *res = B->results_on_host ? B->h_results : reinterpret_cast<double *>(base + im.o_res);
    batch::BCirc *hc = reinterpret_cast<batch::BCirc *>(im.host.data() + im.o_circs);
    for (int i = 0; i < im.count; i++) {
        hc[i].ops = reinterpret_cast<const BOp *>(base + im.o_ops) + im.op_first[i];
        hc[i].data = base + im.o_data + im.data_first[i];
        hc[i].result = im.hhl ? res + im.meta[i].roff : nullptr;
    }
    if (external) {
        // from pageable memory: the call returns once the source has been staged
        e = cudaMemcpyAsync(dev, im.host.data(), im.host.size(), cudaMemcpyHostToDevice, st);
    } else {
        e = cudaMemcpy(dev, im.host.data(), im.host.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("uploading batch tables: ") + cudaGetErrorString(e));
    B->d_circs = reinterpret_cast<batch::BCirc *>(base + im.o_circs);
    B->d_order = reinterpret_cast<int *>(base + im.o_order);
    B->d_counter = reinterpret_cast<unsigned *>(base + im.o_counter);
    B->d_results = reinterpret_cast<double *>(base + im.o_res);
    B->results_doubles = im.results;
    if (im.results && external) B->h_results = pinned_results;
    const int cap_amps = 1 << batch_smem_log(im.dtype);
    B->smem_amps = std::min(cap_amps, 1 << im.max_n);
    B->nbig = im.nbig;
    B->stage_bytes = (int)im.stage_bytes;
    if (im.dtype == QSIM_C128) configure_batch<double>(B.get());
    else configure_batch<float>(B.get());
    return B.release();
}

qsim_batch *make_batch(const std::vector<const qsim_circuit *> &cs, const std::vector<const hhl_circuit *> &hs,
                       void *const *states, int dtype) {
    BatchImage im = batch_image(cs, hs, states, dtype);
    return batch_from_image(im, nullptr, nullptr, nullptr);
}

bool batch_supported(const qsim_circuit *c) {
    build_ops(const_cast<qsim_circuit *>(c));
    if (c->n > 30) return false;
    for (const Op &op : c->ops) {
        if (op.kind == OP_DFT &&
            (op.targets.size() > 10 || op.targets.size() + op.controls.size() > 20 ||
             !contiguous_ascending(op.targets) || !contiguous_ascending(op.controls)))
            return false;
        if (op.kind == OP_WALSH) {
            std::vector<int> q = op.targets;
            std::sort(q.begin(), q.end());
            if (q.size() > 10 || !contiguous_ascending(q)) return false;
        }
        if (op.kind == OP_DENSE && op.targets.size() > 5) return false;
        if (op.kind == OP_DIAG && op.targets.size() > 8) return false;
        if (op.kind == OP_UCRY && !contiguous_ascending(op.controls)) return false;
        if (op.kind == OP_HHL_INVERT && register_rotation(op.controls) < 0) return false;
        if (op.kind == OP_QPE_PHASE) {
            for (size_t i = 0; i < op.targets.size(); i++)
                if (op.targets[i] != (int)i) return false;
            for (size_t j = 0; j < op.controls.size(); j++)
                if (op.controls[j] != (int)(op.targets.size() + j)) return false;
        }
    }
    return true;
}

BatchImage *batch_plan(const std::vector<const qsim_circuit *> &cs, const std::vector<const hhl_circuit *> &hs,
                       void *const *states, int dtype) {
    return new BatchImage(batch_image(cs, hs, states, dtype));
}
size_t batch_plan_device_bytes(const BatchImage *im) { return im->total; }
size_t batch_plan_result_doubles(const BatchImage *im) { return im->results; }
void batch_plan_free(BatchImage *im) { delete im; }
qsim_batch *batch_instantiate(BatchImage *im, void *dev, double *pinned, cudaStream_t st) {
    return batch_from_image(*im, dev, pinned, st);
}

namespace {

// Kernel attributes and the grid are fixed when the batch is created, so that a run is only a
// launch (capturable into a CUDA graph).
constexpr int kTeamCTAs = 4;  // CTAs of a cluster team (a 16-qubit complex64 state is 4 tiles of 2^14)

// Occupancy of the two batched kernels for a dynamic shared-memory size, queried once per
// (device, type, size): batches are created on the serving pool's hot path.
struct BatchOcc {
    int per_sm = 1, clusters = 0;
};

template <typename R>
BatchOcc batch_occupancy(size_t smem, bool need_clusters) {
    static std::mutex mu;
    static std::map<std::pair<int, size_t>, BatchOcc> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const std::pair<int, size_t> key(dev, smem);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end() && (!need_clusters || it->second.clusters > 0)) return it->second;
    }
    constexpr int kThreads = batch::Threads<typename batch::C2<R>::T>::n;
    BatchOcc o;
    // the kernels' dynamic shared-memory limit is set once to the device's opt-in maximum, so
    // that a launch of any batch size is covered whatever size was configured last
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // (less the kernel's own static shared memory)
    auto dyn_max = [&](const void *k) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) throw Error(QSIM_ECUDA, "batched kernel attributes");
        const int m = optin - (int)fa.sharedSizeBytes;
        QSIM_REQUIRE((size_t)m >= smem, "batched kernel: shared memory per CTA exceeds the device limit");
        return m;
    };
    auto kern = batch::batched_kernel<R, 1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         dyn_max(reinterpret_cast<const void *>(kern)));
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("batched kernel attribute: ") + cudaGetErrorString(e));
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.per_sm, kern, kThreads, smem);
    if (e != cudaSuccess || o.per_sm < 1) o.per_sm = 1;
    if (need_clusters) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        auto kc = batch::batched_kernel<R, kTeamCTAs>;
        e = cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dyn_max(reinterpret_cast<const void *>(kc)));
        if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("batched kernel attribute: ") + cudaGetErrorString(e));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = kTeamCTAs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(kTeamCTAs * std::max(1, sms / kTeamCTAs)));
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(&o.clusters, kc, &cfg);
        if (e != cudaSuccess || o.clusters < 1) {
            cudaGetLastError();
            throw Error(QSIM_ECUDA, "batched kernel: no cluster of 4 CTAs fits on the device");
        }
    }
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = o;
    return o;
}

template <typename R>
void configure_batch(qsim_batch *B) {
    const size_t smem = (((size_t)B->smem_amps * vbytes(B->dtype) + 15) & ~(size_t)15) + (size_t)B->stage_bytes;
    const BatchOcc o = batch_occupancy<R>(smem, B->nbig > 0);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    B->grid = std::max(1, std::min(B->count - B->nbig, sms * o.per_sm));
    B->smem_bytes = smem;
    B->grid_big = B->nbig > 0 ? kTeamCTAs * std::min(B->nbig, o.clusters) : 0;
}

// The work counters are zero when the batch is uploaded and the kernels leave them at zero:
// the cluster teams take the first nbig circuits of the order (counter 0), single CTAs the rest
// (counter 32, its own cache line).
template <typename R>
void launch_batch(qsim_batch *B, cudaStream_t st) {
    constexpr int kThreads = batch::Threads<typename batch::C2<R>::T>::n;
    if (B->nbig > 0) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = kTeamCTAs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)B->grid_big);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = B->smem_bytes;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const batch::BCirc *circs = B->d_circs;
        const int *order = B->d_order;
        cudaError_t e = cudaLaunchKernelEx(&cfg, batch::batched_kernel<R, kTeamCTAs>, circs, order, B->nbig, B->d_counter,
                                           B->smem_amps, B->stage_bytes);
        if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("batched kernel (teams): ") + cudaGetErrorString(e));
        note_launches(1, QSIM_KERNEL_BATCHED);
    }
    if (B->count > B->nbig) {
        batch::batched_kernel<R, 1><<<B->grid, kThreads, B->smem_bytes, st>>>(B->d_circs, B->d_order + B->nbig, B->count - B->nbig,
                                                                             B->d_counter + 32, B->smem_amps, B->stage_bytes);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("batched kernel: ") + cudaGetErrorString(e));
        note_launches(1, QSIM_KERNEL_BATCHED);
    }
}

void run_batch(qsim_batch *B, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (B->count == 0) return;
    if (B->dtype == QSIM_C128) launch_batch<double>(B, st);
    else launch_batch<float>(B, st);
}

}  // namespace

void batch_launch(qsim_batch *b, cudaStream_t st) { run_batch(b, st); }

void batch_enqueue_results(qsim_batch *b, cudaStream_t st) {
    if (!b->results_doubles || b->results_on_host) return;
    cudaError_t e = cudaMemcpyAsync(b->h_results, b->d_results, sizeof(double) * b->results_doubles,
                                    cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("batch results: ") + cudaGetErrorString(e));
}

void batch_host_result(const qsim_batch *b, int i, double *x_out, hhl_readout_stats *stats) {
    const qsim_batch::Meta &m = b->meta[i];
    const double *r = b->h_results + m.roff;
    const double P = r[1], P0 = r[2];
    const double inv = P0 > 0 ? 1.0 / std::sqrt(P0) : 0.0;
    const double norm_x = std::sqrt(P) / m.C;
    if (x_out)
        for (int j = 0; j < m.N; j++) {
            x_out[2 * j] = r[4 + 2 * (m.x_off + j)] * inv * norm_x * m.norm_b;
            x_out[2 * j + 1] = r[4 + 2 * (m.x_off + j) + 1] * inv * norm_x * m.norm_b;
        }
    if (stats) {
        stats->p_success = P;
        stats->p_clock0 = P0;
        stats->leakage = P - P0;
        stats->norm2 = r[0];
        stats->norm_x = norm_x;
        stats->norm_b = m.norm_b;
    }
}

}  // namespace qsim

using namespace qsim;

extern "C" {

int qsim_batch_create(const qsim_circuit *const *cs, void *const *states, int count, int dtype, qsim_batch **out) {
    return guarded([&] {
        QSIM_REQUIRE(out != nullptr && count >= 0 && (count == 0 || (cs && states)), "bad arguments");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        std::vector<const qsim_circuit *> v(cs, cs + count);
        for (auto *c : v) QSIM_REQUIRE(c != nullptr, "NULL circuit");
        *out = make_batch(v, {}, states, dtype);
    });
}

int hhl_batch_create(const hhl_circuit *const *hs, const qsim_circuit *const *fused, void *const *states, int count,
                     int dtype, qsim_batch **out) {
    return guarded([&] {
        QSIM_REQUIRE(out != nullptr && count >= 0 && (count == 0 || (hs && states)), "bad arguments");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        std::vector<const qsim_circuit *> v(count);
        std::vector<const hhl_circuit *> h(hs, hs + count);
        for (int i = 0; i < count; i++) {
            QSIM_REQUIRE(h[i] != nullptr, "NULL HHL circuit");
            v[i] = (fused && fused[i]) ? fused[i] : &h[i]->circ;
        }
        *out = make_batch(v, h, states, dtype);
    });
}

int qsim_batch_run(qsim_batch *b, void *stream) {
    return guarded([&] {
        QSIM_REQUIRE(b != nullptr, "NULL batch");
        run_batch(b, stream);
    });
}

}  // extern "C"

namespace {

void collect_results(qsim_batch *b, void *stream, double *x_out, hhl_readout_stats *stats) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (b->results_doubles) {
        cudaError_t e = cudaSuccess;
        if (!b->results_on_host)
            e = cudaMemcpyAsync(b->h_results, b->d_results, sizeof(double) * b->results_doubles,
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("batch results: ") + cudaGetErrorString(e));
    }
    size_t xo = 0;
    for (int i = 0; i < b->count; i++) {
        const qsim_batch::Meta &m = b->meta[i];
        const double *r = b->h_results + m.roff;
        const double P = r[1], P0 = r[2];
        const double inv = P0 > 0 ? 1.0 / std::sqrt(P0) : 0.0;
        const double norm_x = std::sqrt(P) / m.C;
        if (x_out)
            for (int j = 0; j < m.N; j++) {
                x_out[2 * (xo + j)] = r[4 + 2 * (m.x_off + j)] * inv * norm_x * m.norm_b;
                x_out[2 * (xo + j) + 1] = r[4 + 2 * (m.x_off + j) + 1] * inv * norm_x * m.norm_b;
            }
        xo += m.N;
        if (stats) {
            stats[i].p_success = P;
            stats[i].p_clock0 = P0;
            stats[i].leakage = P - P0;
            stats[i].norm2 = r[0];
            stats[i].norm_x = norm_x;
            stats[i].norm_b = m.norm_b;
        }
    }
}

}  // namespace

extern "C" {

int hhl_batch_results(qsim_batch *b, void *stream, double *x_out, hhl_readout_stats *stats) {
    return guarded([&] {
        QSIM_REQUIRE(b != nullptr && b->hhl, "not an HHL batch");
        collect_results(b, stream, x_out, stats);
    });
}

int hhl_batch_solve(qsim_batch *b, void *stream, double *x_out, hhl_readout_stats *stats) {
    return guarded([&] {
        QSIM_REQUIRE(b != nullptr && b->hhl, "not an HHL batch");
        run_batch(b, stream);
        collect_results(b, stream, x_out, stats);
    });
}

void qsim_batch_free(qsim_batch *b) { delete b; }

int hhl_batch_autotune(const hhl_circuit *const *hs, void *const *states, int count, int dtype,
                       const int *candidates, int ncand, void *stream, int *best_k, double *ms_out) {
    return guarded([&] {
        QSIM_REQUIRE(hs && states && best_k && count > 0 && candidates && ncand > 0, "bad arguments");
        QSIM_REQUIRE(dtype == QSIM_C64 || dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        std::vector<const hhl_circuit *> h(hs, hs + count);
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
            throw Error(QSIM_ECUDA, "cudaEventCreate");
        double best = 1e300;
        int bk = -1;
        try {
            for (int ci = 0; ci < ncand; ci++) {
                const int k = candidates[ci];
                QSIM_REQUIRE(k >= 1 && k <= 5, "candidate fusion widths must be in 1..5");
                std::vector<std::unique_ptr<qsim_circuit>> fused;
                std::vector<const qsim_circuit *> v(count);
                for (int i = 0; i < count; i++) {
                    qsim_circuit *f = nullptr;
                    if (qsim_fuse(&h[i]->circ, k, &f) != QSIM_OK) throw Error(QSIM_EINVAL, qsim_last_error());
                    fused.emplace_back(f);
                    v[i] = f;
                }
                std::unique_ptr<qsim_batch> B(make_batch(v, h, states, dtype));
                run_batch(B.get(), stream);  // warm-up
                cudaEventRecord(e0, st);
                for (int r = 0; r < 2; r++) run_batch(B.get(), stream);
                cudaEventRecord(e1, st);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                const double per = ms / 2.0;
                if (ms_out) ms_out[ci] = per;
                if (per < best) {
                    best = per;
                    bk = k;
                }
            }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *best_k = bk;
    });
}

int qsim_apply_batched(void *const *states, const int *n_qubits, const qsim_circuit *const *cs, int count, int dtype,
                       void *stream) {
    return guarded([&] {
        QSIM_REQUIRE(count >= 0 && (count == 0 || (states && n_qubits && cs)), "bad arguments");
        for (int i = 0; i < count; i++)
            QSIM_REQUIRE(cs[i] != nullptr && n_qubits[i] == cs[i]->n, "state qubit count does not match its circuit");
        if (count == 0) return;
        std::vector<const qsim_circuit *> v(cs, cs + count);
        std::unique_ptr<qsim_batch> B(make_batch(v, {}, states, dtype));
        run_batch(B.get(), stream);
        // the batch tables must outlive the launch
        cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("batched apply: ") + cudaGetErrorString(e));
    });
}

}  // extern "C"
