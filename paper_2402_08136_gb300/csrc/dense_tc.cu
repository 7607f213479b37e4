// Dense k-qubit gate on a complex64 state with the 5th-generation tensor cores (sm_103a):
// tcgen05.mma kind::tf32, accumulators in tensor memory, split-precision "3xTF32" products.
//
// The update of every group of 2^k amplitudes (the amplitudes that differ only in the target
// bits) is a complex matrix-vector product; 128 groups at a time it is the real GEMM
//     Y[128 x 2D] = X[128 x 2D] * B^T,   D = 2^k,
// where row m of X holds group m's amplitudes as (re_0, im_0, re_1, im_1, ...) and B is the
// real 2D x 2D form of U: B[2r][2c] = B[2r+1][2c+1] = Re U[r][c], B[2r][2c+1] = -Im U[r][c],
// B[2r+1][2c] = Im U[r][c].  Each FP32 operand is split into a TF32 "hi" part and a TF32 "lo"
// part (x - hi rounded to TF32); Y = Xhi Bhi^T + Xhi Blo^T + Xlo Bhi^T accumulates in FP32,
// which keeps ~22 significant bits per product (Markidis et al., "NVIDIA Tensor Core
// Programmability, Performance & Precision", 2018, for the split scheme).
//
// CTA (persistent, one per SM: it allocates all 512 tensor-memory columns): 21 warps in three
// roles coupled only through mbarriers.  16 producer warps load chunks of 16 amplitudes
// (32 K-columns) per group row, keeping six chunks of loads in flight in registers, and split
// them into TF32 hi/lo; one lane of the MMA warp waits for full chunks, issues the 3 x 4 MMAs of
// a chunk and commits them to the chunk's "empty" barrier (and, after a tile's last chunk, to
// the accumulator's barrier); 4 epilogue warps (one per TMEM lane subpartition) read a finished
// accumulator, store its outputs straight to HBM and hand it back.  Two accumulators alternate
// between tiles, so the MMAs of one tile overlap the epilogue of the previous one.
//
// The operand the MMA reads once per issue from shared memory is the bound: a 128 x 128 x 8
// TF32 MMA with both operands in shared memory reads 8 KB, more than shared memory delivers in
// the MMA's own time.  So one operand always lives in tensor memory:
//   - group-major form (dense_tc_gm_kernel, any targets but the transposed case): X in tensor
//     memory, written by the producers with tcgen05.st into a ring of chunk slots, U (B
//     operand) in shared memory;
//   - transposed form (dense_tc_tr_kernel, 6 targets on the low qubits: qubits 0 and 1, or
//     qubit 0 or qubit 1 with the other free and few free qubits below 4; gates of 1..5
//     targets there are widened to it by the host) and real 7-target gates
//     (dense_tc_real7_kernel): U is the A operand and sits in tensor memory, X chunks (B
//     operand) in a six-deep shared-memory ring.
//
// Shared-memory operand layout (no swizzle, K-major): 8-row x 16-byte core matrices; core
// matrices adjacent along K are 128 bytes apart (leading byte offset), adjacent along M/N
// (K/4) * 128 bytes apart (stride byte offset).  The host packs U in that layout; u_to_tmem
// reads it from there into tensor memory.
//
// Every wait on an mbarrier is bounded; on timeout the kernel raises a flag in device memory
// (read by qsim_device_status), skips the remaining work, releases its tensor memory and exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "common.h"

namespace qsim {

__device__ unsigned int g_device_error = 0;

namespace tc {

constexpr int kM = 128;      // groups per tile (MMA M)
constexpr int kCH = 32;      // K-columns per chunk (16 complex amplitudes)
constexpr int kMaxFix = 40;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s

struct Args {
    void *psi;
    const float *Bg;          // B_hi then B_lo, canonical layout, N*KK floats each
    long long ntiles;         // groups / 128
    unsigned long long cmask;
    int nfix;
    int fix[kMaxFix];         // ascending: targets and controls
    int targets[8];
    // readout sums of the result (real 7-target kernel, when not NULL): sums[0] = 2 G (G = the
    // grid), sums[1 + c] = sum of |y|^2 over CTA c's outputs whose bit `hi_bit` is 0, sums[1 + G + c]
    // over those where it is 1
    double *sums;
    int hi_bit;
};

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t make_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, no swizzle
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
    return t;
}

// Bounded wait for the phase with the given parity to complete: gives up after about one
// second of wall-clock time and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    const unsigned a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (unsigned it = 0;; it++) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255) == 0) {
            const unsigned long long t = global_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kWaitLimitNs) return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mma_tf32(unsigned d_tmem, uint64_t adesc, uint64_t bdesc, unsigned idesc,
                                         unsigned accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on `bar` once every tcgen05 operation issued so far by this thread has completed
__device__ __forceinline__ void commit_to(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// TF32 of a finite float, rounded to nearest with ties away from zero: add half a TF32 unit in
// the last place to the magnitude bits and clear the 13 mantissa bits TF32 drops (integer
// arithmetic, so the producers' split does not queue on the conversion pipe; same bits as
// cvt.rna.tf32.f32 for finite inputs, and the state's entries are at most 1 in magnitude)
__device__ __forceinline__ unsigned to_tf32(float x) {
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

__device__ __forceinline__ unsigned long long insert_zeros(unsigned long long x, const int *pos, int cnt) {
    for (int i = 0; i < cnt; i++) {
        const int p = pos[i];
        x = ((x >> p) << (p + 1)) | (x & ((1ull << p) - 1ull));
    }
    return x;
}

template <int K>
struct Cfg {
    static constexpr int D = 1 << K;
    static constexpr int N = 2 * D;       // output reals per group
    static constexpr int KK = 2 * D;      // reduction length
    static constexpr int BBYTES = N * KK * 4;
    static constexpr unsigned IDESC = (1u << 4)          // D format F32
                                      | (2u << 7)        // A format TF32
                                      | (2u << 10)       // B format TF32
                                      | ((unsigned)(N >> 3) << 17) | ((unsigned)(kM >> 4) << 24);
};

// Warp roles: warps 0-15 produce (512 threads; thread t owns group row t % 128 and quarter
// t / 128 of every chunk), warps 16-19 run the epilogue (warp 16+i reads TMEM lanes
// 32i..32i+31), warp 20 issues the MMAs.  Roles hand chunks and accumulators to each other through
// mbarriers only, so no role waits for another except for data it needs.
constexpr int kProducers = 512;
constexpr int kAmpsPT = 16 * kM / kProducers;  // amplitudes of each chunk per producer thread
constexpr int kEpiWarp0 = kProducers / 32;
constexpr int kMmaWarp = kEpiWarp0 + 4;
constexpr int kThreadsWS = (kMmaWarp + 1) * 32;
constexpr int kPrefetch = 6;  // chunks of loads in flight per producer thread

// ---------------------------------------------------------------------------------------
// Group-major form with the X operand in tensor memory (any targets the transposed form does not
// take).  The same GEMM Y[128 x 2D] = X[128 x 2D] * B^T, but the MMA reads X (the A operand) from
// tensor memory instead of shared memory: producer thread (warp w, lane l) owns group row
// m = 32 (w mod 4) + l, which is exactly the TMEM lane its warp may write, and stores its hi and
// lo TF32 parts of each chunk with tcgen05.st into a ring of TMEM slots (64 columns: 32 hi, 32
// lo).  Shared memory then serves only B, which halves the shared-memory operand traffic of
// every MMA (a 128 x 2D x 8 MMA read 8 KB of shared memory per issue, more than the SM's shared
// memory delivers in the MMA's own time for 2D = 128), and the producers no longer write
// shared memory at all.  Tensor memory: NACC accumulators of 2D columns (two for 6 targets, four
// for 4 and 5, eight for 3) and chunk slots in the rest of the 512 columns.  21 warps (the register file is split over the SM's four sub-partitions, so the sub-partition
// holding 6 warps caps a thread at 80 registers: the producers keep 6 chunks of loads in flight
// within that).
template <int K>
struct GmCfg {
    static constexpr int D = 1 << K, N = 2 * D, KK = 2 * D;
    static constexpr int CA = D < 16 ? D : 16;         // amplitudes per chunk and group
    static constexpr int CK = 2 * CA;                  // K-columns per chunk
    static constexpr int NCH = KK / CK;                // chunks per tile
    // tiles per chunk: a 3-target tile is only 8 KB, so a chunk carries four of them (producer
    // warp h loads all 8 amplitudes of its row of tile h) and the hand-offs per chunk are paid
    // once per 32 KB
    static constexpr int TPC = K == 3 ? 4 : 1;
    static constexpr int APT = TPC > 1 ? CA : CA * kM / kProducers;  // amplitudes per chunk and thread
    static constexpr int PF = TPC > 1 ? 3 : kPrefetch * 4 / APT;     // chunks of loads in flight
    static constexpr int BBYTES = N * KK * 4;
    static constexpr int SLOT = TPC * 2 * CK;          // tensor-memory columns per chunk (hi, lo per tile)
    // accumulators in flight: narrow gates finish a tile every few hundred cycles, so more of
    // them keep the MMA -> epilogue hand-off off the critical path
    static constexpr int NACC = K == 3 ? 8 : (K == 6 ? 2 : 4);
    static constexpr int NB = (512 - NACC * N) / SLOT;  // tensor-memory chunk slots
    static constexpr int NBAR = 2 * NB + 2 * NACC + 1;   // full/empty per slot, accfull/accempty, drain
    static constexpr int SMEM = 2 * BBYTES + 8 * NBAR + 16 + 8 * D;
    static constexpr unsigned IDESC = Cfg<K>::IDESC;
};

// MMA with the A operand in tensor memory
__device__ __forceinline__ void mma_tf32_ta(unsigned d_tmem, unsigned a_tmem, uint64_t bdesc, unsigned idesc,
                                            unsigned accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tmem_st(unsigned taddr, const unsigned (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_st(unsigned taddr, const unsigned (&v)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
                 "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
                 : "memory");
}
__device__ __forceinline__ void tmem_st(unsigned taddr, const unsigned (&v)[4]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(taddr), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3])
                 : "memory");
}

template <int K>
__global__ void __launch_bounds__(kThreadsWS, 1) dense_tc_gm_kernel(const Args a) {
    using C = GmCfg<K>;
    constexpr int D = C::D, N = C::N, KK = C::KK, NCH = C::NCH, NB = C::NB, APT = C::APT, PF = C::PF;
    constexpr int TPC = C::TPC;
    static_assert(TPC == 1 || NCH == 1, "several tiles per chunk only when a tile is one chunk");
    extern __shared__ __align__(1024) unsigned char sm[];
    float *Bs = reinterpret_cast<float *>(sm);  // [2][N*KK]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + 2 * C::BBYTES);
    uint64_t *full = bars;                       // [NB] producer warps -> MMA (count 16)
    uint64_t *empty = bars + NB;                 // [NB] MMA completion -> producers (commit)
    uint64_t *accfull = bars + 2 * NB;           // [NACC] MMA completion -> epilogue (commit)
    uint64_t *accempty = accfull + C::NACC;      // [NACC] epilogue warps -> MMA (count 4)
    uint64_t *drain = accempty + C::NACC;        // MMA completion before tensor memory is freed
    unsigned *tslot = reinterpret_cast<unsigned *>(bars + C::NBAR);
    long long *toff = reinterpret_cast<long long *>(tslot + 4);  // D entries

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        const float4 *src = reinterpret_cast<const float4 *>(a.Bg);
        float4 *dst = reinterpret_cast<float4 *>(Bs);
        for (int i = tid; i < 2 * C::BBYTES / 16; i += kThreadsWS) dst[i] = src[i];
        for (int c = tid; c < D; c += kThreadsWS) {
            long long o = 0;
            for (int b = 0; b < K; b++)
                if ((c >> b) & 1) o |= 1ll << a.targets[b];
            toff[c] = o;
        }
        if (tid == 0) {
            for (int i = 0; i < NB; i++) {
                mbar_init(&full[i], kProducers / 32);
                mbar_init(&empty[i], 1);
            }
            for (int i = 0; i < C::NACC; i++) {
                mbar_init(&accfull[i], 1);
                mbar_init(&accempty[i], 4);
            }
            mbar_init(drain, 1);
        }
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                         "r"(512u)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    const unsigned tmem = *tslot;
    float2 *psi = reinterpret_cast<float2 *>(a.psi);
    const long long first = blockIdx.x, stride = gridDim.x;
    const long long ntl = first < a.ntiles ? (a.ntiles - first + stride - 1) / stride : 0;
    const long long total = (ntl + TPC - 1) / TPC * NCH;  // chunks
    bool failed = false;
    auto group_base = [&](long long tile_i, int m) -> unsigned long long {
        const unsigned long long gidx = (unsigned long long)(first + tile_i * stride) * kM + m;
        return insert_zeros(gidx, a.fix, a.nfix) | a.cmask;
    };

    if (warp < kEpiWarp0) {
        // ------------------------------------------------------------------ producers
        // thread: group row m (its TMEM lane), amplitudes APT h .. APT h + APT-1 of every chunk
        // (K-columns 2 APT h .. of the slot's hi and lo halves); with several tiles per chunk,
        // every amplitude of its row of the chunk's tile h
        const int q = warp & 3, h = warp >> 2, m = 32 * q + lane;
        float2 r[PF][APT];
        long long gb_tile = -1;
        unsigned long long gb_row = 0;
        auto load = [&](long long qq, float2(&rr)[APT]) {
            if (qq < total) {
                const long long t = TPC > 1 ? (qq / NCH) * TPC + h : qq / NCH;
                if (t >= ntl) return;  // past the CTA's last tile: the MMAs skip it
                if (t != gb_tile) {
                    gb_tile = t;
                    gb_row = group_base(t, m);
                }
                const int c0 = (int)(qq % NCH) * C::CA + (TPC > 1 ? 0 : APT * h);
#pragma unroll
                for (int e = 0; e < APT; e++) rr[e] = __ldcs(psi + gb_row + toff[c0 + e]);
            }
        };
#pragma unroll
        for (int p = 0; p < PF; p++) load(p, r[p]);
        for (long long q0 = 0; q0 < total && !failed; q0 += PF) {
#pragma unroll
            for (int p = 0; p < PF; p++) {
                const long long qq = q0 + p;
                if (qq >= total) break;
                const int b = (int)(qq % NB);
                if (qq >= NB) {  // the slot's previous chunk has been consumed by its MMAs
                    bool ok = mbar_wait(&empty[b], (unsigned)(((qq / NB) - 1) & 1));
                    ok = __all_sync(0xffffffffu, ok);  // the warp leaves together
                    if (!ok) {
                        failed = true;
                        break;
                    }
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const unsigned ta = tmem + ((unsigned)(32 * q) << 16) + (unsigned)(C::NACC * N + b * C::SLOT + (TPC > 1 ? h * 2 * C::CK : 2 * APT * h));
                unsigned v[2 * APT];
#pragma unroll
                for (int e = 0; e < APT; e++) {
                    v[2 * e] = to_tf32(r[p][e].x);
                    v[2 * e + 1] = to_tf32(r[p][e].y);
                }
                tmem_st(ta, v);
#pragma unroll
                for (int e = 0; e < APT; e++) {
                    v[2 * e] = to_tf32(r[p][e].x - __uint_as_float(to_tf32(r[p][e].x)));
                    v[2 * e + 1] = to_tf32(r[p][e].y - __uint_as_float(to_tf32(r[p][e].y)));
                }
                tmem_st(ta + (unsigned)C::CK, v);
                load(qq + PF, r[p]);
                asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[b]);
            }
        }
    } else if (warp < kMmaWarp) {
        // ------------------------------------------------------------------ epilogue
        const int sub = warp - kEpiWarp0;  // TMEM lane subpartition
        const int m = sub * 32 + lane;     // group row == TMEM lane
        for (long long t = 0; t < ntl && !failed; t++) {
            const int ab = (int)(t % C::NACC);
            bool ok = mbar_wait(&accfull[ab], (unsigned)((t / C::NACC) & 1));
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const unsigned long long gb = group_base(t, m);
            const unsigned acc = tmem + (unsigned)(ab * N) + ((unsigned)(sub * 32) << 16);
#pragma unroll
            for (int col = 0; col < N; col += 16) {
                unsigned v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                      "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(acc + (unsigned)col));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int i = 0; i < 8; i++)
                    __stcs(psi + gb + toff[col / 2 + i], make_float2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1])));
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[ab]);
        }
    } else if (lane == 0) {
        // ------------------------------------------------------------------ MMA issuer
        const unsigned b_hi = smem_u32(Bs), b_lo = b_hi + C::BBYTES;
        for (long long qq = 0; qq < total && !failed; qq++) {
            const int b = (int)(qq % NB);
            const int j = (int)(qq % NCH);         // chunk within its tile
            const long long t0 = (qq / NCH) * TPC;  // the chunk's first tile
            // before a tile's first chunk: its accumulator has been read out by the epilogue
            if (j == 0)
                for (int i = 0; i < TPC && !failed; i++) {
                    const long long t = t0 + i;
                    if (t < ntl && t >= C::NACC &&
                        !mbar_wait(&accempty[t % C::NACC], (unsigned)(((t / C::NACC) - 1) & 1)))
                        failed = true;
                }
            if (failed || !mbar_wait(&full[b], (unsigned)((qq / NB) & 1))) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            for (int i = 0; i < TPC; i++) {
                const long long t = t0 + i;
                if (t >= ntl) break;
                const int ab = (int)(t % C::NACC);
                const unsigned acc = tmem + (unsigned)(ab * N);
                const unsigned x_hi = tmem + (unsigned)(C::NACC * N + b * C::SLOT + i * 2 * C::CK),
                               x_lo = x_hi + (unsigned)C::CK;
#pragma unroll
                for (int kk = 0; kk < C::CK / 8; kk++) {
                    const unsigned boff = (j * (C::CK / 4) + kk * 2) * 128;  // 2 core matrices along K
                    const uint64_t dBh = make_desc(b_hi + boff, 128, KK * 32);
                    const uint64_t dBl = make_desc(b_lo + boff, 128, KK * 32);
                    mma_tf32_ta(acc, x_hi + 8u * kk, dBh, C::IDESC, (j == 0 && kk == 0) ? 0u : 1u);
                    mma_tf32_ta(acc, x_hi + 8u * kk, dBl, C::IDESC, 1u);
                    mma_tf32_ta(acc, x_lo + 8u * kk, dBh, C::IDESC, 1u);
                }
                if (j == NCH - 1) commit_to(&accfull[ab]);
            }
            commit_to(&empty[b]);
        }
        // every MMA issued has completed (or the bounded wait ran out) before tensor memory is
        // released
        commit_to(drain);
        if (!mbar_wait(drain, 0u)) failed = true;
    }
    if (failed) atomicOr(&g_device_error, 1u);
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512u) : "memory");
    }
}

// U as an MMA A operand in tensor memory.  Ug holds U's hi part and then its lo part, each 128
// rows n x 128 columns k in the canonical shared-memory layout (8-row x 16-byte core matrices,
// K-major).  Row n goes to TMEM lane n, column k to columns col0 + k (hi) and col0 + 128 + k (lo).
// Called by the 16 producer warps: warp w writes lanes 32 (w mod 4) .. +31 (the lanes its warp
// may access) and columns 32 (w / 4) .. +31 of each half.
__device__ __forceinline__ void u_to_tmem(const float *Ug, unsigned tmem, unsigned col0, int warp, int lane) {
    constexpr int KK = 128;
    const int q = warp & 3, part = warp >> 2, n = 32 * q + lane;
#pragma unroll
    for (int half = 0; half < 2; half++) {
        const char *src = reinterpret_cast<const char *>(Ug + (size_t)half * 128 * KK);
        unsigned v[32];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = 32 * part + 4 * i;
            const float4 f = __ldg(reinterpret_cast<const float4 *>(src + (size_t)(n >> 3) * (KK * 32) + (size_t)(k >> 2) * 128 +
                                                                    (size_t)(n & 7) * 16));
            v[4 * i] = __float_as_uint(f.x);
            v[4 * i + 1] = __float_as_uint(f.y);
            v[4 * i + 2] = __float_as_uint(f.z);
            v[4 * i + 3] = __float_as_uint(f.w);
        }
        const unsigned ta = tmem + ((unsigned)(32 * q) << 16) + col0 + (unsigned)(half * KK + 32 * part);
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
            "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(ta),
            "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
            "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
            "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
            "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
            : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// A tile's share of an epilogue thread's readout sums: 8 FP32 sums of 16 squares each, added in
// FP32 (at most 24 roundings: within 1.5e-6 of the exact sum of the 128 squares), then into the
// FP64 total of the tile's ancilla half.  One FP64 conversion and add per tile: FP64 runs at 1/64
// of the FP32 rate, and per 16 columns it held up the epilogue's stores.
__device__ __forceinline__ void tile_sum_into(float t, bool hi, double &s_lo, double &s_hi) {
    if (hi) s_hi += (double)t;
    else s_lo += (double)t;
}

// The CTA's readout sums (see Args::sums) from its 4 epilogue warps, in a fixed order: warp
// shuffles, then the warps in order (named barrier 1 holds only them).  Every epilogue thread
// calls it, also after a failed wait.
__device__ __forceinline__ void epi_store_sums(double s_lo, double s_hi, int sub, int lane, const Args &a) {
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) {
        s_lo += __shfl_down_sync(0xffffffffu, s_lo, o);
        s_hi += __shfl_down_sync(0xffffffffu, s_hi, o);
    }
    if (lane == 0) {
        red[2 * sub] = s_lo;
        red[2 * sub + 1] = s_hi;
    }
    asm volatile("bar.sync 1, 128;\n" ::: "memory");
    if (sub == 0 && lane == 0) {
        double lo = 0.0, hi = 0.0;
        for (int w = 0; w < 4; w++) {
            lo += red[2 * w];
            hi += red[2 * w + 1];
        }
        a.sums[1 + blockIdx.x] = lo;
        a.sums[1 + gridDim.x + blockIdx.x] = hi;
        if (blockIdx.x == 0) a.sums[0] = 2.0 * (double)gridDim.x;
    }
}

// ---------------------------------------------------------------------------------------
// Transposed form (6 targets on the low qubits, see launch_dense_tc).  When the targets are the lowest qubits,
// a group's amplitudes are contiguous but consecutive groups are 2^k amplitudes apart, and the
// group-major form would read and write 8-byte pieces at that stride.  This form computes
//     Y^T[2D x 128] = B[2D x 2D] * X^T,
// with B (the real form of U, hi and lo) as the MMA's A operand, held in tensor memory next to
// the two accumulators (U columns 256..511), and the tile's 128 groups as its B operand (N =
// 128), a ring of six shared-memory chunks of 32 K-columns.  Producers load each group's 16
// amplitudes of a chunk as 16-byte vectors (a warp reads 4 groups x 128 contiguous bytes).  With
// PAIRG (qubit 1 a target, qubit 0 free: a group bit) a 16-byte load is one amplitude of two
// sibling groups instead, and a warp reads 4 group pairs x 8 amplitudes.  The accumulator's TMEM
// lanes are output reals, so the epilogue's warp stores write 32 consecutive floats of one group;
// with PAIRG, lanes 2j and 2j+1 (re and im of output amplitude j) swap one value per pair of tile
// columns (sibling groups) and each writes one whole amplitude of one of the two: 256 contiguous
// bytes per warp store.  Roles, barriers and bounded waits as in the group-major kernels.
namespace tct {
constexpr int K = 6, D = 64, N = 128, KK = 128, NCH = KK / kCH;
constexpr int ABYTES = kM * kCH * 4;  // one chunk (hi or lo)
constexpr int NBUF = 6;
constexpr int NBAR = 2 * NBUF + 5;
constexpr int SMEM = NBUF * 2 * ABYTES + 8 * NBAR + 16 + 8 * D + 8 * kM;
constexpr int UCOL = 2 * N;  // tensor memory: two accumulators, then U hi and U lo
}  // namespace tct

template <bool PAIRG>
__global__ void __launch_bounds__(kThreadsWS, 1) dense_tc_tr_kernel(const Args a) {
    using namespace tct;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *Aring = sm;  // [NBUF][2][ABYTES]
    uint64_t *bars = reinterpret_cast<uint64_t *>(Aring + NBUF * 2 * ABYTES);
    uint64_t *full = bars;                 // [NBUF] producers -> MMA (count 512)
    uint64_t *empty = bars + NBUF;         // [NBUF] MMA completion -> producers (commit)
    uint64_t *accfull = bars + 2 * NBUF;   // [2] MMA completion -> epilogue (commit)
    uint64_t *accempty = accfull + 2;      // [2] epilogue -> MMA (count 128)
    uint64_t *drain = accfull + 4;         // MMA completion before tensor memory is freed
    unsigned *tslot = reinterpret_cast<unsigned *>(bars + NBAR);
    long long *toff = reinterpret_cast<long long *>(tslot + 4);  // D entries
    long long *goff = toff + D;  // kM entries: offset of group m of a tile from the tile's group 0

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        for (int c = tid; c < D; c += kThreadsWS) {
            long long o = 0;
            for (int b = 0; b < K; b++)
                if ((c >> b) & 1) o |= 1ll << a.targets[b];
            toff[c] = o;
        }
        // group index = tile * 128 + m, whose zero-inserted offset splits into the tile's part and
        // m's part (disjoint bits)
        for (int mm = tid; mm < kM; mm += kThreadsWS) goff[mm] = (long long)insert_zeros((unsigned long long)mm, a.fix, a.nfix);
        if (tid == 0) {
            for (int i = 0; i < NBUF; i++) {
                mbar_init(&full[i], kProducers);
                mbar_init(&empty[i], 1);
            }
            for (int i = 0; i < 2; i++) {
                mbar_init(&accfull[i], 1);
                mbar_init(&accempty[i], 128);
            }
            mbar_init(drain, 1);
        }
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                         "r"(512u)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    const unsigned tmem = *tslot;
    if (warp < kEpiWarp0) u_to_tmem(a.Bg, tmem, (unsigned)UCOL, warp, lane);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float2 *psi = reinterpret_cast<float2 *>(a.psi);
    const long long first = blockIdx.x, stride = gridDim.x;
    const long long ntl = first < a.ntiles ? (a.ntiles - first + stride - 1) / stride : 0;
    const long long total = ntl * NCH;
    bool failed = false;
    auto tile_base = [&](long long tile_i) -> unsigned long long {
        const unsigned long long gidx = (unsigned long long)(first + tile_i * stride) * kM;
        return insert_zeros(gidx, a.fix, a.nfix) | a.cmask;
    };

    if (warp < kEpiWarp0) {
        // ------------------------------------------------------------------ producers
        // Without PAIRG, thread (warp w, lane l): amplitude pair h = l / 4 (amplitudes 2h, 2h+1 of
        // the chunk's 16) of group rows 8w + (l mod 4) and 8w + 4 + (l mod 4).  A warp's vector
        // load reads 4 rows x 16 amplitudes, which are 4 whole 128-byte lines whether qubits 2 and
        // 3 are targets or free (one free: its two rows share a line).  The 16-byte shared-memory
        // stores alternate the rows between lanes of odd and even h, so a quarter-warp covers all
        // 8 row slots of a core matrix (no bank conflict).
        // With PAIRG, thread (w, l): amplitudes c = l / 4 and c + 8 of the chunk for the sibling
        // rows 8w + 2(l mod 4) and 8w + 2(l mod 4) + 1; a vector load reads 4 row pairs x 8
        // amplitudes.  Its 8-byte stores (one amplitude of one row) take the even or the odd row
        // first by bit 1 of c, so a half-warp covers the 16 distinct 8-byte slots of a 128-byte
        // core-matrix row group (no bank conflict).
        const int rw = lane & 3, h = lane >> 2;
        float2 r[kPrefetch][kAmpsPT];
        long long gb_tile = -1;
        unsigned long long gb_base = 0;
        const long long gA = PAIRG ? goff[8 * warp + 2 * rw] : goff[8 * warp + rw];
        const long long gB = PAIRG ? gA : goff[8 * warp + 4 + rw];
        auto load = [&](long long qq, float2(&rr)[kAmpsPT]) {
            if (qq < total) {
                if (qq / NCH != gb_tile) {
                    gb_tile = qq / NCH;
                    gb_base = tile_base(gb_tile);
                }
                const int c0 = (int)(qq % NCH) * 16;
                // without PAIRG qubit 0 is a target (amplitudes 2h, 2h+1 adjacent); with it the two
                // rows are siblings in qubit 0 (amplitude c of both adjacent)
                const long long ta0 = toff[c0 + (PAIRG ? h : 2 * h)];
                const long long ta1 = PAIRG ? toff[c0 + h + 8] : ta0;
                const float4 u0 = __ldcs(reinterpret_cast<const float4 *>(psi + gb_base + gA + ta0));
                const float4 u1 = __ldcs(reinterpret_cast<const float4 *>(psi + gb_base + gB + ta1));
                rr[0] = make_float2(u0.x, u0.y);
                rr[1] = make_float2(u0.z, u0.w);
                rr[2] = make_float2(u1.x, u1.y);
                rr[3] = make_float2(u1.z, u1.w);
            }
        };
#pragma unroll
        for (int p = 0; p < kPrefetch; p++) load(p, r[p]);
        for (long long q0 = 0; q0 < total && !failed; q0 += kPrefetch) {
#pragma unroll
            for (int p = 0; p < kPrefetch; p++) {
                const long long qq = q0 + p;
                if (qq >= total || failed) break;
                const int b = (int)(qq % NBUF);
                const long long use = qq / NBUF;
                if (use > 0 && !mbar_wait(&empty[b], (unsigned)((use - 1) & 1))) {
                    failed = true;
                    break;
                }
                unsigned char *ahi = Aring + b * 2 * ABYTES;
                unsigned char *alo = ahi + ABYTES;
                if constexpr (PAIRG) {
                    // r[0], r[1]: amplitude h of the even and odd row; r[2], r[3]: amplitude h + 8
#pragma unroll
                    for (int hv = 0; hv < 2; hv++) {
                        const int c = h + 8 * hv;  // amplitude of the chunk: K columns 2c, 2c + 1
#pragma unroll
                        for (int pi = 0; pi < 2; pi++) {
                            const int odd = pi ^ ((h >> 1) & 1);
                            const float2 x = odd ? r[p][2 * hv + 1] : r[p][2 * hv];
                            const unsigned off =
                                warp * 1024 + (c >> 1) * 128 + (2 * rw + odd) * 16 + (c & 1) * 8;
                            const unsigned h0 = to_tf32(x.x), h1 = to_tf32(x.y);
                            *reinterpret_cast<uint2 *>(ahi + off) = make_uint2(h0, h1);
                            *reinterpret_cast<uint2 *>(alo + off) =
                                make_uint2(to_tf32(x.x - __uint_as_float(h0)), to_tf32(x.y - __uint_as_float(h1)));
                        }
                    }
                } else {
#pragma unroll
                    for (int pi = 0; pi < 2; pi++) {  // row 8w + rw (pi = h mod 2) or 8w + 4 + rw
                        const int rowB = pi ^ (h & 1);
                        const float2 x0 = rowB ? r[p][2] : r[p][0], x1 = rowB ? r[p][3] : r[p][1];
                        const unsigned off = warp * 1024 + h * 128 + (4 * rowB + rw) * 16;
                        const unsigned h0 = to_tf32(x0.x), h1 = to_tf32(x0.y);
                        const unsigned h2 = to_tf32(x1.x), h3 = to_tf32(x1.y);
                        *reinterpret_cast<uint4 *>(ahi + off) = make_uint4(h0, h1, h2, h3);
                        *reinterpret_cast<uint4 *>(alo + off) =
                            make_uint4(to_tf32(x0.x - __uint_as_float(h0)), to_tf32(x0.y - __uint_as_float(h1)),
                                       to_tf32(x1.x - __uint_as_float(h2)), to_tf32(x1.y - __uint_as_float(h3)));
                    }
                }
                load(qq + kPrefetch, r[p]);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive(&full[b]);
            }
        }
    } else if (warp < kMmaWarp) {
        // ------------------------------------------------------------------ epilogue
        const int sub = warp - kEpiWarp0;          // TMEM lane subpartition
        const int m = sub * 32 + lane;             // output real
        const long long ta = toff[m >> 1];         // its amplitude
        const int odd = m & 1;                     // im lane: with PAIRG, writes the odd column of each pair
        float *psif = reinterpret_cast<float *>(a.psi);
        double s_lo = 0.0, s_hi = 0.0;  // readout sums of this thread's outputs
        const bool sums = a.sums != nullptr;
        for (long long t = 0; t < ntl && !failed; t++) {
            const int ab = (int)(t & 1);
            if (!mbar_wait(&accfull[ab], (unsigned)((t >> 1) & 1))) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const unsigned long long gb = tile_base(t);
            const unsigned acc = tmem + (unsigned)(ab * N) + ((unsigned)(sub * 32) << 16);
            float tsum = 0.f;  // the squares of the thread's outputs in this tile
#pragma unroll 1
            for (int col = 0; col < N; col += 16) {
                unsigned v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                      "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(acc + (unsigned)col));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                // v[i] = output real m of tile group col + i
                float q16 = 0.f;
                if constexpr (PAIRG) {
                    // columns i, i+1 are sibling groups (adjacent amplitudes): per pair the re lane
                    // gives its value of column i+1 for the im lane's value of column i, so the re
                    // lane holds amplitude m/2 of group col + i, the im lane that of group col + i + 1
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        const float y0 = __uint_as_float(v[i]), y1 = __uint_as_float(v[i + 1]);
                        const float got = __shfl_xor_sync(0xffffffffu, odd ? y0 : y1, 1);
                        __stcs(psi + gb + goff[col + i + odd] + ta, odd ? make_float2(got, y1) : make_float2(y0, got));
                        if (sums) q16 = __fmaf_rn(y1, y1, __fmaf_rn(y0, y0, q16));
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        const float y = __uint_as_float(v[i]);
                        __stcs(psif + 2 * (long long)(gb + goff[col + i] + ta) + (m & 1), y);
                        if (sums) q16 = __fmaf_rn(y, y, q16);
                    }
                }
                tsum += q16;
            }
            if (sums) tile_sum_into(tsum, (gb >> a.hi_bit) & 1ull, s_lo, s_hi);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(&accempty[ab]);
        }
        if (sums) epi_store_sums(s_lo, s_hi, sub, lane, a);
    } else if (lane == 0) {
        // ------------------------------------------------------------------ MMA issuer
        const unsigned aring_u32 = smem_u32(Aring);
        const unsigned u_hi = tmem + (unsigned)UCOL, u_lo = u_hi + (unsigned)KK;
        for (long long qq = 0; qq < total && !failed; qq++) {
            const int b = (int)(qq % NBUF);
            const int j = (int)(qq % NCH);
            const long long t = qq / NCH;
            const int ab = (int)(t & 1);
            if (j == 0 && t >= 2 && !mbar_wait(&accempty[ab], (unsigned)(((t >> 1) - 1) & 1))) {
                failed = true;
                break;
            }
            if (!mbar_wait(&full[b], (unsigned)((qq / NBUF) & 1))) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const unsigned acc = tmem + (unsigned)(ab * N);
            const unsigned x_hi = aring_u32 + b * 2 * ABYTES, x_lo = x_hi + ABYTES;
#pragma unroll
            for (int kk = 0; kk < kCH / 8; kk++) {
                const unsigned uc = (unsigned)(j * kCH + kk * 8);  // U columns of this K-step
                const uint64_t dXh = make_desc(x_hi + kk * 256, 128, 1024);  // 2 core matrices along K
                const uint64_t dXl = make_desc(x_lo + kk * 256, 128, 1024);
                // Y^T = U X^T in 3xTF32: Uhi Xhi + Ulo Xhi + Uhi Xlo
                mma_tf32_ta(acc, u_hi + uc, dXh, Cfg<K>::IDESC, (j == 0 && kk == 0) ? 0u : 1u);
                mma_tf32_ta(acc, u_lo + uc, dXh, Cfg<K>::IDESC, 1u);
                mma_tf32_ta(acc, u_hi + uc, dXl, Cfg<K>::IDESC, 1u);
            }
            commit_to(&empty[b]);
            if (j == NCH - 1) commit_to(&accfull[ab]);
        }
        commit_to(drain);  // tensor memory is released only after every MMA has completed
        if (!mbar_wait(drain, 0u)) failed = true;
    }
    if (failed) atomicOr(&g_device_error, 1u);
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512u) : "memory");
    }
}

// ---------------------------------------------------------------------------------------
// Real 7-target gates (a real U, e.g. the eigenvector matrix of a real symmetric system) on the
// lowest qubits, complex64.  For real U the complex product splits into two real ones,
// Y_re = U X_re and Y_im = U X_im, so one real GEMM does both:
//     Y^T[128 out amps x 128 rows] = U[128 x 128] * X^T,   row = (group, re or im),
// U (TF32 hi/lo) is the MMA's A operand, held in tensor memory next to the two accumulators, a
// chunk of 32 input amplitudes of 64 groups (128 rows) its B operand, in a six-deep shared-memory
// ring, and the accumulator's TMEM lanes are output amplitudes, so each epilogue warp stores 32
// consecutive complex amplitudes of one group.  Roles, barriers and bounded waits as in the
// other tensor-core kernels.
namespace tcr {
constexpr int D = 128;           // amplitudes per group (7 targets)
constexpr int KK = 128;          // reduction length: input amplitudes
constexpr int MG = 64;           // groups per tile (128 rows: re and im of each)
constexpr int NCH = KK / kCH;    // chunks of 32 input amplitudes
constexpr int BBYTES = D * KK * 4;
constexpr int ABYTES = 2 * MG * kCH * 4;
constexpr int NBUF = 6;         // chunk ring (U lives in tensor memory, so shared memory holds X only)
constexpr int NBAR = 2 * NBUF + 5;
constexpr int SMEM = NBUF * 2 * ABYTES + 8 * NBAR + 16 + 8 * D + 8 * MG;
constexpr int UCOL = 2 * 2 * MG;  // tensor memory: two accumulators, then U hi and U lo (512 columns)
constexpr unsigned IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)((2 * MG) >> 3) << 17) |
                           ((unsigned)(D >> 4) << 24);
}  // namespace tcr

__global__ void __launch_bounds__(kThreadsWS, 1) dense_tc_real7_kernel(const Args a) {
    using namespace tcr;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *Aring = sm;
    uint64_t *bars = reinterpret_cast<uint64_t *>(Aring + NBUF * 2 * ABYTES);
    uint64_t *full = bars, *empty = bars + NBUF, *accfull = bars + 2 * NBUF, *accempty = bars + 2 * NBUF + 2;
    uint64_t *drain = bars + 2 * NBUF + 4;
    unsigned *tslot = reinterpret_cast<unsigned *>(bars + NBAR);
    long long *toff = reinterpret_cast<long long *>(tslot + 4);  // D entries
    long long *goff = toff + D;                                  // MG entries

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        for (int c = tid; c < D; c += kThreadsWS) {
            long long o = 0;
            for (int b = 0; b < 7; b++)
                if ((c >> b) & 1) o |= 1ll << a.targets[b];
            toff[c] = o;
        }
        for (int g = tid; g < MG; g += kThreadsWS) goff[g] = (long long)insert_zeros((unsigned long long)g, a.fix, a.nfix);
        if (tid == 0) {
            for (int i = 0; i < NBUF; i++) {
                mbar_init(&full[i], kProducers);
                mbar_init(&empty[i], 1);
            }
            for (int i = 0; i < 2; i++) {
                mbar_init(&accfull[i], 1);
                mbar_init(&accempty[i], 128);
            }
            mbar_init(drain, 1);
        }
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                         "r"(512u)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    const unsigned tmem = *tslot;
    if (warp < kEpiWarp0) u_to_tmem(a.Bg, tmem, (unsigned)UCOL, warp, lane);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float2 *psi = reinterpret_cast<float2 *>(a.psi);
    const long long first = blockIdx.x, stride = gridDim.x;
    const long long ntl = first < a.ntiles ? (a.ntiles - first + stride - 1) / stride : 0;
    const long long total = ntl * NCH;
    bool failed = false;
    auto tile_base = [&](long long tile_i) -> unsigned long long {
        const unsigned long long gidx = (unsigned long long)(first + tile_i * stride) * MG;
        return insert_zeros(gidx, a.fix, a.nfix) | a.cmask;
    };

    if (warp < kEpiWarp0) {
        // ------------------------------------------------------------------ producers
        // thread t: group gi = 4 w + (l mod 4), amplitude pairs p and p + 8 (p = l / 4) of every
        // chunk.  A warp's vector load reads 4 groups x 128 contiguous bytes; a quarter-warp's
        // 8-byte stores (rows 2 gi, 2 gi + 1) fill 8 distinct bank slots.
        const int gi = 4 * warp + (lane & 3), p0 = lane >> 2;
        unsigned off[2][2];  // [pair][re, im]
#pragma unroll
        for (int pi = 0; pi < 2; pi++) {
            const int k = 2 * (p0 + 8 * pi);
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const int r = 2 * gi + c;
                off[pi][c] = (r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
            }
        }
        float4 rr[kPrefetch][2];
        long long gb_tile = -1;
        unsigned long long gb_row = 0;
        auto load = [&](long long qq, float4(&q4)[2]) {
            if (qq < total) {
                if (qq / NCH != gb_tile) {
                    gb_tile = qq / NCH;
                    gb_row = tile_base(gb_tile) + (unsigned long long)goff[gi];
                }
                const int c0 = (int)(qq % NCH) * kCH;
#pragma unroll
                for (int pi = 0; pi < 2; pi++)
                    q4[pi] = __ldcs(reinterpret_cast<const float4 *>(psi + gb_row + toff[c0 + 2 * (p0 + 8 * pi)]));
            }
        };
#pragma unroll
        for (int p = 0; p < kPrefetch; p++) load(p, rr[p]);
        for (long long q0 = 0; q0 < total && !failed; q0 += kPrefetch) {
#pragma unroll
            for (int p = 0; p < kPrefetch; p++) {
                const long long qq = q0 + p;
                if (qq >= total || failed) break;
                const int b = (int)(qq % NBUF);
                const long long use = qq / NBUF;
                if (use > 0 && !mbar_wait(&empty[b], (unsigned)((use - 1) & 1))) {
                    failed = true;
                    break;
                }
                unsigned char *ahi = Aring + b * 2 * ABYTES;
                unsigned char *alo = ahi + ABYTES;
#pragma unroll
                for (int pi = 0; pi < 2; pi++) {
                    const float4 x = rr[p][pi];  // (re, im) of amplitudes k and k + 1
                    const unsigned hr0 = to_tf32(x.x), hr1 = to_tf32(x.z);
                    const unsigned hi0 = to_tf32(x.y), hi1 = to_tf32(x.w);
                    *reinterpret_cast<uint2 *>(ahi + off[pi][0]) = make_uint2(hr0, hr1);
                    *reinterpret_cast<uint2 *>(ahi + off[pi][1]) = make_uint2(hi0, hi1);
                    *reinterpret_cast<uint2 *>(alo + off[pi][0]) =
                        make_uint2(to_tf32(x.x - __uint_as_float(hr0)), to_tf32(x.z - __uint_as_float(hr1)));
                    *reinterpret_cast<uint2 *>(alo + off[pi][1]) =
                        make_uint2(to_tf32(x.y - __uint_as_float(hi0)), to_tf32(x.w - __uint_as_float(hi1)));
                }
                load(qq + kPrefetch, rr[p]);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive(&full[b]);
            }
        }
    } else if (warp < kMmaWarp) {
        // ------------------------------------------------------------------ epilogue
        const int sub = warp - kEpiWarp0;
        const int n = sub * 32 + lane;  // output amplitude == TMEM lane
        const long long ta = toff[n];
        double s_lo = 0.0, s_hi = 0.0;  // readout sums of this thread's outputs
        const bool sums = a.sums != nullptr;
        for (long long t = 0; t < ntl && !failed; t++) {
            const int ab = (int)(t & 1);
            if (!mbar_wait(&accfull[ab], (unsigned)((t >> 1) & 1))) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const unsigned long long tb = tile_base(t);
            const unsigned acc = tmem + (unsigned)(ab * 2 * MG) + ((unsigned)(sub * 32) << 16);
            float tsum = 0.f;  // the squared magnitudes of the thread's outputs in this tile
#pragma unroll 1
            for (int col = 0; col < 2 * MG; col += 16) {  // 16 columns = re, im of 8 groups
                unsigned v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                      "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(acc + (unsigned)col));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                float q8 = 0.f;
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const unsigned long long idx = tb + goff[col / 2 + i] + ta;
                    const float yr = __uint_as_float(v[2 * i]), yi = __uint_as_float(v[2 * i + 1]);
                    __stcs(psi + idx, make_float2(yr, yi));
                    if (sums) q8 = __fmaf_rn(yi, yi, __fmaf_rn(yr, yr, q8));
                }
                tsum += q8;
            }
            if (sums) tile_sum_into(tsum, (tb >> a.hi_bit) & 1ull, s_lo, s_hi);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(&accempty[ab]);
        }
        if (sums) epi_store_sums(s_lo, s_hi, sub, lane, a);
    } else if (lane == 0) {
        // ------------------------------------------------------------------ MMA issuer
        const unsigned aring_u32 = smem_u32(Aring);
        const unsigned u_hi = tmem + (unsigned)UCOL, u_lo = u_hi + (unsigned)KK;
        for (long long qq = 0; qq < total && !failed; qq++) {
            const int b = (int)(qq % NBUF);
            const int j = (int)(qq % NCH);
            const long long t = qq / NCH;
            const int ab = (int)(t & 1);
            if (j == 0 && t >= 2 && !mbar_wait(&accempty[ab], (unsigned)(((t >> 1) - 1) & 1))) {
                failed = true;
                break;
            }
            if (!mbar_wait(&full[b], (unsigned)((qq / NBUF) & 1))) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const unsigned acc = tmem + (unsigned)(ab * 2 * MG);
            const unsigned x_hi = aring_u32 + b * 2 * ABYTES, x_lo = x_hi + ABYTES;
#pragma unroll
            for (int kk = 0; kk < kCH / 8; kk++) {
                const unsigned uc = (unsigned)(j * kCH + kk * 8);  // U columns of this K-step
                const uint64_t dXh = make_desc(x_hi + kk * 256, 128, 1024);
                const uint64_t dXl = make_desc(x_lo + kk * 256, 128, 1024);
                mma_tf32_ta(acc, u_hi + uc, dXh, IDESC, (j == 0 && kk == 0) ? 0u : 1u);
                mma_tf32_ta(acc, u_lo + uc, dXh, IDESC, 1u);
                mma_tf32_ta(acc, u_hi + uc, dXl, IDESC, 1u);
            }
            commit_to(&empty[b]);
            if (j == NCH - 1) commit_to(&accfull[ab]);
        }
        commit_to(drain);  // tensor memory is released only after every MMA has completed
        if (!mbar_wait(drain, 0u)) failed = true;
    }
    if (failed) atomicOr(&g_device_error, 1u);
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512u) : "memory");
    }
}

}  // namespace tc

// Host-side split of the real form of U into TF32 hi/lo in the canonical shared-memory
// layout (row n = output real index, column k = input real index).
static unsigned tf32_rne_bits(float x) {
    unsigned u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return u;  // inf/nan: keep
    u += 0xFFFu + ((u >> 13) & 1u);
    return u & 0xFFFFE000u;
}

size_t dense_tc_blob_bytes(int k) {
    const size_t D = (size_t)1 << k;
    return 2 * (2 * D) * (2 * D) * 4;
}

bool dense_tc_supported(int k) { return k >= 3 && k <= 6; }

bool dense_tc_real7_applies(const Op &op) {
    return op.real_u && op.targets.size() == 7 && op.targets[0] == 0 && op.targets[1] == 1;
}

size_t dense_tc_real7_blob_bytes() { return 2 * (size_t)tc::tcr::BBYTES; }

// Real U (rows = output amplitudes, columns = input amplitudes) split into TF32 hi/lo in the
// canonical K-major layout of the real 7-target kernel.
void dense_tc_pack_real7(const std::vector<cd> &U, unsigned char *out) {
    constexpr int D = tc::tcr::D, KK = tc::tcr::KK;
    float *hi = reinterpret_cast<float *>(out);
    float *lo = hi + (size_t)D * KK;
    for (int n = 0; n < D; n++)
        for (int k = 0; k < KK; k++) {
            const float f = (float)U[(size_t)n * D + k].real();
            const unsigned hb = tf32_rne_bits(f);
            float hf;
            std::memcpy(&hf, &hb, 4);
            const unsigned lb = tf32_rne_bits(f - hf);
            float lf;
            std::memcpy(&lf, &lb, 4);
            const size_t idx = ((size_t)(n >> 3) * (KK * 32) + (size_t)(k >> 2) * 128 + (n & 7) * 16 + (k & 3) * 4) / 4;
            hi[idx] = hf;
            lo[idx] = lf;
        }
}

// The readout-sum epilogues classify a whole tile (2^tile_bits groups) by bit hi_bit of its base:
// valid when that bit is above the state, or a group bit with at least tile_bits group bits below.
static bool tile_classifies(int n, const std::vector<int> &targets, int hi_bit, int tile_bits) {
    if (hi_bit >= n) return true;
    int below = 0;
    for (int q : targets)
        if (q == hi_bit) return false;
    for (int q = 0; q < hi_bit; q++)
        if (std::find(targets.begin(), targets.end(), q) == targets.end()) below++;
    return below >= tile_bits;
}

bool launch_dense_tc_real7(void *state, int n, const std::vector<int> &targets, const std::vector<int> &controls,
                           const void *Bdev, int sms, cudaStream_t st, double *sums, int hi_bit, bool *sums_written) {
    const int free_bits = n - 7 - (int)controls.size();
    if (free_bits < 6) return false;  // fewer than 64 groups
    tc::Args a;
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    a.Bg = static_cast<const float *>(Bdev);
    a.ntiles = 1ll << (free_bits - 6);
    std::vector<int> fix(targets);
    for (int q : controls) {
        fix.push_back(q);
        a.cmask |= 1ull << q;
    }
    std::sort(fix.begin(), fix.end());
    if ((int)fix.size() > tc::kMaxFix) return false;
    a.nfix = (int)fix.size();
    for (int i = 0; i < a.nfix; i++) a.fix[i] = fix[i];
    for (int b = 0; b < 7; b++) a.targets[b] = targets[b];
    QSIM_REQUIRE(sums == nullptr || controls.empty(), "readout sums need every amplitude written");
    if (sums && !tile_classifies(n, targets, hi_bit, 6)) sums = nullptr;
    if (sums_written) *sums_written = sums != nullptr;
    a.sums = sums;
    a.hi_bit = hi_bit;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc::dense_tc_real7_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tc::tcr::SMEM);
        if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("dense_tc_real7_kernel attribute: ") + cudaGetErrorString(e));
        attr = true;
    }
    const long long grid = std::min<long long>(a.ntiles, (long long)sms);  // one CTA per SM (TMEM, smem)
    tc::dense_tc_real7_kernel<<<(int)grid, tc::kThreadsWS, tc::tcr::SMEM, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("dense_tc_real7_kernel: ") + cudaGetErrorString(e));
    note_launches(1, QSIM_KERNEL_DENSE_TC);
    return true;
}

void dense_tc_pack(int k, const std::vector<cd> &U, unsigned char *out) {
    const int D = 1 << k, N = 2 * D, KK = 2 * D;
    float *hi = reinterpret_cast<float *>(out);
    float *lo = hi + (size_t)N * KK;
    for (int n = 0; n < N; n++)
        for (int kc = 0; kc < KK; kc++) {
            const int r = n >> 1, pr = n & 1, c = kc >> 1, pc = kc & 1;
            const cd u = U[(size_t)r * D + c];
            double v;
            if (pr == 0) v = pc == 0 ? u.real() : -u.imag();
            else v = pc == 0 ? u.imag() : u.real();
            const float f = (float)v;
            const unsigned hb = tf32_rne_bits(f);
            float hf;
            std::memcpy(&hf, &hb, 4);
            const unsigned lb = tf32_rne_bits(f - hf);
            float lf;
            std::memcpy(&lf, &lb, 4);
            const size_t idx = ((size_t)(n >> 3) * (KK * 32) + (size_t)(kc >> 2) * 128 + (n & 7) * 16 + (kc & 3) * 4) / 4;
            hi[idx] = hf;
            lo[idx] = lf;
        }
}

template <int K>
static void launch_tc_gm(const tc::Args &a, int sms, cudaStream_t st) {
    using C = tc::GmCfg<K>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc::dense_tc_gm_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("dense_tc_gm_kernel attribute: ") + cudaGetErrorString(e));
        attr = true;
    }
    // one CTA per SM: it holds all 512 tensor-memory columns
    const long long grid = std::min<long long>(a.ntiles, (long long)sms);
    tc::dense_tc_gm_kernel<K><<<(int)grid, tc::kThreadsWS, C::SMEM, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("dense_tc_gm_kernel: ") + cudaGetErrorString(e));
    note_launches(1, QSIM_KERNEL_DENSE_TC);
}

template <bool PAIRG>
static void launch_tc_tr(const tc::Args &a, int sms, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc::dense_tc_tr_kernel<PAIRG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tc::tct::SMEM);
        if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("dense_tc_tr_kernel attribute: ") + cudaGetErrorString(e));
        attr = true;
    }
    // one CTA per SM: it holds all 512 tensor-memory columns
    const long long grid = std::min<long long>(a.ntiles, (long long)sms);
    tc::dense_tc_tr_kernel<PAIRG><<<(int)grid, tc::kThreadsWS, tc::tct::SMEM, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("dense_tc_tr_kernel: ") + cudaGetErrorString(e));
    note_launches(1, QSIM_KERNEL_DENSE_TC);
}

// Returns false if this gate shape is not handled by the tensor-core kernel.
bool launch_dense_tc(void *state, int n, const std::vector<int> &targets, const std::vector<int> &controls,
                     const void *Bdev, int sms, cudaStream_t st, double *sums, int hi_bit, bool *sums_written) {
    const int K = (int)targets.size();
    if (!dense_tc_supported(K)) return false;
    const int free_bits = n - K - (int)controls.size();
    if (free_bits < 7) return false;  // fewer than 128 groups
    tc::Args a;
    std::memset(&a, 0, sizeof(a));
    a.psi = state;
    a.Bg = static_cast<const float *>(Bdev);
    a.ntiles = 1ll << (free_bits - 7);
    std::vector<int> fix(targets);
    for (int q : controls) {
        fix.push_back(q);
        a.cmask |= 1ull << q;
    }
    std::sort(fix.begin(), fix.end());
    if ((int)fix.size() > tc::kMaxFix) return false;
    a.nfix = (int)fix.size();
    for (int i = 0; i < a.nfix; i++) a.fix[i] = fix[i];
    for (int b = 0; b < K; b++) a.targets[b] = targets[b];
    // targets ascending (canonical order).  6 targets with qubit 0 (its amplitude pairs are the
    // transposed form's 16-byte loads): the transposed form when qubit 1 is a target too, or when
    // at most one of qubits 0..3 is free, where the group-major form's warp loads touch 16-32
    // lines.  6 targets with qubit 1 and a free qubit 0 (sibling groups in each 16-byte load):
    // the transposed form's PAIRG variant when qubit 0 is the only free one of qubits 0..3.  The
    // transposed form is the only one that also writes readout sums
    int free_low = 0;
    for (int q = 0; q < 4 && q < n; q++)
        free_low += std::find(fix.begin(), fix.end(), q) == fix.end();
    const bool q0_free = std::find(fix.begin(), fix.end(), 0) == fix.end();
    const bool trp = K == 6 && targets[0] == 1 && q0_free && free_low == 1;
    const bool tr = trp || (K == 6 && targets[0] == 0 && (targets[1] == 1 || free_low <= 1));
    QSIM_REQUIRE(sums == nullptr || controls.empty(), "readout sums need every amplitude written");
    if (sums && (!tr || !tile_classifies(n, targets, hi_bit, 7))) sums = nullptr;
    if (sums_written) *sums_written = sums != nullptr;
    a.sums = sums;
    a.hi_bit = hi_bit;
    switch (K) {
        case 3: launch_tc_gm<3>(a, sms, st); break;
        case 4: launch_tc_gm<4>(a, sms, st); break;
        case 5: launch_tc_gm<5>(a, sms, st); break;
        case 6:
            if (trp) launch_tc_tr<true>(a, sms, st);
            else if (tr) launch_tc_tr<false>(a, sms, st);
            else launch_tc_gm<6>(a, sms, st);
            break;
        default: return false;
    }
    return true;
}

unsigned read_device_error() {
    unsigned v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_device_error, sizeof(v));
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("reading device status: ") + cudaGetErrorString(e));
    return v | dft_tma_read_error() | dft_merge_read_error();  // bit 0 either way: a bounded wait ran out
}

void clear_device_error() {
    const unsigned z = 0;
    cudaError_t e = cudaMemcpyToSymbol(g_device_error, &z, sizeof(z));
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("clearing device status: ") + cudaGetErrorString(e));
    dft_tma_clear_error();
    dft_merge_clear_error();
}

}  // namespace qsim

extern "C" int qsim_device_status(unsigned *flags, int clear) {
    using namespace qsim;
    return guarded([&] {
        QSIM_REQUIRE(flags != nullptr, "NULL argument");
        *flags = read_device_error();
        if (clear) clear_device_error();
    });
}
