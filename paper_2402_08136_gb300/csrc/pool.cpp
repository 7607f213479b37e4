// Serving pool: HHL solves of different sizes admitted as they arrive, state vectors resident in
// one device arena with memory-budget admission, continuous batching across CUDA streams.
//
// Threads
//   builders  (n_builders): hhl_build + qsim_fuse of submitted requests on the host;
//   scheduler (1)         : admits built requests while the arena has room for their state
//                           (S * 2^n bytes, S = 8 or 16) and a stream slot is free, launches
//                           them, and retires finished work by polling CUDA events.
// Small requests (at most `small_n` qubits, every fused operation supported by the batched
// executor) that are ready together are launched as one
// persistent batched kernel (one CTA per circuit, state in shared memory); larger requests run
// alone on a stream with the full-GPU kernels (tensor cores for complex64 dense gates).  Work
// keeps arriving while earlier launches run: every free stream slot takes the next admitted
// group, so launches overlap on the device.
//
// The hot path allocates nothing from CUDA: states, batch tables, gate matrices and readout
// scratch are carved out of the arena (first fit, coalescing), copies to the host land in
// pinned per-slot buffers allocated when the pool is created, and table uploads are
// cudaMemcpyAsync from pageable memory (returns once staged).  cudaFree, which would
// synchronize the device, is only called when the pool is destroyed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>

#include "common.h"

namespace qsim {
namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, cap) with coalescing free list; 256-byte granularity.
class Arena {
  public:
    explicit Arena(size_t cap) : cap_(cap) { free_[0] = cap; }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t cap() const { return cap_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    size_t cap_, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

struct Block {
    size_t off = 0, bytes = 0;
};

struct PoolReq {
    uint64_t id = 0;
    std::vector<double> A, b;
    int N = 0, n_clock = 0, dtype = QSIM_C64, flags = 0;
    double t = 0, C = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = QSIM_EBUSY;  // EBUSY while pending
    std::string err;
    hhl_circuit *h = nullptr;
    qsim_circuit *fused = nullptr;
    int n = 0;
    bool small = false;  // runs in a batched launch
    std::vector<Block> blocks;  // arena blocks held while running
    void *state = nullptr;
    std::vector<double> x;
    hhl_readout_stats stats{};
    ~PoolReq() {
        if (fused) qsim_circuit_free(fused);
        if (h) hhl_circuit_free(h);
    }
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;  // device time of the launch (launch log)
    double *pinned = nullptr;  // results / readout landing zone
    size_t pinned_doubles = 0;
    bool busy = false;
    std::vector<PoolReq *> reqs;
    qsim_batch *batch = nullptr;
    std::vector<Block> blocks;  // tables / matrices / scratch of this launch
    bool large = false;
};

}  // namespace
}  // namespace qsim

struct qsim_pool {
    int device = 0;
    void *arena_base = nullptr;
    std::unique_ptr<qsim::Arena> arena;
    std::vector<qsim::Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<qsim::PoolReq *> submitted, built;
    std::deque<uint64_t> completed;  // tickets finished (ok or failed), not yet handed out
    std::unordered_map<uint64_t, std::unique_ptr<qsim::PoolReq>> reqs;
    std::vector<std::thread> builders;
    std::thread scheduler;
    bool stop = false;
    uint64_t next_id = 1;
    int small_n = 16, max_batch = 512, k_small = 2, k_large_c64 = 4, k_large_c128 = 2;
    int n_building = 0, n_running = 0, n_done = 0, n_failed = 0, n_ready = 0;
    long long batches = 0, singles = 0;
    cudaEvent_t ev_ref = nullptr;             // device time zero of the launch log
    std::deque<qsim_pool_launch> launch_log;  // the most recent retired launches (guarded by mu)
};

namespace qsim {
namespace {

size_t amp_bytes(int dtype) { return dtype == QSIM_C128 ? 16 : 8; }

void fail(qsim_pool *p, PoolReq *r, int code, const std::string &msg) {
    r->status = code;
    r->err = msg;
    r->t_done = now_s();
    p->n_failed++;
    p->completed.push_back(r->id);
}

void builder_loop(qsim_pool *p) {
    cudaSetDevice(p->device);
    for (;;) {
        PoolReq *r;
        {
            std::unique_lock<std::mutex> lk(p->mu);
            p->cv_work.wait(lk, [&] { return p->stop || !p->submitted.empty(); });
            if (p->stop) return;
            r = p->submitted.front();
            p->submitted.pop_front();
            p->n_building++;
        }
        // QFTs and clock Hadamard layers as passes: both executors run them, and they replace
        // O(m^2) gates by O(m / 10) state passes
        int rc = hhl_build_ex(r->A.data(), r->b.data(), r->N, r->n_clock, r->t, r->C,
                              r->flags | QSIM_HHL_FFT_QFT, &r->h);
        std::string msg = rc == QSIM_OK ? "" : qsim_last_error();
        if (rc == QSIM_OK) {
            r->n = r->h->n;
            const int k = r->n <= p->small_n ? p->k_small
                                             : (r->dtype == QSIM_C64 ? p->k_large_c64 : p->k_large_c128);
            rc = qsim_fuse(&r->h->circ, k, &r->fused);
            if (rc != QSIM_OK) msg = qsim_last_error();
            else r->small = r->n <= p->small_n && batch_supported(r->fused);
        }
        std::lock_guard<std::mutex> lk(p->mu);
        p->n_building--;
        if (rc != QSIM_OK) {
            fail(p, r, rc, msg);
            p->cv_done.notify_all();
        } else {
            p->built.push_back(r);
            p->cv_work.notify_all();
        }
    }
}

void release_blocks(qsim_pool *p, std::vector<Block> &bl) {
    for (const Block &b : bl) p->arena->release(b.off, b.bytes);
    bl.clear();
}

bool take(qsim_pool *p, size_t bytes, std::vector<Block> &into) {
    size_t off;
    if (!p->arena->alloc(bytes, &off)) return false;
    into.push_back({off, bytes});
    return true;
}

void *addr(qsim_pool *p, const Block &b) { return static_cast<unsigned char *>(p->arena_base) + b.off; }

// Results of a finished slot into its requests (scheduler thread, no lock: the requests are
// not visible to pollers until their status is published), memory back to the arena.
void collect(qsim_pool *p, Slot &s, cudaError_t status) {
    for (size_t i = 0; i < s.reqs.size(); i++) {
        PoolReq *r = s.reqs[i];
        if (status == cudaSuccess) {
            r->x.assign(2 * (size_t)r->N, 0.0);
            if (s.batch) {
                batch_host_result(s.batch, (int)i, r->x.data(), &r->stats);
            } else {
                const double *sums = s.pinned;
                const unsigned char *slice = reinterpret_cast<const unsigned char *>(s.pinned + 4);
                const double P = sums[1], P0 = sums[2];
                const double inv = P0 > 0 ? 1.0 / std::sqrt(P0) : 0.0;
                const double norm_x = std::sqrt(P) / r->h->C;
                for (int j = 0; j < r->N; j++) {
                    double re, im;
                    const int jj = r->h->x_off + j;
                    if (r->dtype == QSIM_C128) {
                        re = reinterpret_cast<const double *>(slice)[2 * jj];
                        im = reinterpret_cast<const double *>(slice)[2 * jj + 1];
                    } else {
                        re = reinterpret_cast<const float *>(slice)[2 * jj];
                        im = reinterpret_cast<const float *>(slice)[2 * jj + 1];
                    }
                    r->x[2 * j] = re * inv * norm_x * r->h->norm_b;
                    r->x[2 * j + 1] = im * inv * norm_x * r->h->norm_b;
                }
                r->stats.p_success = P;
                r->stats.p_clock0 = P0;
                r->stats.leakage = P - P0;
                r->stats.norm2 = sums[0];
                r->stats.norm_x = norm_x;
                r->stats.norm_b = r->h->norm_b;
            }
        }
        release_blocks(p, r->blocks);
    }
    if (s.batch) {
        qsim_batch_free(s.batch);  // external tables: no CUDA call
        s.batch = nullptr;
    }
    release_blocks(p, s.blocks);
}

// Publish finished requests (caller holds mu).
void publish(qsim_pool *p, std::vector<PoolReq *> &rs, cudaError_t status) {
    const double t = now_s();
    for (PoolReq *r : rs) {
        p->n_running--;
        if (status != cudaSuccess) {
            fail(p, r, QSIM_ECUDA, std::string("device work failed: ") + cudaGetErrorString(status));
        } else {
            r->status = QSIM_OK;
            r->t_done = t;
            p->n_done++;
            p->completed.push_back(r->id);
        }
    }
}

// Launch a group of small requests as one batch on slot s (scheduler thread, no lock).
void launch_small(qsim_pool *p, Slot &s, std::vector<PoolReq *> &group) {
    std::vector<const qsim_circuit *> cs;
    std::vector<const hhl_circuit *> hs;
    std::vector<void *> states;
    for (PoolReq *r : group) {
        cs.push_back(r->fused);
        hs.push_back(r->h);
        states.push_back(r->state);
    }
    std::unique_ptr<BatchImage, void (*)(BatchImage *)> im(batch_plan(cs, hs, states.data(), group[0]->dtype),
                                                          batch_plan_free);
    QSIM_REQUIRE(batch_plan_result_doubles(im.get()) <= s.pinned_doubles, "batch results exceed the slot buffer");
    Block tb;
    if (!p->arena->alloc(batch_plan_device_bytes(im.get()), &tb.off)) throw Error(QSIM_EBUSY, "arena full");
    tb.bytes = batch_plan_device_bytes(im.get());
    s.blocks.push_back(tb);
    cudaError_t e = cudaEventRecord(s.ev_start, s.st);
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, cudaGetErrorString(e));
    s.batch = batch_instantiate(im.get(), addr(p, tb), s.pinned, s.st);
    batch_launch(s.batch, s.st);
    batch_enqueue_results(s.batch, s.st);
    e = cudaEventRecord(s.ev_end, s.st);
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, cudaGetErrorString(e));
    e = cudaEventRecord(s.ev, s.st);
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, cudaGetErrorString(e));
    s.reqs = group;
    s.busy = true;
    s.large = false;
}

// Launch one large request on slot s (full-GPU kernels; scheduler thread, no lock).
void launch_large(qsim_pool *p, Slot &s, PoolReq *r) {
    const int dtype = r->dtype;
    std::vector<unsigned char> blob = pack_device_blob(r->fused, dtype);
    Block mb, sb;
    if (!p->arena->alloc(blob.size(), &mb.off)) throw Error(QSIM_EBUSY, "arena full");
    mb.bytes = blob.size();
    s.blocks.push_back(mb);
    const size_t scr = readout_scratch_doubles(r->n) * sizeof(double);
    if (!p->arena->alloc(scr, &sb.off)) throw Error(QSIM_EBUSY, "arena full");
    sb.bytes = scr;
    s.blocks.push_back(sb);
    cudaError_t e = cudaEventRecord(s.ev_start, s.st);
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, cudaGetErrorString(e));
    e = cudaMemcpyAsync(addr(p, mb), blob.data(), blob.size(), cudaMemcpyHostToDevice, s.st);
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, std::string("matrix upload: ") + cudaGetErrorString(e));
    attach_external_blob(r->fused, dtype, addr(p, mb), blob.size());
    // only the data register is populated after the preparation (clock and ancilla |0>): the
    // executor widens the live part as the circuit fills it (as hhl_run does)
    launch_prepare_state(r->state, r->n, dtype, r->h->b_pad.data(), r->h->nb, s.st, r->h->nb);
    // the readout partial sums come from the circuit's last kernel when it can write them
    double *scratch = static_cast<double *>(addr(p, sb));
    apply_ops(r->state, r->n, dtype, r->fused, s.st, r->h->nb, scratch);
    readout_launch_async(r->state, dtype, r->n, r->h->nb, s.st, scratch, s.pinned, s.pinned + 4, true);
    e = cudaEventRecord(s.ev_end, s.st);
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, cudaGetErrorString(e));
    e = cudaEventRecord(s.ev, s.st);
    if (e != cudaSuccess) throw Error(QSIM_ECUDA, cudaGetErrorString(e));
    s.reqs = {r};
    s.busy = true;
    s.large = true;
}

// The scheduler owns the arena, the slots and its `ready` queue; the pool mutex only guards
// what other threads see (submitted / built queues, ticket map, completion queue, counters),
// so building plans, packing matrices and launching never block submitters or builders.
void scheduler_loop(qsim_pool *p) {
    cudaSetDevice(p->device);
    std::deque<PoolReq *> ready;
    for (;;) {
        bool progress = false;
        // 1. retire finished launches
        for (Slot &s : p->slots) {
            if (!s.busy) continue;
            cudaError_t q = cudaEventQuery(s.ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) cudaGetLastError();
            qsim_pool_launch rec{};
            rec.slot = (int)(&s - p->slots.data());
            rec.batched = s.large ? 0 : 1;
            rec.n_requests = (int)s.reqs.size();
            rec.first_ticket = s.reqs.empty() ? 0 : s.reqs.front()->id;
            rec.last_ticket = s.reqs.empty() ? 0 : s.reqs.back()->id;
            float t0 = 0.f, t1 = 0.f;
            if (q == cudaSuccess && cudaEventElapsedTime(&t0, p->ev_ref, s.ev_start) == cudaSuccess &&
                cudaEventElapsedTime(&t1, p->ev_ref, s.ev_end) == cudaSuccess) {
                rec.t_start = 1e-3 * t0;
                rec.t_end = 1e-3 * t1;
            } else {
                cudaGetLastError();
                rec.t_start = rec.t_end = -1.0;
            }
            collect(p, s, q);
            {
                std::lock_guard<std::mutex> lk(p->mu);
                publish(p, s.reqs, q);
                p->launch_log.push_back(rec);
                if (p->launch_log.size() > 4096) p->launch_log.pop_front();
            }
            p->cv_done.notify_all();
            s.reqs.clear();
            s.busy = false;
            progress = true;
        }
        // 2. take newly built requests
        bool stopping;
        {
            std::lock_guard<std::mutex> lk(p->mu);
            while (!p->built.empty()) {
                ready.push_back(p->built.front());
                p->built.pop_front();
            }
            p->n_ready = (int)ready.size();
            stopping = p->stop && p->submitted.empty() && p->n_building == 0;
        }
        if (stopping && ready.empty()) {
            bool any = false;
            for (Slot &s : p->slots) any |= s.busy;
            if (!any) return;
        }
        // 3. admit: states first (memory budget), then launches on free slots
        std::vector<std::pair<PoolReq *, std::pair<int, std::string>>> failed;
        for (Slot &s : p->slots) {
            if (s.busy || ready.empty()) continue;
            std::vector<PoolReq *> group;
            PoolReq *large = nullptr;
            for (auto it = ready.begin(); it != ready.end();) {
                PoolReq *r = *it;
                const size_t need = amp_bytes(r->dtype) << r->n;
                if (need > p->arena->cap()) {
                    failed.push_back({r, {QSIM_ENOMEM, "state larger than the pool"}});
                    it = ready.erase(it);
                    continue;
                }
                const bool is_small = r->small;
                if (!is_small && (!group.empty() || large)) {
                    ++it;
                    continue;
                }
                if (is_small && (large || (!group.empty() && r->dtype != group[0]->dtype) ||
                                 (int)group.size() >= p->max_batch)) {
                    ++it;
                    continue;
                }
                if (!take(p, need, r->blocks)) break;  // memory budget: wait for retirements
                r->state = addr(p, r->blocks.back());
                r->t_admit = now_s();
                it = ready.erase(it);
                if (is_small) group.push_back(r);
                else large = r;
                if (large) break;
            }
            if (!large && group.empty()) continue;
            {
                std::lock_guard<std::mutex> lk(p->mu);
                p->n_running += large ? 1 : (int)group.size();
                if (large) p->singles++;
                else p->batches++;
            }
            try {
                if (large) launch_large(p, s, large);
                else launch_small(p, s, group);
                progress = true;
            } catch (const Error &e) {
                // back to the queue if the arena was too full for the tables, fail otherwise.
                // Kernels or copies may already be queued on the slot's stream (preparation, an
                // upload, part of the circuit): its memory goes back to the arena only once they
                // are finished, or the next request on another stream could be handed blocks that
                // are still being read and written.
                if (cudaStreamSynchronize(s.st) != cudaSuccess) cudaGetLastError();
                std::vector<PoolReq *> rs = large ? std::vector<PoolReq *>{large} : group;
                release_blocks(p, s.blocks);
                if (s.batch) {
                    qsim_batch_free(s.batch);
                    s.batch = nullptr;
                }
                {
                    std::lock_guard<std::mutex> lk(p->mu);
                    p->n_running -= (int)rs.size();
                    if (large) p->singles--;
                    else p->batches--;
                }
                for (PoolReq *r : rs) {
                    release_blocks(p, r->blocks);
                    if (e.code == QSIM_EBUSY) ready.push_front(r);
                    else failed.push_back({r, {e.code, e.what()}});
                }
                s.busy = false;
                s.reqs.clear();
                if (e.code == QSIM_EBUSY) break;
            }
        }
        if (!failed.empty()) {
            {
                std::lock_guard<std::mutex> lk(p->mu);
                for (auto &f : failed) fail(p, f.first, f.second.first, f.second.second);
            }
            p->cv_done.notify_all();
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(p->mu);
            p->cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

}  // namespace
}  // namespace qsim

using namespace qsim;

extern "C" {

int qsim_pool_create(size_t bytes, int n_builders, int n_streams, qsim_pool **out) {
    return guarded([&] {
        QSIM_REQUIRE(out != nullptr && bytes >= (1u << 20), "pool needs at least 1 MiB");
        if (n_builders <= 0) n_builders = std::max(1u, std::thread::hardware_concurrency() / 2);
        if (n_streams <= 0) n_streams = 8;
        std::unique_ptr<qsim_pool> p(new qsim_pool());
        if (cudaGetDevice(&p->device) != cudaSuccess) throw Error(QSIM_ECUDA, "no CUDA device");
        cudaError_t e = cudaMalloc(&p->arena_base, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error(QSIM_ENOMEM, std::string("pool arena: ") + cudaGetErrorString(e));
        }
        p->arena.reset(new Arena(bytes));
        p->slots.resize(n_streams);
        const size_t pin = 4 + 2 * ((size_t)1 << 12);  // large readout: sums + 2^12-amplitude slice
        const size_t pin_batch = (size_t)p->max_batch * (4 + 2 * 128);
        for (Slot &s : p->slots) {
            s.pinned_doubles = std::max(pin, pin_batch);
            if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreate(&s.ev_start) != cudaSuccess || cudaEventCreate(&s.ev_end) != cudaSuccess ||
                cudaMallocHost(&s.pinned, s.pinned_doubles * sizeof(double)) != cudaSuccess)
                throw Error(QSIM_ECUDA, "creating pool streams / pinned buffers");
        }
        if (cudaEventCreate(&p->ev_ref) != cudaSuccess || cudaEventRecord(p->ev_ref, p->slots[0].st) != cudaSuccess ||
            cudaEventSynchronize(p->ev_ref) != cudaSuccess)
            throw Error(QSIM_ECUDA, "creating the pool's reference event");
        qsim_pool *raw = p.get();
        for (int i = 0; i < n_builders; i++) raw->builders.emplace_back(builder_loop, raw);
        raw->scheduler = std::thread(scheduler_loop, raw);
        *out = p.release();
    });
}

int qsim_submit(qsim_pool *p, const hhl_request *req, uint64_t *ticket) {
    return guarded([&] {
        QSIM_REQUIRE(p != nullptr && req != nullptr && ticket != nullptr, "NULL argument");
        QSIM_REQUIRE(req->A != nullptr && req->b != nullptr && req->N >= 1 && req->N <= 4096, "bad request shape");
        QSIM_REQUIRE(req->dtype == QSIM_C64 || req->dtype == QSIM_C128, "dtype must be QSIM_C64 or QSIM_C128");
        std::unique_ptr<PoolReq> r(new PoolReq());
        r->A.assign(req->A, req->A + 2 * (size_t)req->N * req->N);
        r->b.assign(req->b, req->b + 2 * (size_t)req->N);
        r->N = req->N;
        r->n_clock = req->n_clock;
        r->t = req->t;
        r->C = req->C;
        r->dtype = req->dtype;
        r->flags = req->flags;
        r->t_submit = now_s();
        std::lock_guard<std::mutex> lk(p->mu);
        QSIM_REQUIRE(!p->stop, "pool is shutting down");
        r->id = p->next_id++;
        *ticket = r->id;
        p->submitted.push_back(r.get());
        p->reqs.emplace(r->id, std::move(r));
        p->cv_work.notify_all();
    });
}

int qsim_poll(qsim_pool *p, uint64_t ticket, double *x_out, hhl_readout_stats *stats, double *latency_s) {
    // status codes are returned directly (EBUSY pending, ENOTFOUND unknown, the request's error)
    if (!p) {
        set_last_error("NULL pool");
        return QSIM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(p->mu);
    auto it = p->reqs.find(ticket);
    if (it == p->reqs.end()) {
        set_last_error("unknown ticket");
        return QSIM_ENOTFOUND;
    }
    PoolReq *r = it->second.get();
    if (r->status == QSIM_EBUSY) {
        set_last_error("not finished");
        return QSIM_EBUSY;
    }
    const int st = r->status;
    if (st == QSIM_OK) {
        if (x_out) std::memcpy(x_out, r->x.data(), r->x.size() * sizeof(double));
        if (stats) *stats = r->stats;
        clear_last_error();
    } else {
        set_last_error(r->err);
    }
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    p->reqs.erase(it);
    return st;
}

int qsim_pool_wait(qsim_pool *p, uint64_t ticket, double timeout_s) {
    if (!p) {
        set_last_error("NULL pool");
        return QSIM_EINVAL;
    }
    std::unique_lock<std::mutex> lk(p->mu);
    auto done = [&] {
        auto it = p->reqs.find(ticket);
        return it == p->reqs.end() || it->second->status != QSIM_EBUSY;
    };
    if (!p->cv_done.wait_for(lk, std::chrono::duration<double>(std::max(0.0, timeout_s)), done)) {
        set_last_error("timed out waiting for the request");
        return QSIM_ETIMEOUT;
    }
    if (p->reqs.find(ticket) == p->reqs.end()) {
        set_last_error("unknown ticket");
        return QSIM_ENOTFOUND;
    }
    clear_last_error();
    return QSIM_OK;
}

int qsim_pool_take_completed(qsim_pool *p, uint64_t *tickets, int capacity, int *count, double timeout_s) {
    return guarded([&] {
        QSIM_REQUIRE(p != nullptr && tickets != nullptr && count != nullptr && capacity > 0, "bad arguments");
        std::unique_lock<std::mutex> lk(p->mu);
        p->cv_done.wait_for(lk, std::chrono::duration<double>(std::max(0.0, timeout_s)),
                            [&] { return !p->completed.empty(); });
        int k = 0;
        while (k < capacity && !p->completed.empty()) {
            tickets[k++] = p->completed.front();
            p->completed.pop_front();
        }
        *count = k;
    });
}

int qsim_pool_get_info(qsim_pool *p, qsim_pool_info *o) {
    return guarded([&] {
        QSIM_REQUIRE(p != nullptr && o != nullptr, "NULL argument");
        std::lock_guard<std::mutex> lk(p->mu);
        o->bytes_total = p->arena->cap();
        o->bytes_in_use = p->arena->used();
        o->bytes_peak = p->arena->peak();
        o->queued = (int)(p->submitted.size() + p->built.size()) + p->n_ready;
        o->building = p->n_building;
        o->running = p->n_running;
        o->done = p->n_done;
        o->failed = p->n_failed;
        o->batches_launched = p->batches;
        o->singles_launched = p->singles;
    });
}

int qsim_pool_launch_log(qsim_pool *p, qsim_pool_launch *out, int capacity, int *count) {
    return guarded([&] {
        QSIM_REQUIRE(p != nullptr && out != nullptr && count != nullptr && capacity >= 0, "bad arguments");
        std::lock_guard<std::mutex> lk(p->mu);
        const int k = std::min<int>(capacity, (int)p->launch_log.size());
        const size_t from = p->launch_log.size() - (size_t)k;
        for (int i = 0; i < k; i++) out[i] = p->launch_log[from + i];
        *count = k;
    });
}

void qsim_pool_destroy(qsim_pool *p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(p->mu);
        p->stop = true;
        // queued, unbuilt requests are dropped
        for (PoolReq *r : p->submitted) fail(p, r, QSIM_EINVAL, "pool destroyed");
        p->submitted.clear();
        p->cv_work.notify_all();
    }
    for (std::thread &t : p->builders) t.join();
    {
        std::lock_guard<std::mutex> lk(p->mu);
        p->cv_work.notify_all();
    }
    if (p->scheduler.joinable()) p->scheduler.join();
    for (Slot &s : p->slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        if (s.ev) cudaEventDestroy(s.ev);
        if (s.ev_start) cudaEventDestroy(s.ev_start);
        if (s.ev_end) cudaEventDestroy(s.ev_end);
        if (s.st) cudaStreamDestroy(s.st);
        if (s.pinned) cudaFreeHost(s.pinned);
    }
    p->reqs.clear();
    if (p->ev_ref) cudaEventDestroy(p->ev_ref);
    if (p->arena_base) cudaFree(p->arena_base);
    delete p;
}

}  // extern "C"
