// Serving loop: continuous batching of whole QAOA evaluations (not in the
// paper; a serving pattern around its simulation).
//
// One scheduler thread per server.  Requests are copied at submit time and
// queued.  Finished work is retired by the host callback enqueued behind it
// (or, if the scheduler sees the completion event first, by the scheduler).
// Each scheduler iteration (1) retires finished work it finds by querying CUDA
// events, (2) admits waiting requests in arrival order while a slot (a CUDA
// stream with its own staging) is free and the device-memory footprint fits
// the budget:
//   * requests with n <= small_n_max are packed, up to max_batch at a time, into
//     one batched cost-table launch plus one small-n evolution launch (one CTA
//     per request, state resident in shared memory, any n and p per request);
//   * a larger request takes the waiting requests of the same shape with it (the
//     same n, m, p and angles: the same pass plan, schedule, phase tables and
//     butterfly coefficients), up to max_batch within the budget, and they run
//     as one batch: one batched cost-table launch, then one multi-pass
//     evolution over all their states (each pass one launch over the batch, the
//     wave-balanced grid of the batched evolution) with the fused p_succ
//     reduction; alone, it is the single-instance pass sequence;
//   * when the oldest request is large and over the budget, small requests
//     behind it are still packed into free slots (their footprint is a table).
// Device memory for tables and states comes from cudaMallocAsync on the slot's
// stream and returns with cudaFreeAsync, so admission never synchronises the
// device.  Results land in pinned host memory; the host callback enqueued
// behind the slot's completion event publishes them (no CUDA call in it) and
// wakes the waiters and the scheduler, which otherwise sleeps (bounded waits
// only).
#include <cuda_runtime.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "qaoa_internal.cuh"

namespace qaoa {

static uint64_t now_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

struct Req {
    uint64_t ticket;
    int n, m, k, p;
    std::vector<int32_t> var;
    std::vector<uint8_t> neg;
    std::vector<double> gamma, beta;
    uint64_t t_submit;
    size_t footprint;
};

enum SlotKind { SLOT_SINGLE = 0, SLOT_PACKED = 1, SLOT_GROUP = 2 };

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<std::shared_ptr<Req>> reqs;  // requests in flight on this slot
    size_t bytes = 0;                        // footprint charged
    uint64_t t_start = 0;
    // staging
    char *h_stage = nullptr, *d_stage = nullptr;
    size_t stage_cap = 0;
    double *d_part = nullptr;                // partials for the pass path
    size_t part_cap = 0;
    void *d_cost = nullptr, *d_state = nullptr;  // large job buffers (freed async)
    int kind = 0;                            // SLOT_SINGLE, SLOT_PACKED or SLOT_GROUP
    size_t res_off = 0;                      // packed / group: offset of the stats block in staging
    uint64_t gen = 0;                        // launches on this slot so far
};

}  // namespace qaoa

struct qaoa_server {
    qaoa_server_opts o;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<qaoa::Req>> waiting;
    std::map<uint64_t, qaoa_result> results;   // finished, not yet polled
    std::map<uint64_t, int> state;             // 0 waiting, 1 running
    std::vector<qaoa::Slot> slots;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t used_bytes = 0;
    uint64_t epoch = 0;  // bumped (under mu) by submits, cancels, shutdown and finished slots
    // submitted, completed, packed launches, single launches, peak bytes, cancelled, errors, grouped requests
    uint64_t counters[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t issue_ns = 0, issues = 0;  // host time spent issuing slots' work (uploads, launches, copies)
    uint64_t t_first = 0;               // first admission (CLOCK_MONOTONIC ns)
    int init_status = QAOA_OK;
};

namespace qaoa {

static size_t es_of(int dtype) { return dtype == QAOA_C64 ? 8 : 16; }

static int ensure_stage(Slot &s, size_t bytes) {
    if (s.stage_cap >= bytes) return QAOA_OK;
    if (s.h_stage) cudaFreeHost(s.h_stage);
    if (s.d_stage) cudaFree(s.d_stage);
    s.h_stage = s.d_stage = nullptr;
    s.stage_cap = 0;
    size_t want = std::max(bytes + bytes / 2, (size_t)1 << 20);
    QAOA_CUDA_TRY(cudaMallocHost((void **)&s.h_stage, want));
    QAOA_CUDA_TRY(cudaMalloc((void **)&s.d_stage, want));
    s.stage_cap = want;
    return QAOA_OK;
}

static void retire(qaoa_server *sv, Slot &s);

// The callback's argument: which launch on which slot it follows.
struct DoneToken {
    qaoa_server *sv;
    Slot *slot;
    uint64_t gen;
};

// Enqueued on a slot's stream behind its completion event, so the slot's
// results are in pinned host memory when it runs: it publishes them (unless
// the scheduler already has, or the slot has moved on to later work) and
// wakes the waiters and the scheduler.  Runs on a CUDA callback thread and
// calls no CUDA function; no thread holds the server's lock across a CUDA call
// that could wait for it, and server destruction synchronises every stream
// before freeing the server.
static void CUDART_CB slot_done_callback(void *arg) {
    DoneToken *tk = static_cast<DoneToken *>(arg);
    qaoa_server *sv = tk->sv;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (tk->slot->busy && tk->slot->gen == tk->gen) retire(sv, *tk->slot);
        sv->epoch++;
    }
    delete tk;
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
}

static int finish_slot(qaoa_server *sv, Slot &s) {
    QAOA_CUDA_TRY(cudaEventRecord(s.done, s.stream));
    DoneToken *tk = new DoneToken{sv, &s, s.gen};
    const cudaError_t e = cudaLaunchHostFunc(s.stream, slot_done_callback, tk);
    if (e != cudaSuccess) {
        delete tk;
        return cuda_error(e, "cudaLaunchHostFunc");
    }
    return QAOA_OK;
}

// Launch one large request on slot s (stream ordered, no host sync).
static int launch_large(qaoa_server *sv, Slot &s, Req &q) {
    const int dtype = sv->o.dtype;
    // with QAOA_Z2_HALF the request keeps only the half state (global-flip symmetry)
    const bool z2 = (sv->o.flags & QAOA_Z2_HALF) != 0;
    const size_t N = (size_t)1 << (z2 ? q.n - 1 : q.n);
    int rc;
    naesat_instance inst{q.n, q.m, q.k, q.var.data(), q.neg.data()};
    // staging: [0..2) stats (u64), [2..4) p_succ, norm; from byte 256 the
    // clause records of a list too long for kernel parameters
    if ((rc = ensure_stage(s, 256 + cost_table_big_bytes(q.m)))) return rc;
    QAOA_CUDA_TRY(cudaMallocAsync(&s.d_cost, N, s.stream));
    QAOA_CUDA_TRY(cudaMallocAsync(&s.d_state, N * es_of(dtype), s.stream));
    unsigned long long *d_stats = reinterpret_cast<unsigned long long *>(s.d_stage);
    double *d_res = reinterpret_cast<double *>(s.d_stage + 16);
    QAOA_CUDA_TRY(cudaMemsetAsync(d_stats, 0, 16, s.stream));
    if ((rc = launch_cost_table_one(&inst, (uint8_t *)s.d_cost, d_stats, s.stream, z2, s.d_stage + 256))) return rc;
    const int gx = pass_grid_x(dtype, z2 ? q.n - 1 : q.n, 1);
    if (gx < 0) return QAOA_ECUDA;
    if (s.part_cap < (size_t)gx * 2) {
        if (s.d_part) cudaFree(s.d_part);
        QAOA_CUDA_TRY(cudaMalloc((void **)&s.d_part, (size_t)gx * 2 * sizeof(double)));
        s.part_cap = (size_t)gx * 2;
    }
    EvolveReq r{1, q.n, table_top(q.m), q.p, dtype, sv->o.flags, (const uint8_t *)s.d_cost, s.d_state, nullptr,
                q.gamma.data(), q.beta.data(), d_res};
    if ((rc = evolve_device_impl(r, s.stream, s.d_part, gx))) return rc;
    QAOA_CUDA_TRY(cudaMemcpyAsync(s.h_stage, s.d_stage, 32, cudaMemcpyDeviceToHost, s.stream));
    QAOA_CUDA_TRY(cudaFreeAsync(s.d_cost, s.stream));
    QAOA_CUDA_TRY(cudaFreeAsync(s.d_state, s.stream));
    s.d_cost = s.d_state = nullptr;
    return finish_slot(sv, s);
}

// Same shape: one pass plan, schedule, phase tables and coefficients.
static bool same_shape(const Req &a, const Req &b) {
    return a.n == b.n && a.m == b.m && a.p == b.p && a.gamma == b.gamma && a.beta == b.beta;
}

// Launch B >= 2 large requests of the same shape on slot s as one batch.
static int launch_group(qaoa_server *sv, Slot &s, std::vector<std::shared_ptr<Req>> &batch) {
    const int B = (int)batch.size();
    const Req &q0 = *batch[0];
    const int dtype = sv->o.dtype;
    const bool z2 = (sv->o.flags & QAOA_Z2_HALF) != 0;
    const int nb = z2 ? q0.n - 1 : q0.n;  // the half table is the first 2^(n-1) entries
    const size_t N = (size_t)1 << nb;
    const int m_stride = std::max(q0.m, 1);
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_recs = 0;
    const size_t o_m = align(o_recs + (size_t)B * m_stride * sizeof(ClauseRec));
    const size_t o_up = align(o_m + (size_t)B * sizeof(int));  // end of the uploaded part
    const size_t o_stats = o_up;
    const size_t o_res = align(o_stats + (size_t)B * 2 * sizeof(unsigned long long));
    const size_t total = align(o_res + (size_t)B * 2 * sizeof(double));
    int rc;
    if ((rc = ensure_stage(s, total))) return rc;
    char *h = s.h_stage, *d = s.d_stage;
    ClauseRec *h_recs = reinterpret_cast<ClauseRec *>(h + o_recs);
    int *h_m = reinterpret_cast<int *>(h + o_m);
    for (int b = 0; b < B; ++b) {
        const Req &q = *batch[b];
        naesat_instance inst{q.n, q.m, q.k, q.var.data(), q.neg.data()};
        encode_instance(&inst, h_recs + (size_t)b * m_stride);
        h_m[b] = q.m;
    }
    // The single-instance grid width: each instance gets the blocks, and so the
    // per-block p_succ partials, it gets alone, so its result is the same bit
    // for bit whether it runs alone or in a batch.
    const int gx = pass_grid_x(dtype, nb, 1);
    if (gx < 0) return QAOA_ECUDA;
    if (s.part_cap < (size_t)B * gx * 2) {
        if (s.d_part) cudaFree(s.d_part);
        s.d_part = nullptr;
        s.part_cap = 0;
        QAOA_CUDA_TRY(cudaMalloc((void **)&s.d_part, (size_t)B * gx * 2 * sizeof(double)));
        s.part_cap = (size_t)B * gx * 2;
    }
    QAOA_CUDA_TRY(cudaMallocAsync(&s.d_cost, (size_t)B * N, s.stream));
    QAOA_CUDA_TRY(cudaMallocAsync(&s.d_state, (size_t)B * N * es_of(dtype), s.stream));
    QAOA_CUDA_TRY(cudaMemcpyAsync(d, h, o_up, cudaMemcpyHostToDevice, s.stream));
    unsigned long long *d_stats = reinterpret_cast<unsigned long long *>(d + o_stats);
    double *d_res = reinterpret_cast<double *>(d + o_res);
    QAOA_CUDA_TRY(cudaMemsetAsync(d_stats, 0, (size_t)B * 2 * sizeof(unsigned long long), s.stream));
    if ((rc = launch_cost_table_batch(B, nb, nullptr, nullptr, reinterpret_cast<const ClauseRec *>(d + o_recs),
                                      reinterpret_cast<const int *>(d + o_m), m_stride, (uint8_t *)s.d_cost, d_stats,
                                      s.stream, !z2)))
        return rc;
    EvolveReq r{B, q0.n, table_top(q0.m), q0.p, dtype, sv->o.flags, (const uint8_t *)s.d_cost, s.d_state, nullptr,
                q0.gamma.data(), q0.beta.data(), d_res};
    if ((rc = evolve_device_impl(r, s.stream, s.d_part, gx))) return rc;
    QAOA_CUDA_TRY(cudaMemcpyAsync(h + o_stats, d + o_stats, total - o_stats, cudaMemcpyDeviceToHost, s.stream));
    QAOA_CUDA_TRY(cudaFreeAsync(s.d_cost, s.stream));
    QAOA_CUDA_TRY(cudaFreeAsync(s.d_state, s.stream));
    s.d_cost = s.d_state = nullptr;
    s.res_off = o_stats;  // stats [B][2] u64, then (after alignment) results [B][2] f64
    return finish_slot(sv, s);
}

// Launch a packed batch of small requests on slot s.
static int launch_packed(qaoa_server *sv, Slot &s, std::vector<std::shared_ptr<Req>> &batch) {
    const int B = (int)batch.size();
    const int sign = (sv->o.flags & QAOA_MIXER_RX2B) ? -1 : 1;
    const int arith = arith_of(sv->o.dtype, sv->o.flags);
    int m_stride = 1, max_n = 1;
    size_t tab_n = 0, coef_n = 0, cost_bytes = 0;
    for (auto &q : batch) {
        m_stride = std::max(m_stride, q->m);
        max_n = std::max(max_n, q->n);
        tab_n += (size_t)std::max(q->p, 1) * (table_top(q->m) + 1);
        coef_n += (size_t)std::max(q->p, 1);
        cost_bytes += ((size_t)1 << q->n);
    }
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_recs = 0;
    const size_t o_m = align(o_recs + (size_t)B * m_stride * sizeof(ClauseRec));
    const size_t o_n = align(o_m + (size_t)B * sizeof(int));
    const size_t o_off = align(o_n + (size_t)B * sizeof(int));
    const size_t o_tab = align(o_off + (size_t)B * sizeof(uint64_t));
    const size_t o_coef = align(o_tab + 2 * tab_n * sizeof(double));
    const size_t o_jobs = align(o_coef + 4 * coef_n * sizeof(double));
    const size_t o_up = align(o_jobs + (size_t)B * sizeof(SmallJob));  // end of the uploaded part
    const size_t o_stats = o_up;
    const size_t o_res = align(o_stats + (size_t)B * 2 * sizeof(unsigned long long));
    const size_t total = align(o_res + (size_t)B * 2 * sizeof(double));
    int rc;
    if ((rc = ensure_stage(s, total))) return rc;
    QAOA_CUDA_TRY(cudaMallocAsync(&s.d_cost, cost_bytes, s.stream));
    char *h = s.h_stage, *d = s.d_stage;
    ClauseRec *h_recs = reinterpret_cast<ClauseRec *>(h + o_recs);
    int *h_m = reinterpret_cast<int *>(h + o_m);
    int *h_n = reinterpret_cast<int *>(h + o_n);
    uint64_t *h_off = reinterpret_cast<uint64_t *>(h + o_off);
    double *h_tab = reinterpret_cast<double *>(h + o_tab);
    double *h_coef = reinterpret_cast<double *>(h + o_coef);
    SmallJob *h_jobs = reinterpret_cast<SmallJob *>(h + o_jobs);
    size_t toff = 0, coff = 0, boff = 0;
    std::vector<double> re, im;
    for (int b = 0; b < B; ++b) {
        Req &q = *batch[b];
        naesat_instance inst{q.n, q.m, q.k, q.var.data(), q.neg.data()};
        encode_instance(&inst, h_recs + (size_t)b * m_stride);
        h_m[b] = q.m;
        h_n[b] = q.n;
        h_off[b] = boff;
        const int pl = std::max(q.p, 1);
        const int mt = table_top(q.m);
        re.resize(mt + 1);
        im.resize(mt + 1);
        for (int l = 0; l < pl; ++l) {
            LayerCoef k = q.p > 0 ? layer_coef(q.beta[l], sign, arith) : LayerCoef{1.0, 1.0, 0.0, true};
            double scale = std::pow(k.sigma, q.n);
            if (l == 0) scale *= std::pow(2.0, -0.5 * q.n);
            phase_table(q.p > 0 ? q.gamma[l] : 0.0, scale, mt, re.data(), im.data());
            for (int c = 0; c <= mt; ++c) {
                h_tab[2 * (toff + (size_t)l * (mt + 1) + c)] = re[c];
                h_tab[2 * (toff + (size_t)l * (mt + 1) + c) + 1] = im[c];
            }
            h_coef[4 * (coff + l)] = k.A;
            h_coef[4 * (coff + l) + 1] = k.B;
            h_coef[4 * (coff + l) + 2] = k.unit_a ? 1.0 : 0.0;
            h_coef[4 * (coff + l) + 3] = 0.0;
        }
        SmallJob j;
        j.cost = reinterpret_cast<const uint8_t *>(s.d_cost) + boff;
        j.state = nullptr;
        j.result = reinterpret_cast<double *>(d + o_res) + 2 * b;
        j.n = q.n;
        j.m = mt;
        j.p = q.p;
        j.table_off = (int)toff;
        j.coef_off = (int)coff;
        h_jobs[b] = j;
        toff += (size_t)pl * (mt + 1);
        coff += pl;
        boff += (size_t)1 << q.n;
    }
    QAOA_CUDA_TRY(cudaMemcpyAsync(d, h, o_up, cudaMemcpyHostToDevice, s.stream));
    QAOA_CUDA_TRY(cudaMemsetAsync(d + o_stats, 0, (size_t)B * 2 * sizeof(unsigned long long), s.stream));
    if ((rc = launch_cost_table_batch(B, max_n, reinterpret_cast<int *>(d + o_n), reinterpret_cast<uint64_t *>(d + o_off),
                                      reinterpret_cast<ClauseRec *>(d + o_recs), reinterpret_cast<int *>(d + o_m),
                                      m_stride, (uint8_t *)s.d_cost, reinterpret_cast<unsigned long long *>(d + o_stats),
                                      s.stream, true)))
        return rc;
    if ((rc = launch_small_batch(sv->o.dtype, B, reinterpret_cast<SmallJob *>(d + o_jobs),
                                 reinterpret_cast<double *>(d + o_tab), reinterpret_cast<double *>(d + o_coef), max_n,
                                 sv->o.flags, s.stream)))
        return rc;
    QAOA_CUDA_TRY(cudaMemcpyAsync(h + o_stats, d + o_stats, total - o_stats, cudaMemcpyDeviceToHost, s.stream));
    QAOA_CUDA_TRY(cudaFreeAsync(s.d_cost, s.stream));
    s.d_cost = nullptr;
    s.res_off = o_stats;  // stats [B][2] u64, then (after alignment) results [B][2] f64
    return finish_slot(sv, s);
}

static size_t footprint(const qaoa_server *sv, int n, bool packed) {
    const size_t N = (size_t)1 << n;
    if (packed) return N;
    return ((sv->o.flags & QAOA_Z2_HALF) ? N / 2 : N) * (1 + es_of(sv->o.dtype));
}

// Publishes the results of a finished slot (scheduler thread, lock held).
static void retire(qaoa_server *sv, Slot &s) {
    const bool packed = s.kind == SLOT_PACKED, group = s.kind == SLOT_GROUP;
    const uint64_t t = now_ns();
    const int B = (int)s.reqs.size();
    for (int b = 0; b < B; ++b) {
        Req &q = *s.reqs[b];
        qaoa_result r{};
        r.t_submit_ns = q.t_submit;
        r.t_start_ns = s.t_start;
        r.t_done_ns = t;
        if (packed) {
            // layout mirrors launch_packed: stats then results after the uploaded part
            const unsigned long long *st = reinterpret_cast<const unsigned long long *>(s.h_stage + s.res_off);
            const double *res = reinterpret_cast<const double *>(
                s.h_stage + ((s.res_off + (size_t)B * 16 + 255) & ~(size_t)255));
            r.n_sol = st[2 * b];
            r.max_cost = (uint32_t)st[2 * b + 1];
            r.p_succ = res[2 * b];
            r.norm = res[2 * b + 1];
        } else if (group) {
            // the same layout as a packed batch; halved tables and states count twice
            const unsigned long long *st = reinterpret_cast<const unsigned long long *>(s.h_stage + s.res_off);
            const double *res = reinterpret_cast<const double *>(
                s.h_stage + ((s.res_off + (size_t)B * 16 + 255) & ~(size_t)255));
            const double f = (sv->o.flags & QAOA_Z2_HALF) ? 2.0 : 1.0;
            r.n_sol = (uint64_t)(f * (double)st[2 * b]);
            r.max_cost = (uint32_t)st[2 * b + 1];
            r.p_succ = f * res[2 * b];
            r.norm = f * res[2 * b + 1];
        } else {
            const unsigned long long *st = reinterpret_cast<const unsigned long long *>(s.h_stage);
            const double *res = reinterpret_cast<const double *>(s.h_stage + 16);
            const double f = (sv->o.flags & QAOA_Z2_HALF) ? 2.0 : 1.0;  // halved state and table
            r.n_sol = (uint64_t)(f * (double)st[0]);
            r.max_cost = (uint32_t)st[1];
            r.p_succ = f * res[0];
            r.norm = f * res[1];
        }
        r.status = r.max_cost > 255 ? QAOA_ERANGE : QAOA_OK;
        if (r.status) sv->counters[6]++;
        sv->results[q.ticket] = r;
        sv->state.erase(q.ticket);
        sv->counters[1]++;
    }
    sv->used_bytes -= s.bytes;
    s.bytes = 0;
    s.reqs.clear();
    s.busy = false;
}

static void fail_slot(qaoa_server *sv, Slot &s, int code) {
    // a launch that failed part-way may still hold its job buffers
    if (s.d_cost) cudaFreeAsync(s.d_cost, s.stream);
    if (s.d_state) cudaFreeAsync(s.d_state, s.stream);
    s.d_cost = s.d_state = nullptr;
    cudaGetLastError();
    const uint64_t t = now_ns();
    for (auto &q : s.reqs) {
        qaoa_result r{};
        r.status = code;
        r.t_submit_ns = q->t_submit;
        r.t_start_ns = s.t_start;
        r.t_done_ns = t;
        sv->results[q->ticket] = r;
        sv->state.erase(q->ticket);
        sv->counters[6]++;
        sv->counters[1]++;
    }
    sv->used_bytes -= s.bytes;
    s.bytes = 0;
    s.reqs.clear();
    s.busy = false;
}

// Packs waiting small requests (any position in the queue) into one batch
// within the budget; returns the batch and its footprint.
static std::vector<std::shared_ptr<Req>> take_small(qaoa_server *sv, size_t *bytes) {
    std::vector<std::shared_ptr<Req>> batch;
    *bytes = 0;
    for (auto it = sv->waiting.begin(); it != sv->waiting.end() && (int)batch.size() < sv->o.max_batch;) {
        if ((*it)->n <= sv->o.small_n_max && sv->used_bytes + *bytes + (*it)->footprint <= sv->o.hbm_budget_bytes) {
            *bytes += (*it)->footprint;
            batch.push_back(*it);
            it = sv->waiting.erase(it);
        } else {
            ++it;
        }
    }
    return batch;
}

// The head (a large request that fits) and the waiting requests of its shape
// behind it, up to max_batch within the budget.
static std::vector<std::shared_ptr<Req>> take_group(qaoa_server *sv, size_t *bytes) {
    std::vector<std::shared_ptr<Req>> batch;
    auto head = sv->waiting.front();
    sv->waiting.pop_front();
    batch.push_back(head);
    *bytes = head->footprint;
    for (auto it = sv->waiting.begin(); it != sv->waiting.end() && (int)batch.size() < sv->o.max_batch;) {
        if (same_shape(**it, *head) && sv->used_bytes + *bytes + (*it)->footprint <= sv->o.hbm_budget_bytes) {
            *bytes += (*it)->footprint;
            batch.push_back(*it);
            it = sv->waiting.erase(it);
        } else {
            ++it;
        }
    }
    return batch;
}

static void scheduler(qaoa_server *sv) {
    cudaSetDevice(sv->o.device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        const uint64_t epoch0 = sv->epoch;
        // (1) retire finished slots
        bool any_busy = false;
        for (size_t i = 0; i < sv->slots.size(); ++i) {
            Slot &s = sv->slots[i];
            if (!s.busy) continue;
            cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaSuccess) {
                retire(sv, s);
                sv->cv_done.notify_all();
            } else if (e != cudaErrorNotReady) {
                cudaGetLastError();
                fail_slot(sv, s, QAOA_ECUDA);
                sv->cv_done.notify_all();
            } else {
                any_busy = true;
            }
        }
        if (sv->stop && sv->waiting.empty() && !any_busy) break;
        // (2) admit waiting requests, oldest first
        for (size_t i = 0; i < sv->slots.size() && !sv->waiting.empty(); ++i) {
            Slot &s = sv->slots[i];
            if (s.busy) continue;
            auto head = sv->waiting.front();
            const bool small = head->n <= sv->o.small_n_max;
            const bool fits = sv->used_bytes + head->footprint <= sv->o.hbm_budget_bytes || sv->used_bytes == 0;
            std::vector<std::shared_ptr<Req>> batch;
            size_t bytes = 0;
            int kind;
            if (small || !fits) {
                // a large head over the budget waits for retirements; small
                // requests behind it still run (their footprint is a table)
                batch = take_small(sv, &bytes);
                if (batch.empty()) break;
                kind = SLOT_PACKED;
            } else {
                batch = take_group(sv, &bytes);
                kind = batch.size() > 1 ? SLOT_GROUP : SLOT_SINGLE;
            }
            s.busy = true;
            s.gen++;
            s.bytes = bytes;
            s.reqs = batch;
            s.t_start = now_ns();
            s.kind = kind;
            sv->used_bytes += bytes;
            for (auto &q : batch) sv->state[q->ticket] = 1;
            if (kind == SLOT_PACKED) sv->counters[2]++;
            if (kind == SLOT_SINGLE) sv->counters[3]++;
            if (kind == SLOT_GROUP) sv->counters[7] += batch.size();
            lk.unlock();
            const uint64_t t_issue = now_ns();
            int rc = kind == SLOT_PACKED  ? launch_packed(sv, s, batch)
                     : kind == SLOT_GROUP ? launch_group(sv, s, batch)
                                          : launch_large(sv, s, *batch[0]);
            const uint64_t t_issued = now_ns();
            lk.lock();
            if (!sv->t_first) sv->t_first = t_issue;
            sv->issue_ns += t_issued - t_issue;
            sv->issues++;
            if (rc) {
                fail_slot(sv, s, rc);
                sv->cv_done.notify_all();
            }
            sv->counters[4] = std::max<uint64_t>(sv->counters[4], sv->used_bytes);
        }
        // (3) sleep until something changes: a submit, a cancel, shutdown or a
        // slot's completion callback (bounded, in case a wake-up is missed)
        bool busy = false;
        for (auto &s : sv->slots) busy = busy || s.busy;
        sv->cv_work.wait_for(lk, busy ? std::chrono::milliseconds(2) : std::chrono::milliseconds(20),
                             [&] { return sv->epoch != epoch0; });
    }
}

}  // namespace qaoa

using namespace qaoa;

extern "C" int qaoa_server_create(const qaoa_server_opts *opts, qaoa_server **out) {
    if (!opts || !out) return set_error(QAOA_EINVAL, "NULL argument");
    if (opts->dtype != QAOA_C64 && opts->dtype != QAOA_C128) return set_error(QAOA_EINVAL, "dtype=%d", opts->dtype);
    if (opts->flags & ~(QAOA_MIXER_RX2B | QAOA_Z2_HALF | QAOA_DF64))
        return set_error(QAOA_EINVAL, "server flags=0x%x (mixer sign, halved state, double-float)", opts->flags);
    if ((opts->flags & QAOA_DF64) && (opts->dtype != QAOA_C128 || (opts->flags & QAOA_Z2_HALF)))
        return set_error(QAOA_EINVAL, "QAOA_DF64 serves complex128 full states only");
    std::unique_ptr<qaoa_server> sv(new qaoa_server());
    sv->o = *opts;
    if (sv->o.max_batch <= 0) sv->o.max_batch = 256;
    if (sv->o.n_streams <= 0) sv->o.n_streams = 4;
    if (sv->o.max_n <= 0) sv->o.max_n = 30;
    const int pack = small_n_pack_limit(sv->o.dtype);
    if (sv->o.small_n_max <= 0) sv->o.small_n_max = pack;
    if (sv->o.small_n_max > pack) return set_error(QAOA_ERANGE, "small_n_max=%d above %d", sv->o.small_n_max, pack);
    // requests between small_n_max and the pass path's lower bound run packed alone
    if (sv->o.small_n_max < small_n_limit(sv->o.dtype)) sv->o.small_n_max = small_n_limit(sv->o.dtype);
    QAOA_CUDA_TRY(cudaSetDevice(sv->o.device));
    if (sv->o.hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        QAOA_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        sv->o.hbm_budget_bytes = fr / 2;
    }
    // keep freed stream-ordered allocations in the pool between requests
    cudaMemPool_t pool;
    QAOA_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, sv->o.device));
    uint64_t threshold = UINT64_MAX;
    QAOA_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold));
    sv->slots.resize(sv->o.n_streams);
    for (auto &s : sv->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e != cudaSuccess) {  // release what the earlier slots created
            for (auto &c : sv->slots) {
                if (c.done) cudaEventDestroy(c.done);
                if (c.stream) cudaStreamDestroy(c.stream);
            }
            return cuda_error(e, "server stream or event");
        }
    }
    qaoa_server *raw = sv.release();
    raw->worker = std::thread(scheduler, raw);
    *out = raw;
    return QAOA_OK;
}

extern "C" int qaoa_serve_submit(qaoa_server *sv, const naesat_instance *inst, int p, const double *gamma,
                                 const double *beta, uint64_t *ticket) {
    if (!sv || !ticket) return set_error(QAOA_EINVAL, "NULL argument");
    int rc = validate_instance(inst);
    if (rc) return rc;
    if (inst->n > sv->o.max_n) return set_error(QAOA_ERANGE, "n=%d above the server's max_n=%d", inst->n, sv->o.max_n);
    if (p < 0 || (p > 0 && (!gamma || !beta))) return set_error(QAOA_EINVAL, "p/gamma/beta");
    for (int l = 0; l < p; ++l)
        if (!std::isfinite(gamma[l]) || !std::isfinite(beta[l])) return set_error(QAOA_EINVAL, "angle %d not finite", l);
    auto q = std::make_shared<Req>();
    q->n = inst->n;
    q->m = inst->m;
    q->k = inst->m > 0 ? inst->k : 1;
    q->p = p;
    q->var.assign(inst->var, inst->var + (size_t)inst->m * inst->k);
    q->neg.assign(inst->neg, inst->neg + (size_t)inst->m * inst->k);
    q->gamma.assign(gamma, gamma + p);
    q->beta.assign(beta, beta + p);
    q->t_submit = now_ns();
    q->footprint = footprint(sv, q->n, q->n <= sv->o.small_n_max);
    if (q->footprint > sv->o.hbm_budget_bytes)
        return set_error(QAOA_ENOMEM, "request footprint %zu exceeds the budget %zu", q->footprint,
                         sv->o.hbm_budget_bytes);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) return set_error(QAOA_ECANCELLED, "server is shutting down");
        q->ticket = sv->next_ticket++;
        sv->waiting.push_back(q);
        sv->state[q->ticket] = 0;
        sv->counters[0]++;
        sv->epoch++;
        *ticket = q->ticket;
    }
    sv->cv_work.notify_one();
    return QAOA_OK;
}

extern "C" int qaoa_serve_poll(qaoa_server *sv, uint64_t ticket, qaoa_result *out) {
    if (!sv || !out) return set_error(QAOA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->results.find(ticket);
    if (it != sv->results.end()) {
        *out = it->second;
        sv->results.erase(it);
        return QAOA_OK;
    }
    if (sv->state.count(ticket)) return QAOA_PENDING;
    return set_error(QAOA_ENOTFOUND, "ticket %llu unknown or already retired", (unsigned long long)ticket);
}

extern "C" int qaoa_serve_wait(qaoa_server *sv, uint64_t ticket, qaoa_result *out, double timeout_s) {
    if (!sv || !out) return set_error(QAOA_EINVAL, "NULL argument");
    if (!(timeout_s >= 0.0) || !std::isfinite(timeout_s))
        return set_error(QAOA_EINVAL, "timeout_s=%g (a finite number of seconds >= 0)", timeout_s);
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        auto it = sv->results.find(ticket);
        if (it != sv->results.end()) {
            *out = it->second;
            sv->results.erase(it);
            return QAOA_OK;
        }
        if (!sv->state.count(ticket))
            return set_error(QAOA_ENOTFOUND, "ticket %llu unknown or already retired", (unsigned long long)ticket);
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && std::chrono::steady_clock::now() >= deadline) {
            if (sv->results.count(ticket)) continue;
            return set_error(QAOA_ETIMEOUT, "ticket %llu not done after %.3f s", (unsigned long long)ticket, timeout_s);
        }
    }
}

extern "C" int qaoa_serve_cancel(qaoa_server *sv, uint64_t ticket) {
    if (!sv) return set_error(QAOA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto it = sv->waiting.begin(); it != sv->waiting.end(); ++it) {
        if ((*it)->ticket == ticket) {
            qaoa_result r{};
            r.status = QAOA_ECANCELLED;
            r.t_submit_ns = (*it)->t_submit;
            r.t_done_ns = now_ns();
            sv->results[ticket] = r;
            sv->state.erase(ticket);
            sv->waiting.erase(it);
            sv->counters[5]++;
            sv->cv_done.notify_all();
            return QAOA_OK;
        }
    }
    if (sv->state.count(ticket)) return QAOA_PENDING;
    return set_error(QAOA_ENOTFOUND, "ticket %llu unknown", (unsigned long long)ticket);
}

extern "C" int qaoa_server_stats(qaoa_server *sv, uint64_t *counters) {
    if (!sv || !counters) return set_error(QAOA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    for (int i = 0; i < 8; ++i) counters[i] = sv->counters[i];
    return QAOA_OK;
}

extern "C" int qaoa_server_issue_time(qaoa_server *sv, uint64_t *issue_ns, uint64_t *issues, uint64_t *span_ns) {
    if (!sv || !issue_ns || !issues || !span_ns) return set_error(QAOA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *issue_ns = sv->issue_ns;
    *issues = sv->issues;
    *span_ns = sv->t_first ? now_ns() - sv->t_first : 0;
    return QAOA_OK;
}

extern "C" int qaoa_server_destroy(qaoa_server *sv) {
    if (!sv) return set_error(QAOA_EINVAL, "NULL argument");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->epoch++;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->o.device);
    for (auto &s : sv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.h_stage) cudaFreeHost(s.h_stage);
        if (s.d_stage) cudaFree(s.d_stage);
        if (s.d_part) cudaFree(s.d_part);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    delete sv;
    return QAOA_OK;
}
