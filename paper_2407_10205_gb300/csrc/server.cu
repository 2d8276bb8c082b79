// server.cu -- continuous-batching serving loop for PHIA requests (phia_server_* of the
// C ABI).  A scheduler thread admits queued requests in arrival order as soon as a slot
// and enough of the device-memory budget are free, keeps each admitted request's
// instance and replica state resident on the device, runs it in chunks of iterations on
// the slot's own stream (so requests overlap on the GPU), and retires it when a chunk
// shows its target reached or its step cap spent.  Requests arriving while others run
// are admitted as slots free up.  Every result depends only on the request (instance,
// schedule, replicas, seed, Philox instance id), never on the slot or the mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/phia.h"
#include "phia_internal.h"

using namespace phia;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    // instance copy (host)
    int32_t N = 0, frac_bits = 0;
    std::vector<int8_t> J;                 // dense, or empty
    std::vector<int32_t> row_ptr, col;
    std::vector<int8_t> val;
    std::vector<int32_t> h;
    uint32_t instance_id = 0;
    phia_schedule sched{};
    int32_t replicas = 0;
    int64_t step_cap = 0;
    uint64_t seed = 0;
    int64_t bytes = 0;                     // device-memory estimate
    bool resident = false;                 // dense and small enough for a resident kernel
    // progress
    int state = 0;                         // 0 queued, 1 running, 2 done, < 0 error
    int slot = -1;
    phia_t *h_dev = nullptr;
    float *x = nullptr, *v = nullptr;
    int64_t t_next = 0;                    // next iteration to run
    cudaEvent_t ev = nullptr;
    Clock::time_point t_submit, t_admit, t_done;
    // result
    int32_t hit = 0;
    int64_t energy_k = 0, hit_step = -1, steps_run = 0;
    std::vector<int8_t> spins;
    int32_t path = 0;
};

}  // namespace

struct phia_server_s {
    phia_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<int64_t> queue;
    std::map<int64_t, Request> reqs;
    std::vector<int64_t> slot_req;         // request id in each slot, -1 = free
    std::vector<cudaStream_t> streams;
    int64_t next_id = 1;
    int64_t used_bytes = 0;
    std::atomic<bool> stop{false};
    std::thread worker;
    Clock::time_point t0;
    // statistics
    int64_t completed = 0, spin_updates = 0;
    std::vector<double> ttt_arrival, ttt_admit;    // seconds, requests that hit their target
    int err = 0;
};

namespace {

double secs(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double>(b - a).count();
}

// Device bytes a request keeps resident (couplings, operands, replica state, records).
int64_t estimate_bytes(const Request &r, bool fp32) {
    const int64_t N = r.N, R = std::max(r.replicas, 1);
    const int64_t Rp = (R + 255) / 256 * 256;
    int64_t b = 2 * R * N * 4 + 3 * Rp * 8 + Rp * ((N + 31) / 32) * 4 + N * 4;   // caller x, v; records
    if (fp32) {
        b += N * N * 5 + 2 * R * N + R * N * 8;                       // int8 + FP32 J, spins, state
    } else if (!r.J.empty()) {
        b += N * N;                                                   // int8 J
        const int64_t Kb = (N * 2 + 127) / 128 * 128, Mp = (N + 127) / 128 * 128;
        b += Mp * Kb + 4 * ((R + 127) / 128 * 128) * Kb + R * N * 8;   // operand, spin buffers, state
    } else {
        b += (int64_t)r.col.size() * 5 + (N + 1) * 4;                 // CSR
        b += Rp * N * 8 + 4 * N * (Rp / 32) * 4;                      // state, spin bits
    }
    return b + (1 << 20);
}

void finish(phia_server_s *S, Request &r, int code) {
    r.t_done = Clock::now();
    r.state = code == PHIA_OK ? 2 : code;
    if (r.h_dev) {
        if (code == PHIA_OK) {
            phia_stats st{};
            if (phia_stats_get(r.h_dev, &st) == PHIA_OK) {
                r.hit = st.hit_step >= 0;
                r.hit_step = st.hit_step;
                r.path = st.path;
            }
            r.spins.assign(r.N, 0);
            int64_t e = 0;
            if (phia_best(r.h_dev, &e, r.spins.data()) == PHIA_OK) r.energy_k = e;
        }
        phia_destroy(r.h_dev);
        r.h_dev = nullptr;
    }
    cudaFree(r.x);
    cudaFree(r.v);
    r.x = r.v = nullptr;
    if (r.ev) cudaEventDestroy(r.ev);
    r.ev = nullptr;
    if (r.slot >= 0) S->slot_req[r.slot] = -1;
    r.slot = -1;
    S->used_bytes -= r.bytes;
    ++S->completed;
    S->spin_updates += (int64_t)r.replicas * r.N * r.steps_run;
    if (r.hit) {
        S->ttt_arrival.push_back(secs(r.t_submit, r.t_done));
        S->ttt_admit.push_back(secs(r.t_admit, r.t_done));
    }
    r.J.clear(); r.J.shrink_to_fit();
    r.row_ptr.clear(); r.col.clear(); r.val.clear(); r.h.clear();
}

// Launch the next chunk of a running request on its slot's stream.
int launch_chunk(phia_server_s *S, Request &r) {
    // A resident kernel stops at the target by itself inside its one launch, so such a
    // request runs to its step cap in one chunk; per-iteration paths check between chunks.
    const int64_t per = r.resident && S->opts.path != PHIA_PATH_FP32 ? r.step_cap : S->opts.chunk_iters;
    const int64_t chunk = std::min<int64_t>(per, r.step_cap - r.t_next);
    int rc = phia_run(r.h_dev, &r.sched, r.replicas, r.t_next, chunk, r.step_cap, r.seed, r.x, r.v,
                      r.t_next == 0 ? 1 : 0);
    if (rc) return rc;
    r.t_next += chunk;
    r.steps_run = r.t_next;
    if (cudaEventRecord(r.ev, S->streams[r.slot]) != cudaSuccess) return PHIA_ECUDA;
    return PHIA_OK;
}

int admit(phia_server_s *S, Request &r, int slot) {
    r.slot = slot;
    r.t_admit = Clock::now();
    phia_opts o{};
    o.device = S->opts.device;
    o.instance_id = r.instance_id;
    o.stream = S->streams[slot];
    int rc;
    if (S->opts.path == PHIA_PATH_FP32) {
        // the comparator: every request as a dense FP32 instance
        o.path = PHIA_PATH_FP32;
        if (r.J.empty()) {
            r.J.assign((size_t)r.N * r.N, 0);
            for (int i = 0; i < r.N; ++i)
                for (int32_t p = r.row_ptr[i]; p < r.row_ptr[i + 1]; ++p) r.J[(size_t)i * r.N + r.col[p]] = r.val[p];
        }
        rc = phia_create(&r.h_dev, r.J.data(), r.h.data(), r.N, r.frac_bits, &o);
    } else if (!r.J.empty()) {
        o.path = PHIA_PATH_TC;
        rc = phia_create(&r.h_dev, r.J.data(), r.h.data(), r.N, r.frac_bits, &o);
    } else {
        o.path = PHIA_PATH_CSR;
        rc = phia_create_csr(&r.h_dev, r.row_ptr.data(), r.col.data(), r.val.data(), r.h.data(), r.N, r.frac_bits, &o);
    }
    if (rc) return rc;
    const size_t bytes = (size_t)r.replicas * r.N * 4;
    if (cudaMalloc(&r.x, bytes) != cudaSuccess || cudaMalloc(&r.v, bytes) != cudaSuccess) return PHIA_ENOMEM;
    if (cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess) return PHIA_ECUDA;
    rc = phia_init_state(r.h_dev, r.replicas, r.seed, r.x, r.v);
    if (rc) return rc;
    r.state = 1;
    S->slot_req[slot] = r.id;
    return launch_chunk(S, r);
}

void worker_loop(phia_server_s *S) {
    cudaSetDevice(S->opts.device);
    std::unique_lock<std::mutex> lock(S->mu);
    while (!S->stop) {
        bool progress = false;
        // retire or continue running requests whose last chunk finished
        for (size_t s = 0; s < S->slot_req.size(); ++s) {
            const int64_t id = S->slot_req[s];
            if (id < 0) continue;
            Request &r = S->reqs[id];
            const cudaError_t q = cudaEventQuery(r.ev);
            if (q == cudaErrorNotReady) continue;
            progress = true;
            if (q != cudaSuccess) { finish(S, r, PHIA_ECUDA); continue; }
            phia_stats st{};
            int rc = phia_stats_get(r.h_dev, &st);
            if (rc) { finish(S, r, rc); continue; }
            const bool hit = r.sched.has_target && st.hit_step >= 0;
            if (hit || r.t_next >= r.step_cap) {
                finish(S, r, PHIA_OK);
            } else {
                rc = launch_chunk(S, r);
                if (rc) finish(S, r, rc);
            }
        }
        // admit queued requests in arrival order while a slot and memory are free
        while (!S->queue.empty()) {
            const int64_t id = S->queue.front();
            Request &r = S->reqs[id];
            auto it = std::find(S->slot_req.begin(), S->slot_req.end(), (int64_t)-1);
            if (it == S->slot_req.end()) break;
            if (S->used_bytes + r.bytes > S->opts.hbm_budget_bytes && S->used_bytes > 0) break;
            S->queue.pop_front();
            S->used_bytes += r.bytes;
            const int rc = admit(S, r, (int)(it - S->slot_req.begin()));
            if (rc) finish(S, r, rc);
            progress = true;
        }
        S->cv.notify_all();
        if (!progress) {
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lock.lock();
        }
    }
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return -1.0;
    std::sort(v.begin(), v.end());
    const double pos = p * (v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - lo) * (v[hi] - v[lo]);
}

}  // namespace

extern "C" {

int phia_server_create(phia_server_t **out, const phia_server_opts *opts) {
    if (!out || !opts) return set_last_error(PHIA_EINVAL, "NULL argument");
    *out = nullptr;
    if (opts->max_inflight < 1 || opts->max_inflight > 256) return set_last_error(PHIA_EINVAL, "max_inflight in [1, 256]");
    if (opts->hbm_budget_bytes <= 0) return set_last_error(PHIA_EINVAL, "hbm_budget_bytes must be > 0");
    if (opts->chunk_iters < 1) return set_last_error(PHIA_EINVAL, "chunk_iters must be >= 1");
    if (opts->path != PHIA_PATH_AUTO && opts->path != PHIA_PATH_FP32)
        return set_last_error(PHIA_EINVAL, "server path must be PHIA_PATH_AUTO or PHIA_PATH_FP32");
    if (cudaSetDevice(opts->device) != cudaSuccess) return set_last_error(PHIA_ECUDA, "cudaSetDevice failed");
    phia_server_s *S = new phia_server_s();
    S->opts = *opts;
    S->slot_req.assign(opts->max_inflight, -1);
    for (int s = 0; s < opts->max_inflight; ++s) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            phia_server_destroy(S);
            return set_last_error(PHIA_ECUDA, "stream creation failed");
        }
        S->streams.push_back(st);
    }
    S->t0 = Clock::now();
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return PHIA_OK;
}

int phia_server_submit(phia_server_t *S, const phia_instance_desc *d, const phia_schedule *sched, int32_t replicas,
                       int64_t step_cap, uint64_t seed, int64_t *request_id) {
    if (!S || !d || !sched || !request_id) return set_last_error(PHIA_EINVAL, "NULL argument");
    if (d->N < 1 || !d->h_k || replicas < 1 || step_cap < 1)
        return set_last_error(PHIA_EINVAL, "need N >= 1, h_k, replicas >= 1, step_cap >= 1");
    if (!d->J_k && (!d->row_ptr || !d->col || !d->val_k)) return set_last_error(PHIA_EINVAL, "no couplings given");
    Request r;
    r.N = d->N;
    r.frac_bits = d->frac_bits;
    r.h.assign(d->h_k, d->h_k + d->N);
    if (d->J_k) {
        r.J.assign(d->J_k, d->J_k + (size_t)d->N * d->N);
        int max_abs = 0;
        for (int8_t k : r.J) max_abs = std::max(max_abs, k < 0 ? -(int)k : (int)k);
        r.resident = d->N <= tc_small_max_n(max_abs <= 16 ? kOpE4M3 : kOpBF16);
    } else {
        r.row_ptr.assign(d->row_ptr, d->row_ptr + d->N + 1);
        const int32_t nnz = d->row_ptr[d->N];
        r.col.assign(d->col, d->col + nnz);
        r.val.assign(d->val_k, d->val_k + nnz);
    }
    r.instance_id = d->instance_id;
    r.sched = *sched;
    if (d->has_target) {
        r.sched.has_target = 1;
        r.sched.target_k = d->target_k;
    }
    r.sched.stop_at_target = r.sched.has_target;
    r.replicas = replicas;
    r.step_cap = step_cap;
    r.seed = seed;
    r.bytes = estimate_bytes(r, S->opts.path == PHIA_PATH_FP32);
    r.t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(S->mu);
    if (r.bytes > S->opts.hbm_budget_bytes)
        return set_last_error(PHIA_ENOMEM, "request needs more device memory than the whole budget");
    r.id = S->next_id++;
    *request_id = r.id;
    S->queue.push_back(r.id);
    S->reqs.emplace(r.id, std::move(r));
    return PHIA_OK;
}

int phia_server_poll(phia_server_t *S, int64_t id, phia_request_status *st, int8_t *spins) {
    if (!S || !st) return set_last_error(PHIA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return set_last_error(PHIA_EINVAL, "unknown request id");
    const Request &r = it->second;
    memset(st, 0, sizeof *st);
    st->state = r.state;
    st->hit = r.hit;
    st->energy_k = r.energy_k;
    st->hit_step = r.hit_step;
    st->steps_run = r.steps_run;
    st->path = r.path;
    st->t_submit_s = secs(S->t0, r.t_submit);
    st->t_admit_s = r.state >= 1 || r.state < 0 ? secs(S->t0, r.t_admit) : -1.0;
    st->t_done_s = r.state == 2 || r.state < 0 ? secs(S->t0, r.t_done) : -1.0;
    if (spins && r.state == 2 && (int)r.spins.size() == r.N) memcpy(spins, r.spins.data(), r.N);
    return PHIA_OK;
}

int phia_server_wait_all(phia_server_t *S, int64_t timeout_ms) {
    if (!S) return set_last_error(PHIA_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lock(S->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    auto idle = [&] {
        return S->queue.empty() &&
               std::all_of(S->slot_req.begin(), S->slot_req.end(), [](int64_t x) { return x < 0; });
    };
    while (!idle()) {
        if (S->cv.wait_until(lock, deadline) == std::cv_status::timeout && !idle())
            return set_last_error(PHIA_ETIMEOUT, "requests still pending at the deadline");
    }
    return PHIA_OK;
}

int phia_server_stats_get(phia_server_t *S, phia_server_stats *out) {
    if (!S || !out) return set_last_error(PHIA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    memset(out, 0, sizeof *out);
    out->completed = S->completed;
    out->hits = (int64_t)S->ttt_arrival.size();
    out->spin_updates = S->spin_updates;
    out->ttt_p50_s = percentile(S->ttt_arrival, 0.50);
    out->ttt_p99_s = percentile(S->ttt_arrival, 0.99);
    out->ttt_admit_p50_s = percentile(S->ttt_admit, 0.50);
    out->ttt_admit_p99_s = percentile(S->ttt_admit, 0.99);
    out->elapsed_s = secs(S->t0, Clock::now());
    out->used_bytes = S->used_bytes;
    return PHIA_OK;
}

void phia_server_destroy(phia_server_t *S) {
    if (!S) return;
    S->stop = true;
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->opts.device);
    for (auto &kv : S->reqs) {
        Request &r = kv.second;
        if (r.ev) cudaEventSynchronize(r.ev);
        if (r.h_dev) phia_destroy(r.h_dev);
        cudaFree(r.x);
        cudaFree(r.v);
        if (r.ev) cudaEventDestroy(r.ev);
    }
    for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
    delete S;
}

}  // extern "C"
