// sf_server.cu -- continuous-batching request loop over stabilizer frames.
//
// Requests (one circuit each: qubit count, frame capacity, an sf_op program
// and basis states whose amplitudes are wanted) are queued as they arrive and
// admitted while an execution slot is free and their device footprint
// (sf_footprint_bytes) fits in the HBM budget.  Each slot is a host worker
// with its own CUDA stream and frame handle; the frame stays resident on the
// device for the whole circuit, gate batch after gate batch, and the slots'
// kernels overlap on the GPU.  A request that arrives while others run is
// admitted as soon as a slot and memory free up, without waiting for the
// others to finish.  Admission is in arrival order; a request that does not
// fit may be passed by later ones that do, at most kMaxBypass times, after
// which admission waits for it.
//
// A slot keeps its handle between requests and reuses it (sf_reset) when the
// next request has the same qubit count and no larger capacity.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "sf.h"

namespace {

constexpr int kMaxBypass = 8;

struct Request {
    uint64_t id = 0;
    uint32_t n = 0;
    uint64_t cap = 0;
    double eps = 0.0;
    std::vector<sf_op> ops;
    std::vector<uint64_t> probes;  // n_probes x ceil(n/64) words
    uint32_t n_probes = 0;
    uint64_t bytes = 0;
    double t_submit = 0.0;
    int bypassed = 0;
};

struct Slot {
    std::thread th;
    cudaStream_t stream = nullptr;
    sf_handle h = nullptr;
    uint32_t h_n = 0;
    uint64_t h_cap = 0, h_bytes = 0;
};

}  // namespace

struct sf_server_s {
    std::chrono::steady_clock::time_point t0;
    uint64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::deque<sf_result> done;
    std::vector<Slot> slots;
    uint64_t bytes_in_use = 0;  // handles held by slots (busy or cached)
    uint64_t next_id = 1;
    uint64_t submitted = 0, completed = 0;
    uint32_t active = 0;
    bool stop = false;
    int dev = 0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// run one request on a slot's handle; fills the result's status and outputs.
// The GPU is shared with the other slots, so the program runs without
// whole-GPU launches: on one CTA while the frame is small, then per op.
void execute(sf_handle h, const Request& rq, sf_result& res) {
    const uint32_t Wabi = (rq.n + 63) / 64;
    uint64_t outcomes = 0;
    uint32_t nm = 0;
    sf_status st = sf_run_program(h, rq.ops.data(), rq.ops.size(), rq.eps, &outcomes, &nm, SF_RUN_ONE_CTA);
    uint64_t k = 0;
    if (st == SF_OK) st = sf_size(h, &k);  // synchronises: reports deferred device errors
    for (uint32_t p = 0; p < rq.n_probes && st == SF_OK; p++)
        st = sf_amplitude(h, rq.probes.data() + (size_t)p * Wabi, &res.amp[2 * p], &res.amp[2 * p + 1]);
    res.status = (int32_t)st;
    res.k_final = k;
    res.outcomes = outcomes;
    res.n_meas = nm;
    res.n_probes = rq.n_probes;
}

// index of the next admissible request for this slot (arrival order with
// bounded bypass), or -1.  Admitting a request either reuses the slot's cached
// handle or replaces it (its bytes are released, the new footprint taken).
long pick(sf_server_s* s, const Slot& slot) {
    for (size_t qi = 0; qi < s->queue.size(); qi++) {
        const Request& rq = s->queue[qi];
        const bool reuse = slot.h && slot.h_n == rq.n && slot.h_cap >= rq.cap;
        if (reuse || s->bytes_in_use - slot.h_bytes + rq.bytes <= s->budget) return (long)qi;
        if (rq.bypassed >= kMaxBypass) return -1;  // admission waits for the starved request
    }
    return -1;
}

void drop_handle(Slot& slot) {
    if (slot.h) sf_destroy(slot.h);
    slot.h = nullptr;
    slot.h_n = 0;
    slot.h_cap = 0;
}

void worker(sf_server_s* s, int si) {
    cudaSetDevice(s->dev);
    Slot& slot = s->slots[si];
    for (;;) {
        Request rq;
        bool reuse = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            long qi = -1;
            bool drop = false;
            s->cv_work.wait(lk, [&] {
                if (s->stop) return true;
                qi = pick(s, slot);
                // nothing fits while this idle slot still holds a cached handle:
                // give its memory back so that the queue can move
                drop = qi < 0 && slot.h && !s->queue.empty();
                return qi >= 0 || drop;
            });
            if (s->stop) return;
            if (qi < 0) {
                lk.unlock();
                drop_handle(slot);
                lk.lock();
                s->bytes_in_use -= slot.h_bytes;
                slot.h_bytes = 0;
                lk.unlock();
                s->cv_work.notify_all();
                continue;
            }
            for (long j = 0; j < qi; j++) s->queue[j].bypassed++;
            rq = std::move(s->queue[qi]);
            s->queue.erase(s->queue.begin() + qi);
            reuse = slot.h && slot.h_n == rq.n && slot.h_cap >= rq.cap;
            if (!reuse) {
                s->bytes_in_use = s->bytes_in_use - slot.h_bytes + rq.bytes;
                slot.h_bytes = rq.bytes;
            }
            s->active++;
        }
        sf_result res;
        std::memset(&res, 0, sizeof(res));
        res.id = rq.id;
        res.t_submit = rq.t_submit;
        res.t_start = s->now();
        sf_status st = SF_OK;
        if (reuse) {
            st = sf_reset(slot.h);
        } else {
            drop_handle(slot);
            st = sf_create(rq.n, rq.cap, slot.stream, &slot.h);
            if (st == SF_OK) {
                slot.h_n = rq.n;
                slot.h_cap = rq.cap;
            } else {
                slot.h = nullptr;
            }
        }
        if (st == SF_OK) {
            execute(slot.h, rq, res);
            if (res.status != SF_OK) sf_reset(slot.h);
        } else {
            res.status = (int32_t)st;
        }
        res.t_done = s->now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (!slot.h) {  // creation failed: nothing is held
                s->bytes_in_use -= slot.h_bytes;
                slot.h_bytes = 0;
            }
            s->done.push_back(res);
            s->completed++;
            s->active--;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

sf_status sf_server_create(uint64_t hbm_budget_bytes, uint32_t max_active, sf_server* out) {
    if (!out || max_active < 1 || max_active > 256 || hbm_budget_bytes == 0) return SF_EINVAL;
    *out = nullptr;
    sf_server s = new (std::nothrow) sf_server_s();
    if (!s) return SF_ENOMEM;
    s->t0 = std::chrono::steady_clock::now();
    s->budget = hbm_budget_bytes;
    if (cudaGetDevice(&s->dev) != cudaSuccess) {
        delete s;
        return SF_ECUDA;
    }
    s->slots.resize(max_active);
    for (uint32_t i = 0; i < max_active; i++) {
        if (cudaStreamCreateWithFlags(&s->slots[i].stream, cudaStreamNonBlocking) != cudaSuccess) {
            for (uint32_t j = 0; j < i; j++) cudaStreamDestroy(s->slots[j].stream);
            delete s;
            return SF_ECUDA;
        }
    }
    for (uint32_t i = 0; i < max_active; i++) s->slots[i].th = std::thread(worker, s, (int)i);
    *out = s;
    return SF_OK;
}

sf_status sf_server_submit(sf_server s, const sf_request* r, uint64_t* id) {
    if (!s || !r) return SF_EINVAL;
    if (r->n_qubits < 1 || r->n_qubits > 1024 || r->max_elems < 1 || r->n_probes > SF_SERVER_MAX_PROBES ||
        (r->n_ops && !r->ops) || (r->n_probes && !r->probes) || !(r->drop_eps >= 0.0))
        return SF_EINVAL;
    Request rq;
    rq.n = r->n_qubits;
    rq.cap = r->max_elems;
    rq.eps = r->drop_eps;
    rq.ops.assign(r->ops, r->ops + r->n_ops);
    const uint32_t Wabi = (r->n_qubits + 63) / 64;
    rq.n_probes = r->n_probes;
    rq.probes.assign(r->probes, r->probes + (size_t)r->n_probes * Wabi);
    rq.bytes = sf_footprint_bytes(rq.n, rq.cap);
    if (rq.bytes == 0) return SF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (rq.bytes > s->budget) return SF_ENOMEM;  // could never be admitted
    rq.id = s->next_id++;
    rq.t_submit = s->now();
    if (id) *id = rq.id;
    s->queue.push_back(std::move(rq));
    s->submitted++;
    s->cv_work.notify_all();
    return SF_OK;
}

uint32_t sf_server_poll(sf_server s, sf_result* out, uint32_t max_results) {
    if (!s || !out) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    uint32_t k = 0;
    while (k < max_results && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    return k;
}

sf_status sf_server_wait(sf_server s, double timeout_s) {
    if (!s) return SF_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto pred = [&] { return s->completed == s->submitted; };
    if (timeout_s < 0) {
        s->cv_done.wait(lk, pred);
        return SF_OK;
    }
    return s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred) ? SF_OK : SF_ETIMEOUT;
}

sf_status sf_server_stats_get(sf_server s, sf_server_stats* st) {
    if (!s || !st) return SF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    st->queued = (uint32_t)s->queue.size();
    st->active = s->active;
    st->bytes_in_use = s->bytes_in_use;
    st->submitted = s->submitted;
    st->completed = s->completed;
    return SF_OK;
}

double sf_server_clock(sf_server s) { return s ? s->now() : 0.0; }

sf_status sf_server_destroy(sf_server s) {
    if (!s) return SF_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& sl : s->slots)
        if (sl.th.joinable()) sl.th.join();
    for (auto& sl : s->slots) {
        if (sl.h) sf_destroy(sl.h);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    delete s;
    return SF_OK;
}

}  // extern "C"
