// sf_api.cu -- the extern "C" boundary of libsf (declared in include/sf.h):
// handle lifetime, device memory, argument checks, the launch sequence of each
// operation and the synchronising reads.  All arithmetic of the method runs in
// the kernels of sf_tableau.cu and sf_frame.cu.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "sf.h"
#include "sf_device.cuh"

struct sf_frame_s {
    uint32_t n = 0;
    int Wabi = 1;
    SfDev d{};
    cudaStream_t stream = nullptr;
    int cur = 0;
    uint64_t* gws = nullptr;
    sf_gate_rec* dgates = nullptr;
    size_t dgates_cap = 0;
    sf_gate_rec* hstage = nullptr;
    size_t hstage_cap = 0;
    double2* dtrig = nullptr;   // term coefficients of the grid program's diagonal records, four per record
    size_t dtrig_cap = 0;
    OpRec* dops = nullptr;      // program records copied by sf_run_program
    size_t dops_cap = 0;
    OpRec* hops = nullptr;      // their pinned staging buffer
    size_t hops_cap = 0;
    cudaEvent_t ops_ev = nullptr;  // the last copy out of hops
    unsigned long long* dprog = nullptr;  // records consumed, outcome bits, count (one-CTA program)
    size_t dprog_cap = 0;
    unsigned long long* hprog = nullptr;  // their pinned copy
    cudaEvent_t stage_ev = nullptr;
    uint64_t* dy = nullptr;
    uint64_t* hy = nullptr;
    unsigned long long* hk = nullptr;
    uint32_t* hstatus = nullptr;
    double* hout = nullptr;
    int32_t* hmeta = nullptr;
    std::vector<void*> dallocs;
    std::string err;
    bool idx_ok[2] = {false, false};  // buffer b has a valid phase-vector index
    // no kernel has moved or changed the frame's elements since the last grid
    // program launch (whose layout, if it left one known, is still valid)
    bool layout = false;
    // what the grid program may assume about the hull of the frame (the span of
    // the differences of its phase vectors): 0 nothing, 1 the constraints its
    // last launch left in its workspace, 2 the frame is one element
    int hull = 2;
    uint32_t wait_limit = SF_WAIT_LIMIT_DEFAULT;
    int trace = 0;  // grid program launches record per-phase times
    uint64_t launches = 0;
    int time_id = -1;
    std::vector<cudaEvent_t> ev_pool;  // pairs (start, stop)
    size_t ev_used = 0;
};

namespace {

std::mutex g_err_mu;
std::string g_err;

sf_status fail(sf_handle h, sf_status code, const std::string& msg) {
    if (h) h->err = msg;
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_err = msg;
    return code;
}

sf_status cuda_fail(sf_handle h, cudaError_t e, const char* what) {
    return fail(h, SF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SF_CK(h, call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// handle's stream): creating or destroying a handle, or growing its gate
// buffer, never waits for kernels of other handles, so handles driven from
// several host threads overlap on the GPU.  Freed blocks stay in the device's
// default pool (release threshold raised once per process) for the next handle.
void keep_pool_memory() {
    static const bool once = [] {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        return true;
    }();
    (void)once;
}

template <typename T>
cudaError_t dalloc(sf_handle h, T** p, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMallocAsync(&v, std::max<size_t>(count, 1) * sizeof(T), h->stream);
    if (e == cudaSuccess) {
        h->dallocs.push_back(v);
        *p = static_cast<T*>(v);
    }
    return e;
}

// Pinned host buffers come from a process-wide pool of power-of-two blocks that
// are never returned to the driver (freeing pinned memory synchronises the
// whole device).
std::mutex g_pin_mu;
std::vector<std::vector<void*>> g_pin_free(64);

int pin_class(size_t bytes) {
    int c = 6;
    while ((size_t(1) << c) < bytes) c++;
    return c;
}

cudaError_t pinned_alloc(void** p, size_t bytes) {
    const int c = pin_class(bytes);
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (!g_pin_free[c].empty()) {
            *p = g_pin_free[c].back();
            g_pin_free[c].pop_back();
            return cudaSuccess;
        }
    }
    return cudaMallocHost(p, size_t(1) << c);
}

template <typename T>
cudaError_t pinned_alloc_n(T** p, size_t count) {
    void* v = nullptr;
    cudaError_t e = pinned_alloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    *p = static_cast<T*>(v);
    return e;
}

template <typename T>
void pinned_free(T* p, size_t count) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free[pin_class(std::max<size_t>(count, 1) * sizeof(T))].push_back(static_cast<void*>(p));
}

const char* status_text(uint32_t code) {
    switch (code) {
        case SF_EINVAL: return "invalid gate in a device gate list";
        case SF_ECAPACITY: return "frame would exceed max_elems";
        case SF_ETIMEOUT: return "hash probe limit reached during coalescing";
        case SF_ESTATE: return "invalid state";
        case SF_EINTERNAL: return "device-side consistency check of the tableau algebra failed";
        default: return "device error";
    }
}

// Launch one kernel of class `id`: count it and, when that class is being
// timed, bracket it with a pair of events from the handle's pool.
template <typename F>
sf_status launch(sf_handle h, int id, const char* what, F&& fn) {
    const bool timed = (h->time_id == id);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) {
        while (h->ev_pool.size() < 2 * (h->ev_used + 1)) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return fail(h, SF_ECUDA, "event creation failed");
            h->ev_pool.push_back(e);
        }
        e0 = h->ev_pool[2 * h->ev_used];
        e1 = h->ev_pool[2 * h->ev_used + 1];
        h->ev_used++;
    }
    // inside stream capture the pair must become event-record nodes of the graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (timed) cudaStreamIsCapturing(h->stream, &cap);
    const unsigned rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (timed) cudaEventRecordWithFlags(e0, h->stream, rec_flags);
    fn();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    if (timed) cudaEventRecordWithFlags(e1, h->stream, rec_flags);
    h->launches++;
    // a kernel that moves phase vectors to other coordinates or adds new ones
    // invalidates what the grid program knows about the frame's hull; subsets
    // of the frame (coalescing, collapse) keep it valid
    // the grid program's layout survives kernels that leave the elements where
    // and as they are
    switch (id) {
        case SF_K_GPROG:
            h->layout = true;
            break;
        case SF_K_INDEX: case SF_K_PROB: case SF_K_REDUCE: case SF_K_AMP_PREP: case SF_K_AMPLITUDE:
        case SF_K_EXPORT: case SF_K_MEASURE_PREP:
            break;
        default:
            h->layout = false;
    }
    switch (id) {
        case SF_K_CLIFFORD:
        case SF_K_AFFINE:
            if (h->hull != 2) h->hull = 0;  // one element stays one element
            break;
        case SF_K_RESET: case SF_K_GPROG: case SF_K_INDEX: case SF_K_INSERT: case SF_K_COMPACT: case SF_K_FILTER:
        case SF_K_PROB: case SF_K_REDUCE: case SF_K_AMP_PREP: case SF_K_AMPLITUDE: case SF_K_EXPORT:
        case SF_K_MEASURE_PREP:
            break;
        default:
            h->hull = 0;
    }
    return SF_OK;
}

#define SF_LAUNCH(h, id, call)                                  \
    do {                                                        \
        sf_status s_ = launch((h), (id), #call, [&] { call; }); \
        if (s_ != SF_OK) return s_;                             \
    } while (0)

sf_status clean_table(sf_handle h);

// wait for the stream and report a deferred device error, restoring the frame
// buffer that was current when it happened and clearing the error
sf_status sync_check(sf_handle h) {
    SF_CK(h, cudaMemcpyAsync(h->hstatus, h->d.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    SF_CK(h, cudaStreamSynchronize(h->stream));
    const uint32_t st = *h->hstatus;
    if (st) {
        h->cur = (int)((st >> 8) & 1u);
        h->idx_ok[0] = h->idx_ok[1] = false;
        h->hull = 0;
        h->layout = false;
        SF_CK(h, cudaMemsetAsync(h->d.status, 0, sizeof(uint32_t), h->stream));
        SF_CK(h, cudaMemsetAsync(h->d.done, 0, sizeof(unsigned int), h->stream));
        SF_CK(h, cudaMemsetAsync(h->d.ocnt, 0, sizeof(unsigned long long), h->stream));
        if (h->d.gp) SF_CK(h, sf_gprog_reset(h->d, h->stream));
        sf_status cs = clean_table(h);
        if (cs) return cs;
        SF_CK(h, cudaStreamSynchronize(h->stream));
        const uint32_t code = SF_ST_CODE(st);
        char site[32];
        snprintf(site, sizeof(site), " (check %u)", st >> 16);
        return fail(h, (sf_status)code, std::string(status_text(code)) + site);
    }
    return SF_OK;
}

// generic coalescing of in_buf into out_buf through the slot table
sf_status merge_seq(sf_handle h, double eps, int in_buf, int out_buf) {
    const SfDev& d = h->d;
    cudaStream_t s = h->stream;
    SF_LAUNCH(h, SF_K_INSERT, sf_launch_insert(d, in_buf, out_buf, s));
    SF_LAUNCH(h, SF_K_COMPACT, sf_launch_compact(d, eps, out_buf, s));
    h->idx_ok[out_buf] = sf_emit_index(d.W);
    return SF_OK;
}

// the index of buffer b, built if the last writer of b did not leave one
sf_status need_index(sf_handle h, int b) {
    if (!h->idx_ok[b]) {
        SF_LAUNCH(h, SF_K_INDEX, sf_launch_build_index(h->d, b, h->stream));
        h->idx_ok[b] = true;
    }
    return SF_OK;
}

// empty the slot table (after an error left it partly filled)
sf_status clean_table(sf_handle h) {
    const SfDev& d = h->d;
    if (d.W == 1) SF_CK(h, cudaMemsetAsync(d.tkey, 0xff, d.tcap * sizeof(uint64_t), h->stream));
    else SF_CK(h, cudaMemsetAsync(d.tstate, 0, d.tcap * sizeof(uint32_t), h->stream));
    SF_CK(h, cudaMemsetAsync(d.tacc, 0, d.tcap * sizeof(double2), h->stream));
    return SF_OK;
}

bool one_qubit(uint32_t kind) { return kind <= SF_Z; }

sf_status check_gate(sf_handle h, const sf_gate& g) {
    if (g.kind > SF_SWAP) return fail(h, SF_EINVAL, "unknown Clifford kind");
    if (g.q0 >= h->n) return fail(h, SF_EINVAL, "qubit out of range");
    if (!one_qubit(g.kind) && (g.q1 >= h->n || g.q1 == g.q0)) return fail(h, SF_EINVAL, "bad second qubit");
    return SF_OK;
}

sf_status run_clifford(sf_handle h, const sf_gate_rec* dev, uint64_t ng) {
    const uint64_t chunk = 1u << 20;
    for (uint64_t off = 0; off < ng; off += chunk) {
        const int m = (int)std::min<uint64_t>(chunk, ng - off);
        SF_LAUNCH(h, SF_K_CLIFFORD, sf_launch_clifford(h->d, dev + off, m, h->cur, h->gws, h->stream));
        // the affine map of each chunk is applied before the next chunk overwrites it
        SF_LAUNCH(h, SF_K_AFFINE, sf_launch_affine(h->d, h->cur, h->stream));
    }
    h->idx_ok[h->cur] = false;  // phase vectors changed; the index is rebuilt when needed
    return SF_OK;
}

// a device buffer of the handle that grows stream-ordered (earlier launches may
// still read the old one)
template <typename T>
sf_status grow_dev(sf_handle h, T** p, size_t& cap, size_t need) {
    if (need <= cap && *p) return SF_OK;
    size_t c = cap ? cap : 256;
    while (c < need) c *= 2;
    void* v = nullptr;
    SF_CK(h, cudaMallocAsync(&v, c * sizeof(T), h->stream));
    auto it = std::find(h->dallocs.begin(), h->dallocs.end(), (void*)*p);
    if (*p && it != h->dallocs.end()) {
        cudaFreeAsync(*it, h->stream);
        *it = v;
    } else {
        h->dallocs.push_back(v);
    }
    *p = static_cast<T*>(v);
    cap = c;
    return SF_OK;
}

}  // namespace

extern "C" {

sf_status sf_create(uint32_t n_qubits, uint64_t max_elems, void* cuda_stream, sf_handle* out) {
    if (!out) return fail(nullptr, SF_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > SF_MAX_N) return fail(nullptr, SF_EINVAL, "n_qubits must be in [1, 1024]");
    if (max_elems < 1 || max_elems > (1ull << 31)) return fail(nullptr, SF_EINVAL, "max_elems must be in [1, 2^31]");
    sf_handle h = new (std::nothrow) sf_frame_s();
    if (!h) return fail(nullptr, SF_ENOMEM, "host allocation failed");
    keep_pool_memory();
    h->n = n_qubits;
    h->Wabi = (int)((n_qubits + 63) / 64);
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    SfDev& d = h->d;
    d.n = (int)n_qubits;
    // words per phase vector: a power of two >= ceil(n/64); with one word, bit
    // 63 stays free (the slot table marks empty one-word keys with all ones),
    // so n = 64 takes two
    d.W = n_qubits <= 63 ? 1 : std::max(2, pow2_at_least((int)((n_qubits + 63) / 64)));
    d.NT = std::max(32, (int)((n_qubits + 31) / 32) * 32);
    d.cap = max_elems;
    d.lowrank = 1;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        sf_status st = cuda_fail(nullptr, e, "device query");
        delete h;
        return st;
    }
    int per_sm = 4;  // CTAs of 256 threads per SM for the per-element kernels
    if (const char* env = getenv("SF_CTAS_PER_SM")) per_sm = std::max(1, std::min(16, atoi(env)));
    d.nblk = std::max(1, sms) * per_sm;
    const size_t n = n_qubits, W = d.W, cap = max_elems;
    unsigned long long slots = 1024;
    while (slots < 2 * cap) slots <<= 1;
    d.tcap = slots;
#define SF_ALLOC(p, cnt)                                       \
    if ((e = dalloc(h, &(p), (cnt))) != cudaSuccess) {         \
        sf_destroy(h);                                         \
        return fail(nullptr, SF_ENOMEM, "device allocation failed"); \
    }
    SF_ALLOC(d.mx, W * n);
    SF_ALLOC(d.mz, W * n);
    SF_ALLOC(d.dx, W * n);
    SF_ALLOC(d.dz, W * n);
    SF_ALLOC(d.de, n);
    SF_ALLOC(d.piv, n);
    SF_ALLOC(d.meta, 4);
    SF_ALLOC(d.g, 1);
    for (int b = 0; b < 2; b++) {
        SF_ALLOC(d.sig[b], W * cap);
        SF_ALLOC(d.amp[b], cap);
    }
    SF_ALLOC(d.kcnt, 2);
    SF_ALLOC(d.status, 1);
    SF_ALLOC(d.plan, plan_words((int)n, (int)W));
    if (W > 1) SF_ALLOC(d.tstate, slots);
    SF_ALLOC(d.tkey, W * slots);
    SF_ALLOC(d.tacc, slots);
    SF_ALLOC(d.tsize, 1);
    unsigned long long icap = 64;
    while (icap < 2 * cap) icap <<= 1;
    d.icap = icap;
    for (int b = 0; b < 2; b++) SF_ALLOC(d.islot[b], (size_t)slot_words((int)W) * icap);
    SF_ALLOC(d.itag, 2);
    SF_ALLOC(d.isize, 2);
    SF_ALLOC(d.done, 1);
    SF_ALLOC(d.ocnt, 1);
    SF_ALLOC(d.ipend, 1);
    SF_ALLOC(d.red, 4 * (size_t)d.nblk);
    SF_ALLOC(d.out, 8);
    if (W == 1) SF_ALLOC(d.gp, sf_gprog_work_words());
    SF_ALLOC(h->dy, W);
    h->dgates_cap = 256;
    SF_ALLOC(h->dgates, h->dgates_cap);
    const size_t wsb = sf_tableau_smem_bytes((int)n, (int)W, d.NT);
    if (wsb > 200 * 1024) SF_ALLOC(h->gws, (wsb + 7) / 8);
#undef SF_ALLOC
    h->hstage_cap = 256;
    if (pinned_alloc_n(&h->hstage, h->hstage_cap) != cudaSuccess ||
        pinned_alloc_n(&h->hy, W) != cudaSuccess ||
        pinned_alloc_n(&h->hk, 2) != cudaSuccess ||
        pinned_alloc_n(&h->hstatus, 1) != cudaSuccess ||
        pinned_alloc_n(&h->hout, 8) != cudaSuccess ||
        pinned_alloc_n(&h->hmeta, 4) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->stage_ev, cudaEventDisableTiming) != cudaSuccess) {
        sf_destroy(h);
        return fail(nullptr, SF_ENOMEM, "pinned host allocation failed");
    }
    cudaMemsetAsync(d.status, 0, sizeof(uint32_t), h->stream);
    for (int b = 0; b < 2; b++)
        cudaMemsetAsync(d.islot[b], 0, (size_t)slot_words((int)W) * icap * sizeof(uint64_t), h->stream);
    cudaMemsetAsync(d.itag, 0, 2 * sizeof(uint32_t), h->stream);
    cudaMemsetAsync(d.isize, 0, 2 * sizeof(unsigned long long), h->stream);
    cudaMemsetAsync(d.done, 0, sizeof(unsigned int), h->stream);
    cudaMemsetAsync(d.ocnt, 0, sizeof(unsigned long long), h->stream);
    if (d.gp) cudaMemsetAsync(d.gp, 0, sf_gprog_work_words() * sizeof(uint64_t), h->stream);
    if (clean_table(h) != SF_OK) {
        sf_destroy(h);
        return fail(nullptr, SF_ECUDA, "table initialisation failed");
    }
    cudaMemsetAsync(d.plan, 0, plan_words((int)n, (int)W) * sizeof(uint64_t), h->stream);
    cudaEventRecord(h->stage_ev, h->stream);
    h->cur = 0;
    sf_launch_reset(d, 0, h->stream);
    h->launches++;
    h->idx_ok[0] = true;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        sf_status st = cuda_fail(nullptr, e, "create");
        sf_destroy(h);
        return st;
    }
    *out = h;
    return SF_OK;
}

sf_status sf_destroy(sf_handle h) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    cudaStreamSynchronize(h->stream);  // pending copies may still use the pinned buffers
    for (void* p : h->dallocs) cudaFreeAsync(p, h->stream);
    cudaStreamSynchronize(h->stream);
    pinned_free(h->hstage, h->hstage_cap);
    pinned_free(h->hy, (size_t)h->d.W);
    pinned_free(h->hk, 2);
    pinned_free(h->hstatus, 1);
    pinned_free(h->hout, 8);
    pinned_free(h->hmeta, 4);
    pinned_free(h->hops, h->hops_cap);
    pinned_free(h->hprog, 4);
    if (h->ops_ev) cudaEventDestroy(h->ops_ev);
    if (h->stage_ev) cudaEventDestroy(h->stage_ev);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    delete h;
    return SF_OK;
}

sf_status sf_reset(sf_handle h) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    h->cur = 0;
    SF_LAUNCH(h, SF_K_RESET, sf_launch_reset(h->d, 0, h->stream));
    h->idx_ok[0] = true;
    h->idx_ok[1] = false;
    h->hull = 2;
    return SF_OK;
}

sf_status sf_apply_clifford(sf_handle h, const sf_gate* gates, uint64_t n_gates) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (n_gates == 0) return SF_OK;
    if (!gates) return fail(h, SF_EINVAL, "gates is NULL");
    for (uint64_t i = 0; i < n_gates; i++) {
        sf_status st = check_gate(h, gates[i]);
        if (st) return st;
    }
    // the previous staging copy must have left the pinned buffer
    SF_CK(h, cudaEventSynchronize(h->stage_ev));
    if (n_gates > h->hstage_cap) {
        pinned_free(h->hstage, h->hstage_cap);
        h->hstage = nullptr;
        size_t c = h->hstage_cap;
        while (c < n_gates) c *= 2;
        SF_CK(h, pinned_alloc_n(&h->hstage, c));
        h->hstage_cap = c;
    }
    if (n_gates > h->dgates_cap) {  // stream-ordered: earlier launches still read the old buffer
        size_t c = h->dgates_cap;
        while (c < n_gates) c *= 2;
        sf_gate_rec* p = nullptr;
        SF_CK(h, cudaMallocAsync(&p, c * sizeof(sf_gate_rec), h->stream));
        auto it = std::find(h->dallocs.begin(), h->dallocs.end(), (void*)h->dgates);
        if (it != h->dallocs.end()) {
            cudaFreeAsync(*it, h->stream);
            *it = p;
        }
        h->dgates = p;
        h->dgates_cap = c;
    }
    for (uint64_t i = 0; i < n_gates; i++) {
        h->hstage[i].kind = gates[i].kind;
        h->hstage[i].q0 = gates[i].q0;
        h->hstage[i].q1 = one_qubit(gates[i].kind) ? 0u : gates[i].q1;
        h->hstage[i].pad = 0;
    }
    SF_CK(h, cudaMemcpyAsync(h->dgates, h->hstage, n_gates * sizeof(sf_gate_rec), cudaMemcpyHostToDevice,
                             h->stream));
    SF_CK(h, cudaEventRecord(h->stage_ev, h->stream));
    return run_clifford(h, h->dgates, n_gates);
}

sf_status sf_apply_clifford_device(sf_handle h, const sf_gate* dev_gates, uint64_t n_gates) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (n_gates == 0) return SF_OK;
    if (!dev_gates) return fail(h, SF_EINVAL, "dev_gates is NULL");
    return run_clifford(h, reinterpret_cast<const sf_gate_rec*>(dev_gates), n_gates);
}

sf_status sf_apply_nonclifford(sf_handle h, uint32_t kind, uint32_t q0, uint32_t q1, double theta) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (kind > SF_CPHASE) return fail(h, SF_EINVAL, "unknown non-Clifford kind");
    if (q0 >= h->n) return fail(h, SF_EINVAL, "qubit out of range");
    if (kind == SF_CPHASE && (q1 >= h->n || q1 == q0)) return fail(h, SF_EINVAL, "bad second qubit");
    const uint32_t q1v = kind == SF_CPHASE ? q1 : 0u;
    SF_LAUNCH(h, SF_K_BRANCH, sf_launch_branch(h->d, kind, q0, q1v, theta, h->cur, h->cur ^ 1, h->stream));
    h->cur ^= 1;
    h->idx_ok[h->cur] = false;  // children may repeat phase vectors until coalesced
    return SF_OK;
}

sf_status sf_apply_nonclifford_coalesce(sf_handle h, uint32_t kind, uint32_t q0, uint32_t q1, double theta,
                                        double drop_eps) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (kind > SF_CPHASE) return fail(h, SF_EINVAL, "unknown non-Clifford kind");
    if (q0 >= h->n) return fail(h, SF_EINVAL, "qubit out of range");
    if (kind == SF_CPHASE && (q1 >= h->n || q1 == q0)) return fail(h, SF_EINVAL, "bad second qubit");
    if (!(drop_eps >= 0.0)) return fail(h, SF_EINVAL, "drop_eps must be >= 0");
    const uint32_t q1v = kind == SF_CPHASE ? q1 : 0u;
    sf_status st = need_index(h, h->cur);
    if (st) return st;
    SF_LAUNCH(h, SF_K_BRANCH_MERGE,
              sf_launch_branch_merge(h->d, kind, q0, q1v, theta, drop_eps, h->cur, h->cur ^ 1, h->stream));
    h->cur ^= 1;
    h->idx_ok[h->cur] = sf_emit_index(h->d.W);
    return SF_OK;
}

sf_status sf_apply_program(sf_handle h, const sf_op* dev_ops, uint64_t n_ops, double drop_eps,
                           uint64_t max_frame, uint64_t* dev_consumed, uint64_t* dev_meas) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (h->d.W != 1) return fail(h, SF_EINVAL, "sf_apply_program needs n_qubits <= 63");
    if (n_ops && !dev_ops) return fail(h, SF_EINVAL, "dev_ops is NULL");
    if (!(drop_eps >= 0.0)) return fail(h, SF_EINVAL, "drop_eps must be >= 0");
    if (n_ops == 0) {
        if (dev_consumed) SF_CK(h, cudaMemsetAsync(dev_consumed, 0, sizeof(uint64_t), h->stream));
        if (dev_meas) SF_CK(h, cudaMemsetAsync(dev_meas, 0, 2 * sizeof(uint64_t), h->stream));
        return SF_OK;
    }
    uint64_t lim = std::min<uint64_t>(h->d.cap, SF_SEGMENT_MAX_ELEMS);
    if (max_frame) lim = std::min<uint64_t>(lim, max_frame);
    const unsigned seg_cap = (unsigned)lim;
    SF_LAUNCH(h, SF_K_SEGMENT,
              sf_launch_segment(h->d, dev_ops, n_ops, drop_eps * drop_eps, seg_cap, h->cur,
                                reinterpret_cast<unsigned long long*>(dev_consumed),
                                reinterpret_cast<unsigned long long*>(dev_meas), h->stream));
    // the kernel leaves the frame in the current buffer; neither index is valid now
    h->idx_ok[0] = h->idx_ok[1] = false;
    return SF_OK;
}

sf_status sf_apply_program_grid(sf_handle h, const sf_op* dev_ops, uint64_t n_ops, double drop_eps,
                                uint64_t* dev_consumed) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (h->d.W != 1) return fail(h, SF_EINVAL, "sf_apply_program_grid needs n_qubits <= 63");
    if (n_ops && !dev_ops) return fail(h, SF_EINVAL, "dev_ops is NULL");
    if (!(drop_eps >= 0.0)) return fail(h, SF_EINVAL, "drop_eps must be >= 0");
    if (n_ops == 0) {
        if (dev_consumed) SF_CK(h, cudaMemsetAsync(dev_consumed, 0, sizeof(uint64_t), h->stream));
        return SF_OK;
    }
    sf_status gs = grow_dev(h, &h->dtrig, h->dtrig_cap, 4 * (size_t)n_ops);  // four term coefficients per record
    if (gs) return gs;
    cudaError_t ge = cudaSuccess;
    SF_LAUNCH(h, SF_K_GPROG,
              ge = sf_launch_gprog(h->d, dev_ops, n_ops, drop_eps * drop_eps, h->cur, h->idx_ok[h->cur] ? 1 : 0,
                                   h->hull, h->wait_limit, h->trace, h->dtrig,
                                   reinterpret_cast<unsigned long long*>(dev_consumed), h->stream));
    if (ge != cudaSuccess) return cuda_fail(h, ge, "grid program launch");
    // the frame ends in the current buffer, without an index; the kernel keeps
    // the hull in its workspace when it started from a known one
    h->idx_ok[0] = h->idx_ok[1] = false;
    h->hull = h->hull ? 1 : 0;
    return SF_OK;
}

// the records of one stretch [i, j) of Clifford and diagonal records, per op
static sf_status run_stretch_per_op(sf_handle h, const sf_op* ops, uint64_t i, uint64_t j, double drop_eps,
                                    std::vector<sf_gate>& gates) {
    for (uint64_t r = i; r < j; r++) {
        const sf_op& q = ops[r];
        if (q.kind <= SF_SWAP) {
            gates.push_back(sf_gate{q.kind, q.q0, q.q1, 0u});
            continue;
        }
        if (!gates.empty()) {
            sf_status st = sf_apply_clifford(h, gates.data(), gates.size());
            gates.clear();
            if (st) return st;
        }
        sf_status st = sf_apply_nonclifford_coalesce(h, q.kind - SF_OP_DIAG, q.q0, q.q1, q.param, drop_eps);
        if (st) return st;
    }
    return SF_OK;
}

sf_status sf_run_program(sf_handle h, const sf_op* ops, uint64_t n_ops, double drop_eps, uint64_t* outcomes,
                         uint32_t* n_meas, uint32_t flags) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (n_ops && !ops) return fail(h, SF_EINVAL, "ops is NULL");
    if (!(drop_eps >= 0.0)) return fail(h, SF_EINVAL, "drop_eps must be >= 0");
    if (flags & ~(uint32_t)SF_RUN_ONE_CTA) return fail(h, SF_EINVAL, "unknown flags");
    uint32_t nm = 0;
    for (uint64_t i = 0; i < n_ops; i++) {
        const sf_op& o = ops[i];
        const uint32_t k = o.kind == SF_OP_COND ? o.arg : o.kind;
        const bool two = (k >= SF_CNOT && k <= SF_SWAP) || k == SF_OP_DIAG + SF_CPHASE;
        bool ok = o.q0 < h->n && (!two || (o.q1 < h->n && o.q1 != o.q0));
        if (o.kind == SF_OP_COND) ok &= o.arg <= SF_SWAP;
        else ok &= k <= SF_SWAP || (k >= SF_OP_DIAG && k <= SF_OP_DIAG + SF_CPHASE) || k == SF_OP_MEASURE;
        if (!ok) return fail(h, SF_EINVAL, "bad program record " + std::to_string(i));
        nm += o.kind == SF_OP_MEASURE;
    }
    if (nm > 64) return fail(h, SF_EINVAL, "more than 64 measurements");
    const bool w1 = h->d.W == 1 && h->d.gp;
    const bool one_cta = (flags & SF_RUN_ONE_CTA) != 0;
    if (w1 && n_ops) {
        // the records go to the device once, through the pinned staging buffer
        if (!h->ops_ev) SF_CK(h, cudaEventCreateWithFlags(&h->ops_ev, cudaEventDisableTiming));
        SF_CK(h, cudaEventSynchronize(h->ops_ev));  // the previous copy has left the staging buffer
        if (n_ops > h->hops_cap) {
            pinned_free(h->hops, h->hops_cap);
            h->hops = nullptr;
            size_t c = h->hops_cap ? h->hops_cap : 256;
            while (c < n_ops) c *= 2;
            SF_CK(h, pinned_alloc_n(&h->hops, c));
            h->hops_cap = c;
        }
        sf_status gs = grow_dev(h, &h->dops, h->dops_cap, n_ops);
        if (gs) return gs;
        std::memcpy(h->hops, ops, n_ops * sizeof(OpRec));
        SF_CK(h, cudaMemcpyAsync(h->dops, h->hops, n_ops * sizeof(OpRec), cudaMemcpyHostToDevice, h->stream));
        SF_CK(h, cudaEventRecord(h->ops_ev, h->stream));
    }
    uint64_t bits = 0;
    uint32_t done_m = 0;
    uint64_t i = 0;
    if (w1 && one_cta && n_ops) {
        // the program from its first record on one CTA while the frame is small;
        // where it stops, the per-op calls continue (outcomes so far carried over)
        sf_status gs = grow_dev(h, &h->dprog, h->dprog_cap, 4);
        if (gs) return gs;
        if (!h->hprog) SF_CK(h, pinned_alloc_n(&h->hprog, 4));
        sf_status st = sf_apply_program(h, reinterpret_cast<const sf_op*>(h->dops), n_ops, drop_eps, 0,
                                        reinterpret_cast<uint64_t*>(h->dprog),
                                        reinterpret_cast<uint64_t*>(h->dprog + 1));
        if (st) return st;
        SF_CK(h, cudaMemcpyAsync(h->hprog, h->dprog, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 h->stream));
        st = sync_check(h);
        if (st) return st;
        i = h->hprog[0];
        bits = h->hprog[1];
        done_m = (uint32_t)h->hprog[2];
    }
    std::vector<sf_gate> gates;
    auto flush = [&]() -> sf_status {
        if (gates.empty()) return SF_OK;
        sf_status st = sf_apply_clifford(h, gates.data(), gates.size());
        gates.clear();
        return st;
    };
    while (i < n_ops) {
        const sf_op& o = ops[i];
        if (o.kind <= SF_SWAP || (o.kind >= SF_OP_DIAG && o.kind <= SF_OP_DIAG + SF_CPHASE)) {
            uint64_t j = i;
            while (j < n_ops && (ops[j].kind <= SF_SWAP ||
                                 (ops[j].kind >= SF_OP_DIAG && ops[j].kind <= SF_OP_DIAG + SF_CPHASE)))
                j++;
            sf_status st = SF_OK;
            if (w1 && !one_cta) {
                st = flush();
                if (!st) st = sf_apply_program_grid(h, reinterpret_cast<const sf_op*>(h->dops + i), j - i, drop_eps,
                                                    nullptr);
            } else {
                st = run_stretch_per_op(h, ops, i, j, drop_eps, gates);
            }
            if (st) return st;
            i = j;
            continue;
        }
        if (o.kind == SF_OP_COND) {
            uint64_t mask;
            std::memcpy(&mask, &o.param, sizeof(mask));
            if (__builtin_popcountll(bits & mask) & 1) gates.push_back(sf_gate{o.arg, o.q0, o.q1, 0u});
            i++;
            continue;
        }
        // measurement: outcome 1 iff the caller's draw is below p(1), then collapse
        sf_status st = flush();
        double p0 = 0.0, p1 = 0.0;
        if (!st) st = sf_measure(h, o.q0, -1, &p0, &p1);
        const int x = o.param < p1 ? 1 : 0;
        if (!st) st = sf_measure(h, o.q0, x, nullptr, nullptr);
        if (st) return st;
        if (x) bits |= 1ull << done_m;
        done_m++;
        i++;
    }
    sf_status st = flush();
    if (st) return st;
    if (outcomes) *outcomes = bits;
    if (n_meas) *n_meas = done_m;
    return SF_OK;
}

sf_status sf_grid_program_bytes(sf_handle h, uint64_t* bytes) {
    if (!h || !bytes) return fail(h, SF_EINVAL, "NULL argument");
    if (!h->d.gp) return fail(h, SF_EINVAL, "no grid program on this handle (n_qubits > 63)");
    SF_CK(h, sf_gprog_moved(h->d, h->hk, h->stream));
    sf_status st = sync_check(h);
    if (st) return st;
    *bytes = h->hk[0];
    return SF_OK;
}

sf_status sf_set_trace(sf_handle h, int32_t on) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    h->trace = on ? 1 : 0;
    return SF_OK;
}

sf_status sf_grid_program_trace(sf_handle h, uint64_t* rec, uint32_t cap, uint32_t* n) {
    if (!h || !n || (cap && !rec)) return fail(h, SF_EINVAL, "NULL argument");
    if (!h->d.gp) return fail(h, SF_EINVAL, "no grid program on this handle (n_qubits > 63)");
    sf_status st = sync_check(h);
    if (st) return st;
    unsigned m = 0;
    std::vector<uint64_t> base((size_t)cap * 5), marks((size_t)cap * 8);
    SF_CK(h, sf_gprog_trace(h->d, base.data(), cap, &m, h->stream));
    SF_CK(h, sf_gprog_marks(h->d, marks.data(), m, h->stream));
    SF_CK(h, cudaStreamSynchronize(h->stream));
    for (unsigned i = 0; i < m; i++) {
        std::memcpy(rec + 13 * (size_t)i, base.data() + 5 * (size_t)i, 5 * sizeof(uint64_t));
        std::memcpy(rec + 13 * (size_t)i + 5, marks.data() + 8 * (size_t)i, 8 * sizeof(uint64_t));
    }
    *n = m;
    return SF_OK;
}

sf_status sf_grid_program_plan_trace(sf_handle h, uint64_t* rec, uint32_t cap) {
    if (!h || (cap && !rec)) return fail(h, SF_EINVAL, "NULL argument");
    if (!h->d.gp) return fail(h, SF_EINVAL, "no grid program on this handle (n_qubits > 63)");
    sf_status st = sync_check(h);
    if (st) return st;
    SF_CK(h, sf_gprog_plan_marks(h->d, rec, cap, h->stream));
    SF_CK(h, cudaStreamSynchronize(h->stream));
    return SF_OK;
}

sf_status sf_set_wait_limit(sf_handle h, uint32_t polls) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    h->wait_limit = polls;
    return SF_OK;
}

sf_status sf_set_lowrank(sf_handle h, int32_t on) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    h->d.lowrank = on ? 1 : 0;
    return SF_OK;
}

sf_status sf_lowrank_ranks(sf_handle h, int32_t* ranks) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (!ranks) return fail(h, SF_EINVAL, "ranks is NULL");
    const int n = h->d.n, W = h->d.W;
    const size_t off[3] = {plan_lr_aff(n, W), plan_lr_u(n, W), plan_lr_v(n, W)};
    uint64_t v[3] = {SF_LR_NONE, SF_LR_NONE, SF_LR_NONE};
    if (W >= 8) {
        for (int i = 0; i < 3; i++)
            SF_CK(h, cudaMemcpyAsync(&v[i], h->d.plan + off[i], sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream));
        sf_status st = sync_check(h);
        if (st) return st;
    }
    for (int i = 0; i < 3; i++) ranks[i] = v[i] > SF_LR_MAX ? -1 : (int32_t)v[i];
    return SF_OK;
}

sf_status sf_coalesce(sf_handle h, double drop_eps, uint64_t* out_size) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (!(drop_eps >= 0.0)) return fail(h, SF_EINVAL, "drop_eps must be >= 0");
    sf_status cs = merge_seq(h, drop_eps, h->cur, h->cur ^ 1);
    if (cs) return cs;
    h->cur ^= 1;
    if (out_size) {
        SF_CK(h, cudaMemcpyAsync(h->hk, h->d.kcnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 h->stream));
        sf_status st = sync_check(h);
        if (st) return st;
        *out_size = h->hk[h->cur];
    }
    return SF_OK;
}

// COFACTOR(F, q) (Sec. III): the tableau update and, if q is random, the
// merged split of every element into its two cofactors.  Synchronises (the
// host learns whether q was random).  prob_done (optional): set when the
// cofactor kernel also left the per-CTA probability partials of q.
static sf_status cofactor_q(sf_handle h, uint32_t q, bool* prob_done = nullptr) {
    if (prob_done) *prob_done = false;
    SF_LAUNCH(h, SF_K_MEASURE_PREP, sf_launch_measure_prep(h->d, q, h->cur, h->gws, h->stream));
    SF_CK(h, cudaMemcpyAsync(h->hmeta, h->d.meta, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    // the layout the last grid program left, read in the same round trip
    // (hmeta[3]: its ok word, when no kernel has moved the elements since)
    const bool lay = h->d.W == 1 && h->layout && h->d.gp;
    if (lay)
        SF_CK(h, cudaMemcpyAsync(&h->hmeta[3], &reinterpret_cast<const GpLayout*>(h->d.gp)->ok, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, h->stream));
    sf_status st = sync_check(h);
    if (st) return st;
    if (h->hmeta[2]) {
        if (lay && h->hmeta[3]) {
            // partners by position: no index read or written
            SF_LAUNCH(h, SF_K_COFACTOR, sf_launch_cof_pos(h->d, h->cur, h->cur ^ 1, prob_done != nullptr, h->stream));
            h->cur ^= 1;
            h->idx_ok[h->cur] = false;
            if (prob_done) *prob_done = true;
        } else {
            st = need_index(h, h->cur);
            if (st) return st;
            SF_LAUNCH(h, SF_K_COFACTOR, sf_launch_cof_merge(h->d, h->cur, h->cur ^ 1, h->stream));
            h->cur ^= 1;
            h->idx_ok[h->cur] = sf_emit_index(h->d.W);
        }
    }
    return SF_OK;
}

sf_status sf_apply_toffoli(sf_handle h, uint32_t c1, uint32_t c2, uint32_t t) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (c1 >= h->n || c2 >= h->n || t >= h->n || c1 == c2 || c1 == t || c2 == t)
        return fail(h, SF_EINVAL, "bad Toffoli qubits");
    sf_status st = cofactor_q(h, c1);
    if (!st) st = cofactor_q(h, c2);
    if (st) return st;
    SF_LAUNCH(h, SF_K_COND, sf_launch_cond(h->d, h->cur, 0, (int)c1, (int)c2, (int)t, 0.0, h->stream));
    h->idx_ok[h->cur] = false;  // phase vectors changed
    return SF_OK;
}

sf_status sf_apply_cr_cofactor(sf_handle h, uint32_t c, uint32_t t, double alpha) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (c >= h->n || t >= h->n || c == t) return fail(h, SF_EINVAL, "bad controlled-phase qubits");
    sf_status st = cofactor_q(h, c);
    if (!st) st = cofactor_q(h, t);
    if (st) return st;
    SF_LAUNCH(h, SF_K_COND, sf_launch_cond(h->d, h->cur, 1, (int)c, (int)t, 0, alpha, h->stream));
    return SF_OK;  // phase vectors unchanged: the index stays valid
}

sf_status sf_measure(sf_handle h, uint32_t q, int32_t collapse_to, double* p0, double* p1) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (q >= h->n || collapse_to < -1 || collapse_to > 1) return fail(h, SF_EINVAL, "bad measurement arguments");
    bool prob_done = false;
    sf_status st = cofactor_q(h, q, &prob_done);
    if (st) return st;
    // the probabilities' last CTA (or the positional cofactor's) leaves them in d.out
    if (!prob_done) SF_LAUNCH(h, SF_K_PROB, sf_launch_prob(h->d, h->cur, h->stream));
    SF_CK(h, cudaMemcpyAsync(h->hout, h->d.out, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    st = sync_check(h);
    if (st) return st;
    const double pr[2] = {h->hout[0], h->hout[1]};
    if (p0) *p0 = pr[0];
    if (p1) *p1 = pr[1];
    if (collapse_to >= 0) {
        if (!(pr[collapse_to] > 0.0)) return fail(h, SF_ESTATE, "collapse onto an outcome of probability 0");
        const int in = h->cur, outb = h->cur ^ 1;
        SF_CK(h, cudaMemsetAsync(h->d.kcnt + outb, 0, sizeof(unsigned long long), h->stream));
        SF_LAUNCH(h, SF_K_FILTER, sf_launch_filter(h->d, collapse_to, in, outb, h->stream));
        h->cur ^= 1;
        h->idx_ok[h->cur] = sf_emit_index(h->d.W);
    }
    return SF_OK;
}

sf_status sf_amplitude(sf_handle h, const uint64_t* x_bits, double* re, double* im) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (!x_bits || !re || !im) return fail(h, SF_EINVAL, "NULL argument");
    const int W = h->d.W;
    for (int w = 0; w < W; w++) h->hy[w] = w < h->Wabi ? x_bits[w] : 0ull;
    if (h->n % 64) h->hy[h->Wabi - 1] &= (1ull << (h->n % 64)) - 1ull;
    SF_CK(h, cudaMemcpyAsync(h->dy, h->hy, W * sizeof(uint64_t), cudaMemcpyHostToDevice, h->stream));
    SF_LAUNCH(h, SF_K_AMP_PREP, sf_launch_amp_prep(h->d, h->dy, h->stream));
    SF_LAUNCH(h, SF_K_AMPLITUDE, sf_launch_amplitude(h->d, h->cur, h->stream));  // its last CTA sums
    SF_CK(h, cudaMemcpyAsync(h->hout, h->d.out, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    sf_status st = sync_check(h);
    if (st) return st;
    *re = h->hout[2];
    *im = h->hout[3];
    return SF_OK;
}

sf_status sf_size(sf_handle h, uint64_t* k) {
    if (!h || !k) return fail(h, SF_EINVAL, "NULL argument");
    SF_CK(h, cudaMemcpyAsync(h->hk, h->d.kcnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    sf_status st = sync_check(h);
    if (st) return st;
    *k = h->hk[h->cur];
    return SF_OK;
}

sf_status sf_sync(sf_handle h) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    return sync_check(h);
}

sf_status sf_get_tableau(sf_handle h, uint64_t* x, uint64_t* z, uint32_t* n_xblock) {
    if (!h || !x || !z || !n_xblock) return fail(h, SF_EINVAL, "NULL argument");
    sf_status st = sync_check(h);
    if (st) return st;
    const size_t n = h->n, W = h->d.W;
    std::vector<uint64_t> bx(W * n), bz(W * n);
    int32_t r = 0;
    SF_CK(h, cudaMemcpyAsync(bx.data(), h->d.mx, W * n * 8, cudaMemcpyDeviceToHost, h->stream));
    SF_CK(h, cudaMemcpyAsync(bz.data(), h->d.mz, W * n * 8, cudaMemcpyDeviceToHost, h->stream));
    SF_CK(h, cudaMemcpyAsync(&r, h->d.meta, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    SF_CK(h, cudaStreamSynchronize(h->stream));
    for (size_t row = 0; row < n; row++)
        for (int w = 0; w < h->Wabi; w++) {
            x[row * h->Wabi + w] = bx[w * n + row];
            z[row * h->Wabi + w] = bz[w * n + row];
        }
    *n_xblock = (uint32_t)r;
    return SF_OK;
}

sf_status sf_get_frame(sf_handle h, uint64_t* sigma, double* amp, uint64_t capacity, uint64_t* k) {
    if (!h || !k) return fail(h, SF_EINVAL, "NULL argument");
    uint64_t kk = 0;
    sf_status st = sf_size(h, &kk);
    if (st) return st;
    *k = kk;
    if (kk > capacity) return fail(h, SF_ECAPACITY, "capacity smaller than the frame");
    if (kk == 0) return SF_OK;
    if (!sigma || !amp) return fail(h, SF_EINVAL, "NULL output");
    const int stage = h->cur ^ 1;
    SF_LAUNCH(h, SF_K_EXPORT, sf_launch_export(h->d, h->cur, stage, h->stream));
    h->idx_ok[stage] = false;
    st = sync_check(h);
    if (st) return st;
    const size_t W = h->d.W;
    std::vector<uint64_t> xs(kk * W);
    std::vector<double> xa(2 * kk);
    SF_CK(h, cudaMemcpyAsync(xs.data(), h->d.sig[stage], kk * W * 8, cudaMemcpyDeviceToHost, h->stream));
    SF_CK(h, cudaMemcpyAsync(xa.data(), h->d.amp[stage], kk * 16, cudaMemcpyDeviceToHost, h->stream));
    SF_CK(h, cudaStreamSynchronize(h->stream));
    std::vector<uint64_t> idx(kk);
    std::iota(idx.begin(), idx.end(), 0ull);
    std::sort(idx.begin(), idx.end(), [&](uint64_t a, uint64_t b) {
        for (int w = (int)W - 1; w >= 0; w--) {
            const uint64_t va = xs[a * W + w], vb = xs[b * W + w];
            if (va != vb) return va < vb;
        }
        return false;
    });
    for (uint64_t j = 0; j < kk; j++) {
        const uint64_t s = idx[j];
        for (int w = 0; w < h->Wabi; w++) sigma[j * h->Wabi + w] = xs[s * W + w];
        amp[2 * j] = xa[2 * s];
        amp[2 * j + 1] = xa[2 * s + 1];
    }
    return SF_OK;
}

uint32_t sf_words(sf_handle h) { return h ? (uint32_t)h->Wabi : 0u; }

uint32_t sf_host_state(sf_handle h) {
    if (!h) return 0u;
    return (uint32_t)h->cur | ((uint32_t)h->idx_ok[0] << 1) | ((uint32_t)h->idx_ok[1] << 2) |
           ((uint32_t)h->hull << 3) | ((uint32_t)h->layout << 5);
}

sf_status sf_set_host_state(sf_handle h, uint32_t token) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (token > 63u || ((token >> 3) & 3u) > 2u) return fail(h, SF_EINVAL, "invalid host-state token");
    h->cur = (int)(token & 1u);
    h->idx_ok[0] = (token >> 1) & 1u;
    h->idx_ok[1] = (token >> 2) & 1u;
    h->hull = (int)((token >> 3) & 3u);
    h->layout = (token >> 5) & 1u;
    return SF_OK;
}

uint64_t sf_kernel_launches(sf_handle h) { return h ? h->launches : 0ull; }

sf_status sf_get_internal(sf_handle h, uint64_t* dx, uint64_t* dz, uint32_t* de, double* g) {
    if (!h || !dx || !dz || !de || !g) return fail(h, SF_EINVAL, "NULL argument");
    sf_status st = sync_check(h);
    if (st) return st;
    const size_t n = h->n, W = h->d.W;
    std::vector<uint64_t> bx(W * n), bz(W * n);
    SF_CK(h, cudaMemcpyAsync(bx.data(), h->d.dx, W * n * 8, cudaMemcpyDeviceToHost, h->stream));
    SF_CK(h, cudaMemcpyAsync(bz.data(), h->d.dz, W * n * 8, cudaMemcpyDeviceToHost, h->stream));
    SF_CK(h, cudaMemcpyAsync(de, h->d.de, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    SF_CK(h, cudaMemcpyAsync(g, h->d.g, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SF_CK(h, cudaStreamSynchronize(h->stream));
    for (size_t row = 0; row < n; row++)
        for (int w = 0; w < h->Wabi; w++) {
            dx[row * h->Wabi + w] = bx[w * n + row];
            dz[row * h->Wabi + w] = bz[w * n + row];
        }
    return SF_OK;
}

sf_status sf_time_kernel(sf_handle h, int32_t kernel_id) {
    if (!h) return fail(nullptr, SF_EINVAL, "NULL handle");
    if (kernel_id < -1 || kernel_id >= SF_K_COUNT_CLASSES) return fail(h, SF_EINVAL, "unknown kernel class");
    SF_CK(h, cudaStreamSynchronize(h->stream));
    h->time_id = kernel_id;
    if (kernel_id >= 0) h->ev_used = 0;  // -1 stops recording and keeps the pairs
    return SF_OK;
}

sf_status sf_kernel_time(sf_handle h, double* total_ms, uint64_t* launches) {
    if (!h || !total_ms || !launches) return fail(h, SF_EINVAL, "NULL argument");
    SF_CK(h, cudaStreamSynchronize(h->stream));
    double tot = 0.0;
    for (size_t i = 0; i < h->ev_used; i++) {
        float ms = 0.f;
        SF_CK(h, cudaEventElapsedTime(&ms, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]));
        tot += ms;
    }
    *total_ms = tot;
    *launches = h->ev_used;
    return SF_OK;
}

uint64_t sf_footprint_bytes(uint32_t n_qubits, uint64_t max_elems) {
    if (n_qubits < 1 || n_qubits > SF_MAX_N || max_elems < 1) return 0;
    const uint64_t n = n_qubits, cap = max_elems;
    const uint64_t W = n <= 63 ? 1 : (uint64_t)std::max(2, pow2_at_least((int)((n + 63) / 64)));
    const uint64_t NT = std::max<uint64_t>(32, (n + 31) / 32 * 32);
    uint64_t slots = 1024, icap = 64;
    while (slots < 2 * cap) slots <<= 1;
    while (icap < 2 * cap) icap <<= 1;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t b = 8 * 4 * W * n + 8 * n                 // tableau rows, signs, pivots
                 + 2 * (8 * W + 16) * cap               // two frame buffers
                 + 8 * plan_words((int)n, (int)W)       // plan
                 + (W > 1 ? 4 * slots : 0) + (8 * W + 16) * slots  // slot table
                 + 2 * 8 * (uint64_t)slot_words((int)W) * icap  // phase-vector indexes
                 + 32 * (uint64_t)std::max(1, sms) * 4 + 8 * W + 16 * 256 + 4096;
    const size_t wsb = sf_tableau_smem_bytes((int)n, (int)W, (int)NT);
    if (wsb > 200 * 1024) b += (wsb + 7) / 8 * 8;
    return b;
}

const char* sf_last_error(sf_handle h) {
    if (h) return h->err.c_str();
    std::lock_guard<std::mutex> lk(g_err_mu);
    return g_err.c_str();
}

}  // extern "C"

// ---- multiframes (include/sf_multiframe.h, Sec. IV) ------------------------
// A multiframe is a list of frame handles on one stream.  Every operation runs
// as phases over all frames: each phase enqueues the work of every frame and
// its reads into pinned memory, then synchronises once.  COALESCE of a frame
// runs on the device (export of canonical amplitudes, then k_mf_pair); the host
// groups the pairs by (e, d), copies the owners of each group into a new frame
// with the same tableau (k_mf_gather), rotates it by
// C = CNOT_{v1,v2} ... P^d_{v1} H_{v1} with the frame's own Clifford path, and
// keeps the unpaired elements in the old frame.  Frames whose matrices are
// equal are merged by exporting one and importing it into the other in that
// frame's convention (k_mf_import), then coalescing (Def. 1).
#include <map>

#include "sf_multiframe.cuh"
#include "sf_multiframe.h"

struct sf_multiframe_s {
    uint32_t n = 0;
    uint64_t max_elems = 0;
    uint32_t max_frames = 0;
    cudaStream_t stream = nullptr;
    std::vector<sf_handle> all;     // every frame handle created (owned)
    std::vector<sf_handle> frames;  // the multiframe, in list order
    std::vector<sf_handle> spare;   // handles not in use, reused first
    // one COALESCE round: per frame, its pairs and unpaired elements at the
    // frame's element offset, two counts per frame, and the index lists
    MfPair* dpairs = nullptr;
    uint32_t* dkeep = nullptr;
    uint32_t* dcounts = nullptr;
    uint32_t* didx = nullptr;
    size_t dpairs_cap = 0, dkeep_cap = 0, dcounts_cap = 0, didx_cap = 0;
    // pinned mirrors, and the frames' matrices (2n words per frame)
    MfPair* hpairs = nullptr;
    uint32_t* hkeep = nullptr;
    uint32_t* hcounts = nullptr;
    uint32_t* hidx = nullptr;
    uint64_t* hmat = nullptr;
    size_t hpairs_cap = 0, hkeep_cap = 0, hcounts_cap = 0, hidx_cap = 0, hmat_cap = 0;
    std::string err;
};

namespace {

constexpr int kMfKernelId = 1 << 20;  // multiframe kernels are counted, never timed by class
constexpr double kMfTol = 1e-9;

sf_status mf_fail(sf_multiframe m, sf_status code, const std::string& msg) {
    if (m) m->err = msg;
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_err = msg;
    return code;
}

// a failed call on one of the frames: its message becomes the multiframe's
sf_status mf_from(sf_multiframe m, sf_handle h, sf_status st) {
    if (st != SF_OK) m->err = h ? h->err : std::string(sf_last_error(nullptr));
    return st;
}

#define MF_TRY(m, h, call)                            \
    do {                                              \
        sf_status s_ = (call);                        \
        if (s_ != SF_OK) return mf_from((m), (h), s_); \
    } while (0)

#define MF_CK(m, call)                                                                               \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return mf_fail((m), SF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
sf_status mf_grow_dev(sf_multiframe m, T** p, size_t& cap, size_t need) {
    if (need <= cap) return SF_OK;
    const size_t nc = std::max<size_t>(need, 2 * cap);
    if (*p) cudaFreeAsync(*p, m->stream);
    *p = nullptr;
    cap = 0;
    void* v = nullptr;
    if (cudaMallocAsync(&v, nc * sizeof(T), m->stream) != cudaSuccess)
        return mf_fail(m, SF_ENOMEM, "multiframe scratch allocation failed");
    *p = static_cast<T*>(v);
    cap = nc;
    return SF_OK;
}

template <typename T>
sf_status mf_grow_pin(sf_multiframe m, T** p, size_t& cap, size_t need) {
    if (need <= cap) return SF_OK;
    MF_CK(m, cudaStreamSynchronize(m->stream));  // no copy into the old buffer is in flight
    const size_t nc = std::max<size_t>(need, 2 * cap);
    if (*p) pinned_free(*p, cap);
    *p = nullptr;
    cap = 0;
    if (pinned_alloc_n(p, nc) != cudaSuccess) return mf_fail(m, SF_ENOMEM, "pinned allocation failed");
    cap = nc;
    return SF_OK;
}

sf_status mf_new_frame(sf_multiframe m, sf_handle* out) {
    if (!m->spare.empty()) {
        *out = m->spare.back();
        m->spare.pop_back();
        return SF_OK;
    }
    if (m->all.size() >= m->max_frames) return mf_fail(m, SF_ECAPACITY, "multiframe would exceed max_frames");
    sf_status st = sf_create(m->n, m->max_elems, m->stream, out);
    if (st) return mf_fail(m, st, std::string("frame creation failed: ") + sf_last_error(nullptr));
    m->all.push_back(*out);
    return SF_OK;
}

// the full tableau state of src (matrix, destabilizers, pivots, X-block size,
// global phase) copied into dst; same stream
sf_status mf_copy_tableau(sf_multiframe m, sf_handle dst, sf_handle src) {
    const size_t n = src->n, W = src->d.W;
    cudaStream_t s = m->stream;
    const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
    MF_CK(m, cudaMemcpyAsync(dst->d.mx, src->d.mx, W * n * sizeof(uint64_t), dd, s));
    MF_CK(m, cudaMemcpyAsync(dst->d.mz, src->d.mz, W * n * sizeof(uint64_t), dd, s));
    MF_CK(m, cudaMemcpyAsync(dst->d.dx, src->d.dx, W * n * sizeof(uint64_t), dd, s));
    MF_CK(m, cudaMemcpyAsync(dst->d.dz, src->d.dz, W * n * sizeof(uint64_t), dd, s));
    MF_CK(m, cudaMemcpyAsync(dst->d.de, src->d.de, n * sizeof(uint32_t), dd, s));
    MF_CK(m, cudaMemcpyAsync(dst->d.piv, src->d.piv, n * sizeof(int32_t), dd, s));
    MF_CK(m, cudaMemcpyAsync(dst->d.meta, src->d.meta, 4 * sizeof(int32_t), dd, s));
    MF_CK(m, cudaMemcpyAsync(dst->d.g, src->d.g, sizeof(double2), dd, s));
    return SF_OK;
}

// Enqueue the status read of every frame of fs (with its size, and its matrix
// into m->hmat when `matrices`), synchronise once, then report the first
// device error through that frame's sync_check.  k[i]: size of fs[i].
sf_status mf_read(sf_multiframe m, const std::vector<sf_handle>& fs, std::vector<uint64_t>& k, bool matrices) {
    const size_t n = m->n;
    if (matrices) {
        sf_status st = mf_grow_pin(m, &m->hmat, m->hmat_cap, 2 * n * std::max<size_t>(fs.size(), 1));
        if (st) return st;
    }
    const cudaMemcpyKind d2h = cudaMemcpyDeviceToHost;
    for (size_t i = 0; i < fs.size(); i++) {
        sf_handle F = fs[i];
        MF_CK(m, cudaMemcpyAsync(F->hk, F->d.kcnt, 2 * sizeof(unsigned long long), d2h, m->stream));
        MF_CK(m, cudaMemcpyAsync(F->hstatus, F->d.status, sizeof(uint32_t), d2h, m->stream));
        if (matrices) {
            MF_CK(m, cudaMemcpyAsync(m->hmat + 2 * n * i, F->d.mx, n * sizeof(uint64_t), d2h, m->stream));
            MF_CK(m, cudaMemcpyAsync(m->hmat + 2 * n * i + n, F->d.mz, n * sizeof(uint64_t), d2h, m->stream));
        }
    }
    MF_CK(m, cudaStreamSynchronize(m->stream));
    k.resize(fs.size());
    for (size_t i = 0; i < fs.size(); i++) {
        if (*fs[i]->hstatus) MF_TRY(m, fs[i], sync_check(fs[i]));
        k[i] = fs[i]->hk[fs[i]->cur];
    }
    return SF_OK;
}

// COFACTOR(F, q) of every frame (Sec. III), in two phases: the tableau update
// and the random flag of every frame, one synchronisation, then the merged
// split of the frames where q was random
sf_status mf_cofactor_all(sf_multiframe m, uint32_t q) {
    const cudaMemcpyKind d2h = cudaMemcpyDeviceToHost;
    for (sf_handle F : m->frames) {
        MF_TRY(m, F, launch(F, SF_K_MEASURE_PREP, "measure_prep",
                            [&] { sf_launch_measure_prep(F->d, q, F->cur, F->gws, m->stream); }));
        MF_CK(m, cudaMemcpyAsync(F->hmeta, F->d.meta, 4 * sizeof(int32_t), d2h, m->stream));
        MF_CK(m, cudaMemcpyAsync(F->hstatus, F->d.status, sizeof(uint32_t), d2h, m->stream));
    }
    MF_CK(m, cudaStreamSynchronize(m->stream));
    for (sf_handle F : m->frames) {
        if (*F->hstatus) MF_TRY(m, F, sync_check(F));
        if (!F->hmeta[2]) continue;
        MF_TRY(m, F, need_index(F, F->cur));
        MF_TRY(m, F, launch(F, SF_K_COFACTOR, "cof_merge",
                            [&] { sf_launch_cof_merge(F->d, F->cur, F->cur ^ 1, m->stream); }));
        F->cur ^= 1;
        F->idx_ok[F->cur] = sf_emit_index(F->d.W);
    }
    return SF_OK;
}

// Def. 1 coalescing of every frame (asynchronous)
sf_status mf_coalesce_frames(sf_multiframe m, double eps) {
    for (sf_handle F : m->frames) {
        MF_TRY(m, F, merge_seq(F, eps, F->cur, F->cur ^ 1));
        F->cur ^= 1;
    }
    return SF_OK;
}

// A16: frames with equal matrices merged into the first of them (union, then
// Def. 1 coalescing with eps); empty frames leave the list
sf_status mf_merge(sf_multiframe m, double eps) {
    std::vector<uint64_t> k;
    sf_status st = mf_read(m, m->frames, k, true);
    if (st) return st;
    const size_t n = m->n;
    std::map<std::vector<uint64_t>, size_t> first;
    std::vector<std::vector<size_t>> groups;
    for (size_t i = 0; i < m->frames.size(); i++) {
        std::vector<uint64_t> key(m->hmat + 2 * n * i, m->hmat + 2 * n * (i + 1));
        auto it = first.find(key);
        if (it == first.end()) {
            first.emplace(std::move(key), groups.size());
            groups.push_back({i});
        } else {
            groups[it->second].push_back(i);
        }
    }
    std::vector<sf_handle> out, merged;
    for (const auto& g : groups) {
        sf_handle dst = m->frames[g[0]];
        if (g.size() == 1) {
            (k[g[0]] ? out : m->spare).push_back(dst);
            continue;
        }
        uint64_t kd = k[g[0]];
        for (size_t i = 1; i < g.size(); i++) {
            sf_handle src = m->frames[g[i]];
            const uint64_t ks = k[g[i]];
            if (!st && kd + ks > m->max_elems) st = mf_fail(m, SF_ECAPACITY, "merged frame would exceed max_elems");
            if (!st && ks) {
                const int stage = src->cur ^ 1;
                st = mf_from(m, src, launch(src, kMfKernelId, "export",
                                            [&] { sf_launch_export(src->d, src->cur, stage, m->stream); }));
                src->idx_ok[stage] = false;
                const uint64_t off = kd;
                if (!st)
                    st = mf_from(m, dst, launch(dst, kMfKernelId, "k_mf_import", [&] {
                                     sf_launch_mf_import(dst->d, dst->cur, off, src->d.sig[stage], src->d.amp[stage],
                                                         (uint32_t)ks, m->stream);
                                 }));
                dst->idx_ok[0] = dst->idx_ok[1] = false;
                kd += ks;
            }
            if (st) out.push_back(src);  // after an error every handle stays reachable
            else m->spare.push_back(src);
        }
        if (!st) {
            st = mf_from(m, dst, merge_seq(dst, eps, dst->cur, dst->cur ^ 1));
            dst->cur ^= 1;
        }
        out.push_back(dst);
        merged.push_back(dst);
    }
    m->frames.swap(out);
    if (st || merged.empty()) return st;
    // frames emptied by the drop threshold leave the list
    st = mf_read(m, merged, k, false);
    if (st) return st;
    std::vector<sf_handle> kept;
    for (sf_handle F : m->frames) {
        const auto it = std::find(merged.begin(), merged.end(), F);
        if (it != merged.end() && k[it - merged.begin()] == 0) m->spare.push_back(F);
        else kept.push_back(F);
    }
    m->frames.swap(kept);
    return SF_OK;
}

// One round of COALESCE over every frame; `formed`: the pairs found
sf_status mf_coalesce_round(sf_multiframe m, uint64_t& formed) {
    formed = 0;
    std::vector<uint64_t> k;
    sf_status st = mf_read(m, m->frames, k, true);
    if (st) return st;
    const size_t nf = m->frames.size(), n = m->n;
    std::vector<size_t> part, off(nf, 0);
    size_t total = 0;
    for (size_t i = 0; i < nf; i++) {
        if (k[i] < 2) continue;
        if (k[i] > SF_MF_MAXK) return mf_fail(m, SF_ECAPACITY, "COALESCE takes frames of at most 8192 elements");
        part.push_back(i);
        off[i] = total;
        total += k[i];
    }
    if (part.empty()) return SF_OK;
    if ((st = mf_grow_dev(m, &m->dpairs, m->dpairs_cap, total)) || (st = mf_grow_dev(m, &m->dkeep, m->dkeep_cap, total)) ||
        (st = mf_grow_dev(m, &m->dcounts, m->dcounts_cap, 2 * part.size())) ||
        (st = mf_grow_dev(m, &m->didx, m->didx_cap, total)) ||
        (st = mf_grow_pin(m, &m->hpairs, m->hpairs_cap, total)) || (st = mf_grow_pin(m, &m->hkeep, m->hkeep_cap, total)) ||
        (st = mf_grow_pin(m, &m->hcounts, m->hcounts_cap, 2 * part.size())) ||
        (st = mf_grow_pin(m, &m->hidx, m->hidx_cap, total)))
        return st;
    // phase 1: export and pairing of every frame of two or more elements
    for (size_t j = 0; j < part.size(); j++) {
        sf_handle F = m->frames[part[j]];
        const int stage = F->cur ^ 1;
        const uint64_t kk = k[part[j]], o = off[part[j]];
        MF_TRY(m, F, launch(F, kMfKernelId, "export", [&] { sf_launch_export(F->d, F->cur, stage, m->stream); }));
        F->idx_ok[stage] = false;
        MF_TRY(m, F, launch(F, kMfKernelId, "k_mf_pair", [&] {
                   sf_launch_mf_pair(F->d, F->cur, stage, kk, kMfTol, m->dpairs + o, m->dkeep + o, m->dcounts + 2 * j,
                                     m->stream);
               }));
    }
    MF_CK(m, cudaMemcpyAsync(m->hcounts, m->dcounts, 2 * part.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                             m->stream));
    std::vector<sf_handle> chk;
    for (size_t i : part) chk.push_back(m->frames[i]);
    if ((st = mf_read(m, chk, k, false))) return st;  // statuses of the pairing; sizes unchanged
    // phase 2: the pairs and unpaired elements of the frames that formed pairs
    std::vector<size_t> paired;
    for (size_t j = 0; j < part.size(); j++) {
        const uint32_t np = m->hcounts[2 * j], nk = m->hcounts[2 * j + 1];
        if (2ull * np + nk != k[j]) return mf_fail(m, SF_EINTERNAL, "COALESCE lost elements");
        if (!np) continue;
        formed += np;
        paired.push_back(j);
        const uint64_t o = off[part[j]];
        MF_CK(m, cudaMemcpyAsync(m->hpairs + o, m->dpairs + o, np * sizeof(MfPair), cudaMemcpyDeviceToHost, m->stream));
        if (nk)
            MF_CK(m, cudaMemcpyAsync(m->hkeep + o, m->dkeep + o, nk * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                     m->stream));
    }
    if (paired.empty()) return SF_OK;
    MF_CK(m, cudaStreamSynchronize(m->stream));
    // per frame: owners of each class (e, d) in ascending order, then the unpaired
    std::vector<std::map<std::pair<uint64_t, uint32_t>, std::vector<uint32_t>>> cls(paired.size());
    for (size_t pi = 0; pi < paired.size(); pi++) {
        const size_t j = paired[pi];
        const uint64_t o = off[part[j]];
        const uint32_t np = m->hcounts[2 * j], nk = m->hcounts[2 * j + 1];
        for (uint32_t t = 0; t < np; t++) cls[pi][{m->hpairs[o + t].e, m->hpairs[o + t].d}].push_back(m->hpairs[o + t].owner);
        uint64_t w = o;
        for (const auto& c : cls[pi])
            for (uint32_t x : c.second) m->hidx[w++] = x;
        for (uint32_t t = 0; t < nk; t++) m->hidx[w++] = m->hkeep[o + t];
    }
    MF_CK(m, cudaMemcpyAsync(m->didx, m->hidx, total * sizeof(uint32_t), cudaMemcpyHostToDevice, m->stream));
    // phase 3: new frames from the classes, unpaired elements kept in place
    std::vector<std::vector<sf_handle>> made(nf);
    std::vector<char> gone(nf, 0);
    for (size_t pi = 0; pi < paired.size() && !st; pi++) {
        const size_t j = paired[pi], fi = part[j];
        sf_handle F = m->frames[fi];
        const uint64_t o = off[fi];
        const uint32_t nk = m->hcounts[2 * j + 1];
        const uint64_t* mz = m->hmat + 2 * n * fi + n;
        uint64_t pos = o;
        for (const auto& c : cls[pi]) {
            sf_handle G = nullptr;
            if ((st = mf_new_frame(m, &G))) break;
            made[fi].push_back(G);
            if ((st = mf_copy_tableau(m, G, F))) break;
            const uint32_t cnt = (uint32_t)c.second.size();
            const uint32_t* ix = m->didx + pos;
            st = mf_from(m, G, launch(G, kMfKernelId, "k_mf_gather", [&] {
                             sf_launch_mf_gather(G->d, G->cur, F->d.sig[F->cur], F->d.amp[F->cur], ix, cnt,
                                                 std::sqrt(2.0), m->stream);
                         }));
            if (st) break;
            G->idx_ok[0] = G->idx_ok[1] = false;
            pos += cnt;
            // the qubits v_1 < ... < v_m of the Z_k-rows in e
            std::vector<uint32_t> V;
            for (uint64_t e = c.first.first; e; e &= e - 1) V.push_back((uint32_t)__builtin_ctzll(mz[__builtin_ctzll(e)]));
            std::sort(V.begin(), V.end());
            std::vector<sf_gate> gates;
            gates.push_back(sf_gate{SF_H, V[0], 0, 0});
            for (uint32_t t = 0; t < c.first.second; t++) gates.push_back(sf_gate{SF_S, V[0], 0, 0});
            for (size_t i = 1; i < V.size(); i++) gates.push_back(sf_gate{SF_CNOT, V[0], V[i], 0});
            if ((st = mf_from(m, G, sf_apply_clifford(G, gates.data(), gates.size())))) break;
        }
        if (st) break;
        if (nk) {
            const uint32_t* ix = m->didx + pos;
            st = mf_from(m, F, launch(F, kMfKernelId, "k_mf_gather", [&] {
                             sf_launch_mf_gather(F->d, F->cur ^ 1, F->d.sig[F->cur], F->d.amp[F->cur], ix, nk, 1.0,
                                                 m->stream);
                         }));
            F->cur ^= 1;
            F->idx_ok[0] = F->idx_ok[1] = false;
        } else {
            gone[fi] = 1;
        }
    }
    // the list in order: each frame (unless all its elements paired), then its new frames
    std::vector<sf_handle> out;
    for (size_t i = 0; i < nf; i++) {
        (gone[i] && !st ? m->spare : out).push_back(m->frames[i]);
        out.insert(out.end(), made[i].begin(), made[i].end());
    }
    m->frames.swap(out);
    return st;
}

// merge, then COALESCE every frame and merge again until no pair forms
sf_status mf_coalesce_all(sf_multiframe m, double eps) {
    sf_status st = mf_merge(m, eps);
    for (int iter = 0; !st; iter++) {
        if (iter > (1 << 20)) return mf_fail(m, SF_EINTERNAL, "multiframe coalescing did not terminate");
        uint64_t formed = 0;
        st = mf_coalesce_round(m, formed);
        if (st || formed == 0) break;
        st = mf_merge(m, eps);
    }
    return st;
}

sf_status mf_check_qubits(sf_multiframe m, std::initializer_list<uint32_t> qs) {
    std::vector<uint32_t> v(qs);
    for (size_t i = 0; i < v.size(); i++) {
        if (v[i] >= m->n) return mf_fail(m, SF_EINVAL, "qubit out of range");
        for (size_t j = 0; j < i; j++)
            if (v[i] == v[j]) return mf_fail(m, SF_EINVAL, "repeated qubit");
    }
    return SF_OK;
}

}  // namespace

extern "C" {

sf_status sf_mf_create(uint32_t n_qubits, uint64_t max_elems, uint32_t max_frames, void* cuda_stream,
                       sf_multiframe* out) {
    if (!out) return mf_fail(nullptr, SF_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 63) return mf_fail(nullptr, SF_EINVAL, "multiframes take 1 to 63 qubits");
    if (max_frames < 1) return mf_fail(nullptr, SF_EINVAL, "max_frames must be >= 1");
    sf_multiframe m = new (std::nothrow) sf_multiframe_s();
    if (!m) return mf_fail(nullptr, SF_ENOMEM, "host allocation failed");
    m->n = n_qubits;
    m->max_elems = max_elems;
    m->max_frames = max_frames;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    sf_handle F = nullptr;
    sf_status st = mf_new_frame(m, &F);
    if (st) {
        const std::string msg = m->err;
        sf_mf_destroy(m);
        return mf_fail(nullptr, st, msg);
    }
    m->frames.push_back(F);
    *out = m;
    return SF_OK;
}

sf_status sf_mf_destroy(sf_multiframe m) {
    if (!m) return mf_fail(nullptr, SF_EINVAL, "NULL multiframe");
    for (sf_handle h : m->all) sf_destroy(h);
    for (void* p : {(void*)m->dpairs, (void*)m->dkeep, (void*)m->dcounts, (void*)m->didx})
        if (p) cudaFreeAsync(p, m->stream);
    cudaStreamSynchronize(m->stream);
    pinned_free(m->hpairs, m->hpairs_cap);
    pinned_free(m->hkeep, m->hkeep_cap);
    pinned_free(m->hcounts, m->hcounts_cap);
    pinned_free(m->hidx, m->hidx_cap);
    pinned_free(m->hmat, m->hmat_cap);
    delete m;
    return SF_OK;
}

sf_status sf_mf_apply_clifford(sf_multiframe m, const sf_gate* gates, uint64_t n_gates) {
    if (!m) return mf_fail(nullptr, SF_EINVAL, "NULL multiframe");
    for (sf_handle F : m->frames) MF_TRY(m, F, sf_apply_clifford(F, gates, n_gates));
    return SF_OK;
}

sf_status sf_mf_apply_nonclifford(sf_multiframe m, uint32_t kind, uint32_t q0, uint32_t q1, double theta,
                                  double drop_eps) {
    if (!m) return mf_fail(nullptr, SF_EINVAL, "NULL multiframe");
    for (sf_handle F : m->frames)
        MF_TRY(m, F, sf_apply_nonclifford_coalesce(F, kind, q0, q1, theta, drop_eps));
    std::vector<uint64_t> k;
    sf_status st = mf_read(m, m->frames, k, false);
    if (st) return st;
    std::vector<sf_handle> kept;
    for (size_t i = 0; i < m->frames.size(); i++) (k[i] ? kept : m->spare).push_back(m->frames[i]);
    m->frames.swap(kept);
    return SF_OK;
}

sf_status sf_mf_apply_toffoli(sf_multiframe m, uint32_t c1, uint32_t c2, uint32_t t, double drop_eps) {
    if (!m) return mf_fail(nullptr, SF_EINVAL, "NULL multiframe");
    if (!(drop_eps >= 0.0)) return mf_fail(m, SF_EINVAL, "drop_eps must be >= 0");
    sf_status st = mf_check_qubits(m, {c1, c2, t});
    if (!st) st = mf_cofactor_all(m, c1);
    if (!st) st = mf_cofactor_all(m, c2);
    if (st) return st;
    for (sf_handle F : m->frames) {
        MF_TRY(m, F, launch(F, SF_K_COND, "cond", [&] {
                   sf_launch_cond(F->d, F->cur, 0, (int)c1, (int)c2, (int)t, 0.0, m->stream);
               }));
        F->idx_ok[F->cur] = false;  // phase vectors changed
    }
    if ((st = mf_coalesce_frames(m, drop_eps))) return st;
    return mf_coalesce_all(m, drop_eps);
}

sf_status sf_mf_apply_cr(sf_multiframe m, uint32_t c, uint32_t t, double alpha, double drop_eps) {
    if (!m) return mf_fail(nullptr, SF_EINVAL, "NULL multiframe");
    if (!(drop_eps >= 0.0)) return mf_fail(m, SF_EINVAL, "drop_eps must be >= 0");
    sf_status st = mf_check_qubits(m, {c, t});
    if (!st) st = mf_cofactor_all(m, c);
    if (!st) st = mf_cofactor_all(m, t);
    if (st) return st;
    for (sf_handle F : m->frames)
        MF_TRY(m, F, launch(F, SF_K_COND, "cond", [&] {
                   sf_launch_cond(F->d, F->cur, 1, (int)c, (int)t, 0, alpha, m->stream);
               }));
    if ((st = mf_coalesce_frames(m, drop_eps))) return st;
    return mf_coalesce_all(m, drop_eps);
}

sf_status sf_mf_count(sf_multiframe m, uint32_t* n_frames, uint64_t* n_states) {
    if (!m) return mf_fail(nullptr, SF_EINVAL, "NULL multiframe");
    std::vector<uint64_t> k;
    sf_status st = mf_read(m, m->frames, k, false);
    if (st) return st;
    uint64_t tot = 0;
    for (uint64_t v : k) tot += v;
    if (n_frames) *n_frames = (uint32_t)m->frames.size();
    if (n_states) *n_states = tot;
    return SF_OK;
}

sf_status sf_mf_coalesce(sf_multiframe m, double drop_eps, uint32_t* n_frames, uint64_t* n_states) {
    if (!m) return mf_fail(nullptr, SF_EINVAL, "NULL multiframe");
    if (!(drop_eps >= 0.0)) return mf_fail(m, SF_EINVAL, "drop_eps must be >= 0");
    sf_status st = mf_coalesce_all(m, drop_eps);
    if (st) return st;
    return sf_mf_count(m, n_frames, n_states);
}

// <x|Psi>: the amplitude kernels of every frame, one synchronisation, the sum
sf_status sf_mf_amplitude(sf_multiframe m, const uint64_t* x_bits, double* re, double* im) {
    if (!m) return mf_fail(nullptr, SF_EINVAL, "NULL multiframe");
    if (!x_bits || !re || !im) return mf_fail(m, SF_EINVAL, "NULL argument");
    const uint64_t x = m->n == 64 ? x_bits[0] : x_bits[0] & ((1ull << m->n) - 1ull);
    for (sf_handle F : m->frames) {
        F->hy[0] = x;
        MF_CK(m, cudaMemcpyAsync(F->dy, F->hy, sizeof(uint64_t), cudaMemcpyHostToDevice, m->stream));
        MF_TRY(m, F, launch(F, SF_K_AMP_PREP, "amp_prep", [&] { sf_launch_amp_prep(F->d, F->dy, m->stream); }));
        MF_TRY(m, F, launch(F, SF_K_AMPLITUDE, "amplitude", [&] { sf_launch_amplitude(F->d, F->cur, m->stream); }));
        MF_CK(m, cudaMemcpyAsync(F->hout, F->d.out, 4 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    }
    std::vector<uint64_t> k;
    sf_status st = mf_read(m, m->frames, k, false);  // synchronises, reports device errors
    if (st) return st;
    double sr = 0.0, si = 0.0;
    for (sf_handle F : m->frames) {
        sr += F->hout[2];
        si += F->hout[3];
    }
    *re = sr;
    *im = si;
    return SF_OK;
}

sf_status sf_mf_frame(sf_multiframe m, uint32_t i, sf_handle* out) {
    if (!m || !out) return mf_fail(m, SF_EINVAL, "NULL argument");
    if (i >= m->frames.size()) return mf_fail(m, SF_EINVAL, "frame index out of range");
    *out = m->frames[i];
    return SF_OK;
}

uint64_t sf_mf_launches(sf_multiframe m) {
    uint64_t t = 0;
    if (m)
        for (sf_handle h : m->all) t += h->launches;
    return t;
}

const char* sf_mf_last_error(sf_multiframe m) {
    if (m) return m->err.c_str();
    std::lock_guard<std::mutex> lk(g_err_mu);
    return g_err.c_str();
}

}  // extern "C"
