// sf_noalloc.cu -- sf_coalesce_noalloc: coalescing of caller-owned device
// buffers with no allocation at all.
//
// Who needs it: callers that must not allocate device memory where they merge
// a frame.  A framework that owns the device memory through its own caching
// pool leaves little free memory outside that pool, so an extra cudaMalloc
// behind its back may fail, and cudaMalloc/cudaFree can synchronise the
// device; a serving loop that budgets all device memory up front must not
// fail half way through a request on an allocation.  The caller passes the
// input and output arrays; the hash table, the representative indices and the
// amplitude accumulators live in one file-scope __device__ array of fixed
// size, so the number of input elements is capped.
//
// The scratch array is shared by every call on a device and keeps the
// previous call's contents: each call clears what it relies on before use.
// Calls whose kernels overlap on the GPU (two streams, or two host threads)
// race on the scratch; callers must order them.
//
// Output order: each group of equal phase vectors is represented by its first
// input element (the smallest index, found with atomicMin after the slots are
// claimed), and representatives are written in input order.  The amplitudes of
// a group are summed with atomics, in an order that depends on scheduling, so
// two calls on the same input may differ in the last bits of a merged sum.
#include <mutex>

#include "sf.h"
#include "sf_device.cuh"

namespace {

constexpr uint32_t kNaMax = SF_COALESCE_NOALLOC_MAX_ELEMS;  // elements per call
constexpr int SF_NOALLOC_MAX_DEVICES = 64;
constexpr uint32_t kNaSlots = 2 * kNaMax;                   // hash slots (power of two)
constexpr uint32_t kEmptySlot = 0xffffffffu;
constexpr int kNaThreads = 256;
constexpr int kNaBlocks = 128;

// layout of the scratch array, in 32-bit words:
//   [0, kNaSlots)                      hash slots
//   [kNaSlots, kNaSlots + kNaMax)      representative of each input element
//   then kNaMax double2 accumulators (16-byte aligned), then 4 control words
constexpr size_t kOffRep = kNaSlots;
constexpr size_t kOffAcc = kOffRep + kNaMax;  // multiple of 4 words -> 16-byte aligned
constexpr size_t kOffCtl = kOffAcc + 4 * (size_t)kNaMax;
constexpr size_t kScratchWords = kOffCtl + 8;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

struct NaPtrs {
    uint32_t* slots;
    uint32_t* rep;
    double2* acc;
    unsigned long long* kout;  // output count
    uint32_t* flag;            // probe-limit flag
};

__device__ __forceinline__ NaPtrs na_ptrs(uint32_t* base) {
    NaPtrs p;
    p.slots = base;
    p.rep = base + kOffRep;
    p.acc = reinterpret_cast<double2*>(base + kOffAcc);
    p.kout = reinterpret_cast<unsigned long long*>(base + kOffCtl);
    p.flag = base + kOffCtl + 2;
    return p;
}

__device__ __forceinline__ uint32_t table_slots(uint64_t k) {
    uint32_t t = 1024;
    while (t < 2 * k && t < kNaSlots) t <<= 1;
    return t;
}

__device__ __forceinline__ uint64_t na_hash(const uint64_t* s, int nw) {
    uint64_t h = 0x243F6A8885A308D3ull;
    for (int w = 0; w < nw; w++) {
        uint64_t v = s[w] ^ h;
        v ^= v >> 33;
        v *= 0xFF51AFD7ED558CCDull;
        v ^= v >> 33;
        v *= 0xC4CEB9FE1A85EC53ull;
        v ^= v >> 33;
        h = v + (uint64_t)w;
    }
    return h;
}

// clear the table part this call uses, load the accumulators, zero the controls
__global__ void k_na_init(uint32_t* base, const double2* amp_in, uint64_t k) {
    const NaPtrs p = na_ptrs(base);
    const uint32_t T = table_slots(k);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < T; i += stride) p.slots[i] = kEmptySlot;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < k; j += stride) p.acc[j] = amp_in[j];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *p.kout = 0;
        *p.flag = 0;
    }
}

// find or claim the slot of each phase vector; the slot ends up holding the
// smallest input index of its group, and rep[j] the slot of element j
__global__ void k_na_insert(uint32_t* base, const uint64_t* sig_in, uint64_t k, int nw) {
    const NaPtrs p = na_ptrs(base);
    const uint32_t T = table_slots(k);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < k; j += stride) {
        uint64_t s[SF_MAX_W];
        for (int w = 0; w < nw; w++) s[w] = sig_in[j * nw + w];
        uint32_t slot = (uint32_t)(na_hash(s, nw) & (T - 1));
        uint32_t found = kEmptySlot;
        for (uint32_t probe = 0; probe < T; probe++) {
            uint32_t cur = p.slots[slot];
            if (cur == kEmptySlot) {
                cur = atomicCAS(&p.slots[slot], kEmptySlot, (uint32_t)j);
                if (cur == kEmptySlot) { found = slot; break; }
            }
            // any member of a group has the group's phase vector, so the slot
            // may be lowered by atomicMin while others compare against it
            bool eq = true;
            for (int w = 0; w < nw; w++) eq &= (sig_in[(uint64_t)cur * nw + w] == s[w]);
            if (eq) { found = slot; break; }
            slot = (slot + 1) & (T - 1);
        }
        if (found == kEmptySlot) {
            atomicExch(p.flag, 1u);  // table full: cannot happen with 2k slots, reported if it does
        } else {
            atomicMin(&p.slots[found], (uint32_t)j);
        }
        p.rep[j] = found;
    }
}

// representative of each element (its group's smallest index); the others add
// their amplitude to it
__global__ void k_na_link(uint32_t* base, const double2* amp_in, uint64_t k) {
    const NaPtrs p = na_ptrs(base);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < k; j += stride) {
        const uint32_t slot = p.rep[j];
        const uint32_t rep = slot == kEmptySlot ? (uint32_t)j : p.slots[slot];
        p.rep[j] = rep;
        if (rep != (uint32_t)j) {
            const double2 a = amp_in[j];
            atomicAdd(&p.acc[rep].x, a.x);
            atomicAdd(&p.acc[rep].y, a.y);
        }
    }
}

// one CTA: keep representatives with |a| >= eps in input order
__global__ void __launch_bounds__(1024) k_na_compact(uint32_t* base, const uint64_t* sig_in, uint64_t k, int nw,
                                                     double eps2, uint64_t* sig_out, double2* amp_out) {
    __shared__ int wsum[32];
    __shared__ unsigned long long total;
    const NaPtrs p = na_ptrs(base);
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nwarp = blockDim.x >> 5;
    if (t == 0) total = 0;
    __syncthreads();
    for (uint64_t t0 = 0; t0 < k; t0 += blockDim.x) {
        const uint64_t j = t0 + t;
        bool keep = false;
        double2 a = make_double2(0.0, 0.0);
        if (j < k && p.rep[j] == (uint32_t)j) {
            a = p.acc[j];
            keep = a.x * a.x + a.y * a.y >= eps2;
        }
        const unsigned bal = __ballot_sync(SF_FULL, keep);
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        unsigned long long off = total;
        for (int i = 0; i < wid; i++) off += wsum[i];
        if (keep) {
            const unsigned long long o = off + __popc(bal & ((1u << lane) - 1u));
            for (int w = 0; w < nw; w++) sig_out[o * nw + w] = sig_in[j * nw + w];
            amp_out[o] = a;
        }
        __syncthreads();
        if (t == 0) {
            unsigned long long s = 0;
            for (int i = 0; i < nwarp; i++) s += wsum[i];
            total += s;
        }
        __syncthreads();
    }
    if (t == 0) *p.kout = total;
}

std::mutex g_na_mu;
uint32_t* g_na_addr[SF_NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array for the current device, looked up once
// per device with that device current (the symbol's host-side name is not a
// device address).  The address belongs to the device's primary context, so a
// process that resets the device (cudaDeviceReset) must not call
// sf_coalesce_noalloc on it afterwards.
sf_status na_scratch(uint32_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SF_NOALLOC_MAX_DEVICES) return SF_ECUDA;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SF_ECUDA;
        g_na_addr[dev] = static_cast<uint32_t*>(ptr);
    }
    *out = g_na_addr[dev];
    return SF_OK;
}

}  // namespace

extern "C" sf_status sf_coalesce_noalloc(const uint64_t* sigma_in, const double* amp_in, uint64_t k_in,
                                         uint32_t n_words, double drop_eps, uint64_t* sigma_out, double* amp_out,
                                         uint64_t* k_out, void* cuda_stream) {
    if (!k_out) return SF_EINVAL;
    *k_out = 0;
    if (k_in > kNaMax || n_words < 1 || n_words > SF_MAX_W || !(drop_eps >= 0.0)) return SF_EINVAL;
    if (k_in == 0) return SF_OK;
    if (!sigma_in || !amp_in || !sigma_out || !amp_out) return SF_EINVAL;
    uint32_t* base = nullptr;
    sf_status st = na_scratch(&base);
    if (st != SF_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const double2* ain = reinterpret_cast<const double2*>(amp_in);
    k_na_init<<<kNaBlocks, kNaThreads, 0, s>>>(base, ain, k_in);
    k_na_insert<<<kNaBlocks, kNaThreads, 0, s>>>(base, sigma_in, k_in, (int)n_words);
    k_na_link<<<kNaBlocks, kNaThreads, 0, s>>>(base, ain, k_in);
    k_na_compact<<<1, 1024, 0, s>>>(base, sigma_in, k_in, (int)n_words, drop_eps * drop_eps, sigma_out,
                                    reinterpret_cast<double2*>(amp_out));
    if (cudaGetLastError() != cudaSuccess) return SF_ECUDA;
    unsigned long long ctl[2] = {0, 0};
    if (cudaMemcpyAsync(ctl, base + kOffCtl, sizeof(ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SF_ECUDA;
    if (ctl[1] & 0xffffffffull) return SF_ETIMEOUT;
    *k_out = ctl[0];
    return SF_OK;
}
