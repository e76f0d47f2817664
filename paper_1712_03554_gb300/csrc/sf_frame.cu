// sf_frame.cu -- kernels that stream over the frame elements (phase vectors
// sigma, word-major [W][cap], and FP64 complex amplitudes):
//   k_affine      per-element Clifford update sigma' = A sigma ^ t (Sec. III,
//                 ROTATE: the memoised row operations of Invariant 1 applied
//                 to every phase vector), 4-bit table lookups in shared memory
//   k_branch      diagonal non-Clifford branching (Sec. IV)
//   k_coal_*      COALESCE in the set sense of Def. 1: hash equal phase
//                 vectors, segmented amplitude sum, drop |a| < eps, stable
//                 stream compaction
//   k_cof_split   cofactor children of every element (COFACTOR, Sec. III)
//   k_prob        measurement probabilities (Sec. IV, measuring F)
//   k_amplitude   <y|Psi> (Observation 1)
//   k_export      canonical-convention amplitudes for export
// Per-element kernels use a fixed grid of d.nblk CTAs and read the element
// count from device memory, so no host synchronisation is needed between them.
#include "sf_device.cuh"

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kEmpty = 0xffffffffu;

__device__ __forceinline__ unsigned long long table_size(unsigned long long k, unsigned long long cap) {
    unsigned long long t = 1024;
    while (t < 2 * k && t < cap) t <<= 1;
    return t < cap ? t : cap;
}

// splitmix64 finaliser chained over the words
template <int W>
__device__ __forceinline__ uint64_t hash_sig(const uint64_t* s) {
    uint64_t h = 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int w = 0; w < W; w++) {
        uint64_t v = s[w] + h;
        v ^= v >> 30;
        v *= 0xBF58476D1CE4E5B9ull;
        v ^= v >> 27;
        v *= 0x94D049BB133111EBull;
        v ^= v >> 31;
        h = v + 0x9E3779B97F4A7C15ull * (uint64_t)(w + 1);
    }
    return h;
}

template <int W>
__device__ __forceinline__ void load_sig(const uint64_t* S, uint64_t cap, unsigned long long j, uint64_t* s) {
#pragma unroll
    for (int w = 0; w < W; w++) s[w] = S[(size_t)w * cap + j];
}
template <int W>
__device__ __forceinline__ void store_sig(uint64_t* S, uint64_t cap, unsigned long long j, const uint64_t* s) {
#pragma unroll
    for (int w = 0; w < W; w++) S[(size_t)w * cap + j] = s[w];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(SF_FULL, v, o);
    return v;
}

// block-wide sum of NV doubles; result valid in thread 0
template <int NV>
__device__ void block_sum(double* v, double (*sh)[32]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int c = 0; c < NV; c++) v[c] = warp_sum(v[c]);
    if (lane == 0)
        for (int c = 0; c < NV; c++) sh[c][wid] = v[c];
    __syncthreads();
    if (wid == 0) {
        for (int c = 0; c < NV; c++) {
            double t = lane < nw ? sh[c][lane] : 0.0;
            v[c] = warp_sum(t);
        }
    }
}

// element range of this CTA for chunked (order-preserving) passes
__device__ __forceinline__ void chunk_range(unsigned long long k, int nblk, unsigned long long& lo,
                                            unsigned long long& hi) {
    const unsigned long long ch = (k + nblk - 1) / nblk;
    lo = min(k, ch * blockIdx.x);
    hi = min(k, lo + ch);
}

// ---- per-element amplitude of D^sigma phi_0(M) ------------------------------
// <y| D^sigma phi_0(M)> * 2^{r/2} as an i-power, or -1 if zero.
template <int W>
__device__ int elem_amp_phi(const SfDev& d, const uint64_t* s, const uint64_t* y, int r) {
    const int n = d.n;
    Pauli<W> q;
    pauli_id<W>(q);
#pragma unroll
    for (int w = 0; w < W; w++) {
        uint64_t bits = s[w];
        while (bits) {
            const int b = __ffsll((long long)bits) - 1;
            bits &= bits - 1;
            const int h = 64 * w + b;
            Pauli<W> dh;
#pragma unroll
            for (int u = 0; u < W; u++) { dh.x[u] = __ldg(&d.dx[u * n + h]); dh.z[u] = __ldg(&d.dz[u * n + h]); }
            dh.e = (int)__ldg(&d.de[h]);
            pauli_mul<W>(q, dh);
        }
    }
    uint64_t wv[W];
#pragma unroll
    for (int w = 0; w < W; w++) wv[w] = y[w] ^ q.x[w];
    Pauli<W> p;
    pauli_id<W>(p);
    for (int R = 0; R < r; R++) {
        const int pv = __ldg(&d.piv[R]);
        if ((wv[pv >> 6] >> (pv & 63)) & 1) {
            Pauli<W> m;
#pragma unroll
            for (int u = 0; u < W; u++) { m.x[u] = __ldg(&d.mx[u * n + R]); m.z[u] = __ldg(&d.mz[u * n + R]); }
            m.e = 0;
            pauli_mul<W>(p, m);
        }
    }
#pragma unroll
    for (int w = 0; w < W; w++)
        if (p.x[w] != wv[w]) return -1;
    return (q.e + popc_and<W>(q.x, q.z) + 2 * popc_and<W>(q.z, wv) + p.e + popc_and<W>(p.x, p.z)) & 3;
}

// anchor b*(sigma): bits 1 at the Z-pivot qubits of Z-rows with sigma = 1, then
// the X-pivot bits cleared with the X-rows' x parts.
template <int W>
__device__ void elem_anchor(const SfDev& d, const uint64_t* s, int r, uint64_t* b) {
    const int n = d.n;
#pragma unroll
    for (int w = 0; w < W; w++) b[w] = 0;
    for (int h = r; h < n; h++) {
        if ((s[h >> 6] >> (h & 63)) & 1) {
            const int qz = __ldg(&d.piv[h]) - n;
            b[qz >> 6] ^= 1ull << (qz & 63);
        }
    }
    for (int R = 0; R < r; R++) {
        const int pv = __ldg(&d.piv[R]);
        if ((b[pv >> 6] >> (pv & 63)) & 1) {
#pragma unroll
            for (int u = 0; u < W; u++) b[u] ^= __ldg(&d.mx[u * n + R]);
        }
    }
}

// ---------------------------------------------------------------------------
// sigma' = A sigma ^ t via 4-bit chunk tables: tab[c][w][v] = (A restricted
// to columns 4c..4c+3) applied to v, word w.  16 consecutive words per (c,w)
// keep a warp's lookups free of bank conflicts.
template <int W>
__global__ void __launch_bounds__(kThreads) k_affine(SfDev d, int buf) {
    extern __shared__ uint64_t tab[];
    if (*d.status) return;
    const int n = d.n, nc = (n + 3) >> 2;
    const uint64_t* AT = d.plan + plan_AT(n, W);
    for (int e = threadIdx.x; e < nc * W * 16; e += blockDim.x) {
        const int v = e & 15, cw = e >> 4, w = cw % W, c = cw / W;
        uint64_t acc = 0;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int j = 4 * c + b;
            if (((v >> b) & 1) && j < n) acc ^= AT[(size_t)j * W + w];
        }
        tab[e] = acc;
    }
    uint64_t t[W];
#pragma unroll
    for (int w = 0; w < W; w++) t[w] = d.plan[plan_t(n, W) + w];
    __syncthreads();
    const unsigned long long k = d.kcnt[buf];
    uint64_t* S = d.sig[buf];
    const uint64_t cap = d.cap;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    if constexpr (W == 1) {
        // two elements per thread with 128-bit accesses
        const unsigned long long k2 = k >> 1;
        ulonglong2* S2 = reinterpret_cast<ulonglong2*>(S);
        for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k2; j += stride) {
            ulonglong2 v = S2[j];
            uint64_t o0 = t[0], o1 = t[0];
            for (int c = 0; c < nc; c++) {
                o0 ^= tab[c * 16 + ((v.x >> (4 * c)) & 15)];
                o1 ^= tab[c * 16 + ((v.y >> (4 * c)) & 15)];
            }
            S2[j] = make_ulonglong2(o0, o1);
        }
        if ((k & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
            const uint64_t v = S[k - 1];
            uint64_t o = t[0];
            for (int c = 0; c < nc; c++) o ^= tab[c * 16 + ((v >> (4 * c)) & 15)];
            S[k - 1] = o;
        }
    } else {
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k; j += stride) {
        uint64_t s[W], o[W];
        load_sig<W>(S, cap, j, s);
#pragma unroll
        for (int w = 0; w < W; w++) o[w] = t[w];
        for (int c = 0; c < nc; c++) {
            const int v = (int)((s[c >> 4] >> (4 * (c & 15))) & 15);
#pragma unroll
            for (int w = 0; w < W; w++) o[w] ^= tab[(c * W + w) * 16 + v];
        }
        store_sig<W>(S, cap, j, o);
    }
    }
}

// W = 16 (n > 512): iterate over the set bits of sigma, XOR-ing columns of A.
template <int W>
__global__ void __launch_bounds__(kThreads) k_affine_cols(SfDev d, int buf) {
    if (*d.status) return;
    const int n = d.n;
    const uint64_t* AT = d.plan + plan_AT(n, W);
    uint64_t t[W];
#pragma unroll
    for (int w = 0; w < W; w++) t[w] = d.plan[plan_t(n, W) + w];
    const unsigned long long k = d.kcnt[buf];
    uint64_t* S = d.sig[buf];
    const uint64_t cap = d.cap;
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t s[W], o[W];
        load_sig<W>(S, cap, j, s);
#pragma unroll
        for (int w = 0; w < W; w++) o[w] = t[w];
        for (int w = 0; w < W; w++) {
            uint64_t bits = s[w];
            while (bits) {
                const int b = __ffsll((long long)bits) - 1;
                bits &= bits - 1;
                const uint64_t* col = AT + (size_t)(64 * w + b) * W;
#pragma unroll
                for (int u = 0; u < W; u++) o[u] ^= __ldg(&col[u]);
            }
        }
        store_sig<W>(S, cap, j, o);
    }
}

// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads) k_branch(SfDev d, int in_buf, int out_buf) {
    __shared__ uint64_t sh_u[SF_BR_MAXG][W];
    __shared__ uint64_t sh_v[SF_BR_MAXG][SF_BR_MAXT][W];
    __shared__ double2 sh_c[SF_BR_MAXG][SF_BR_MAXT];
    __shared__ int sh_nt[SF_BR_MAXG];
    if (*d.status) return;
    const int n = d.n;
    const uint64_t* pb = d.plan + plan_br(n, W);
    const int ng = (int)pb[0];
    const size_t gw = br_group_words(W);
    if (threadIdx.x < ng) {
        const uint64_t* G = pb + 1 + threadIdx.x * gw;
        for (int w = 0; w < W; w++) sh_u[threadIdx.x][w] = G[w];
        const int nt = (int)G[W];
        sh_nt[threadIdx.x] = nt;
        for (int t = 0; t < nt; t++) {
            const uint64_t* Tm = G + W + 1 + t * (2 + W);
            sh_c[threadIdx.x][t] = make_double2(__longlong_as_double((long long)Tm[0]),
                                                __longlong_as_double((long long)Tm[1]));
            for (int w = 0; w < W; w++) sh_v[threadIdx.x][t][w] = Tm[2 + w];
        }
    }
    __syncthreads();
    const unsigned long long k = d.kcnt[in_buf];
    if ((unsigned long long)ng * k > d.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_CAPACITY, in_buf);
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) d.kcnt[out_buf] = (unsigned long long)ng * k;
    const uint64_t* Si = d.sig[in_buf];
    uint64_t* So = d.sig[out_buf];
    const double2* Ai = d.amp[in_buf];
    double2* Ao = d.amp[out_buf];
    const uint64_t cap = d.cap;
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t s[W];
        load_sig<W>(Si, cap, j, s);
        const double2 a = Ai[j];
        for (int g = 0; g < ng; g++) {
            double2 cf = make_double2(0.0, 0.0);
            for (int t = 0; t < sh_nt[g]; t++) {
                const double sg = (popc_and<W>(sh_v[g][t], s) & 1) ? -1.0 : 1.0;
                cf.x += sg * sh_c[g][t].x;
                cf.y += sg * sh_c[g][t].y;
            }
            const unsigned long long o = (unsigned long long)g * k + j;
            uint64_t c[W];
#pragma unroll
            for (int w = 0; w < W; w++) c[w] = s[w] ^ sh_u[g][w];
            store_sig<W>(So, cap, o, c);
            Ao[o] = cmul(cf, a);
        }
    }
}

// ---------------------------------------------------------------------------
__global__ void k_coal_clear(SfDev d, int buf) {
    if (*d.status) return;
    const unsigned long long T = table_size(d.kcnt[buf], d.slots_cap);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < T;
         i += (unsigned long long)gridDim.x * blockDim.x)
        d.slots[i] = kEmpty;
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_coal_insert(SfDev d, int buf) {
    if (*d.status) return;
    const unsigned long long k = d.kcnt[buf];
    const unsigned long long T = table_size(k, d.slots_cap);
    const uint64_t* S = d.sig[buf];
    const uint64_t cap = d.cap;
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t s[W];
        load_sig<W>(S, cap, j, s);
        unsigned long long hh = hash_sig<W>(s) & (T - 1);
        uint32_t rep = kEmpty;
        for (unsigned long long probe = 0; probe < T; probe++) {
            uint32_t cur = d.slots[hh];
            if (cur == kEmpty) {
                cur = atomicCAS(&d.slots[hh], kEmpty, (uint32_t)j);
                if (cur == kEmpty) { rep = (uint32_t)j; break; }
            }
            bool eq = true;
#pragma unroll
            for (int w = 0; w < W; w++) eq &= (S[(size_t)w * cap + cur] == s[w]);
            if (eq) { rep = cur; break; }
            hh = (hh + 1) & (T - 1);
        }
        if (rep == kEmpty) set_status(d.status, SF_ST_TIMEOUT, buf);
        d.rep[j] = rep;
    }
}

__global__ void k_coal_accum(SfDev d, int buf) {
    if (*d.status) return;
    const unsigned long long k = d.kcnt[buf];
    double2* A = d.amp[buf];
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t r = d.rep[j];
        if (r != (uint32_t)j) {
            const double2 a = A[j];
            atomicAdd(&A[r].x, a.x);
            atomicAdd(&A[r].y, a.y);
        }
    }
}

// keep predicate.  mode 0: representative with |a| >= eps; mode 1: bit `bit`
// of sigma equals x.
template <int W>
__device__ __forceinline__ bool keep_elem(const SfDev& d, int buf, unsigned long long j, int mode, double eps2,
                                          int bit, int x) {
    if (mode == 0) {
        if (d.rep[j] != (uint32_t)j) return false;
        const double2 a = d.amp[buf][j];
        return a.x * a.x + a.y * a.y >= eps2;
    }
    const uint64_t w = d.sig[buf][(size_t)(bit >> 6) * d.cap + j];
    return (int)((w >> (bit & 63)) & 1) == x;
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_count(SfDev d, int buf, int mode, double eps2, int x) {
    __shared__ double sh[1][32];
    if (*d.status) return;
    const int bit = mode == 1 ? d.meta[1] : 0;
    if (bit < 0 || bit >= d.n) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, buf, 20u);
        return;
    }
    unsigned long long lo, hi;
    chunk_range(d.kcnt[buf], d.nblk, lo, hi);
    double c = 0;
    for (unsigned long long j = lo + threadIdx.x; j < hi; j += blockDim.x)
        c += keep_elem<W>(d, buf, j, mode, eps2, bit, x) ? 1.0 : 0.0;
    block_sum<1>(&c, sh);
    if (threadIdx.x == 0) d.blk[blockIdx.x] = (unsigned long long)c;
}

// exclusive scan of the per-CTA counts; total -> kcnt[out_buf]
__global__ void __launch_bounds__(1024) k_scan(SfDev d, int out_buf) {
    __shared__ unsigned long long sh[1024];
    if (*d.status) return;
    const int nb = d.nblk, t = threadIdx.x;
    unsigned long long carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        const unsigned long long v = (base + t < nb) ? d.blk[base + t] : 0ull;
        sh[t] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            unsigned long long a = t >= o ? sh[t - o] : 0ull;
            __syncthreads();
            sh[t] += a;
            __syncthreads();
        }
        if (base + t < nb) d.blk[nb + base + t] = carry + sh[t] - v;
        carry += sh[1023];
        __syncthreads();
    }
    if (t == 0) d.kcnt[out_buf] = carry;
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_scatter(SfDev d, int in_buf, int out_buf, int mode, double eps2, int x) {
    __shared__ int wc[kThreads / 32];
    __shared__ int wo[kThreads / 32 + 1];
    if (*d.status) return;
    const int bit = mode == 1 ? d.meta[1] : 0;
    if (bit < 0 || bit >= d.n) return;
    double scale = 1.0;
    if (mode == 1) scale = 1.0 / sqrt(d.out[x]);
    unsigned long long lo, hi;
    chunk_range(d.kcnt[in_buf], d.nblk, lo, hi);
    unsigned long long base = d.blk[d.nblk + blockIdx.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint64_t* Si = d.sig[in_buf];
    uint64_t* So = d.sig[out_buf];
    const uint64_t cap = d.cap;
    for (unsigned long long t0 = lo; t0 < hi; t0 += blockDim.x) {
        const unsigned long long j = t0 + threadIdx.x;
        const bool kp = j < hi && keep_elem<W>(d, in_buf, j, mode, eps2, bit, x);
        const unsigned bal = __ballot_sync(SF_FULL, kp);
        if (lane == 0) wc[wid] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int i = 0; i < nw; i++) { wo[i] = s; s += wc[i]; }
            wo[nw] = s;
        }
        __syncthreads();
        if (kp) {
            const unsigned long long o = base + wo[wid] + __popc(bal & ((1u << lane) - 1u));
            uint64_t s[W];
            load_sig<W>(Si, cap, j, s);
            store_sig<W>(So, cap, o, s);
            double2 a = d.amp[in_buf][j];
            a.x *= scale;
            a.y *= scale;
            d.amp[out_buf][o] = a;
        }
        base += wo[nw];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads) k_cof_split(SfDev d, int in_buf, int out_buf) {
    if (*d.status) return;
    if (!d.meta[2]) return;
    const int n = d.n;
    const uint64_t* pl = d.plan;
    const unsigned long long k = d.kcnt[in_buf];
    if (2 * k > d.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_CAPACITY, in_buf);
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) d.kcnt[out_buf] = 2 * k;
    double2 kap[2];
    const size_t ko = cf_kappa(n, W);
    kap[0] = make_double2(__longlong_as_double((long long)pl[ko]), __longlong_as_double((long long)pl[ko + 1]));
    kap[1] = make_double2(__longlong_as_double((long long)pl[ko + 2]), __longlong_as_double((long long)pl[ko + 3]));
    uint64_t vq[W], tau[2][W], eps0[W], eps1[W];
#pragma unroll
    for (int w = 0; w < W; w++) {
        vq[w] = pl[cf_vq(n, W) + w];
        tau[0][w] = pl[cf_tau(n, W) + w];
        tau[1][w] = pl[cf_tau(n, W) + W + w];
        eps0[w] = pl[cf_eps(n, W) + w];
        eps1[w] = pl[cf_eps(n, W) + W + w];
    }
    const uint64_t* U = pl + cf_u(n, W);
    const uint64_t* V = pl + cf_v(n, W);
    const uint64_t* Si = d.sig[in_buf];
    uint64_t* So = d.sig[out_buf];
    const double2* Ai = d.amp[in_buf];
    double2* Ao = d.amp[out_buf];
    const uint64_t cap = d.cap;
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t s[W];
        load_sig<W>(Si, cap, j, s);
        const double2 a = Ai[j];
        const int py = popc_and<W>(vq, s) & 1;
        for (int x = 0; x < 2; x++) {
            const int y = x ^ py;
            uint64_t t[W];
#pragma unroll
            for (int w = 0; w < W; w++) t[w] = tau[y][w];
            int ip = 0;  // i-power accumulated over the old destabilizers of sigma
#pragma unroll
            for (int w = 0; w < W; w++) {
                uint64_t bits = s[w];
                while (bits) {
                    const int b = __ffsll((long long)bits) - 1;
                    bits &= bits - 1;
                    const int h = 64 * w + b;
                    uint64_t vv[W];
#pragma unroll
                    for (int u = 0; u < W; u++) vv[u] = __ldg(&V[(size_t)h * W + u]);
                    ip += (int)((eps0[w] >> b) & 1) + 2 * (int)((eps1[w] >> b) & 1) + 2 * (popc_and<W>(vv, t) & 1);
#pragma unroll
                    for (int u = 0; u < W; u++) t[u] ^= __ldg(&U[(size_t)h * W + u]);
                }
            }
            const double2 c = ipow_mul(cmul(kap[y], a), ip & 3);
            const unsigned long long o = (unsigned long long)x * k + j;
            store_sig<W>(So, cap, o, t);
            Ao[o] = c;
        }
    }
}

// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads) k_prob(SfDev d, int buf) {
    __shared__ double sh[2][32];
    if (*d.status) return;
    const int R = d.meta[1];
    if (R < 0 || R >= d.n) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, buf, 21u);
        return;
    }
    const unsigned long long k = d.kcnt[buf];
    const uint64_t* plane = d.sig[buf] + (size_t)(R >> 6) * d.cap;
    const double2* A = d.amp[buf];
    double p[2] = {0.0, 0.0};
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        const double2 a = A[j];
        const double m = a.x * a.x + a.y * a.y;
        if ((plane[j] >> (R & 63)) & 1) p[1] += m;
        else p[0] += m;
    }
    block_sum<2>(p, sh);
    if (threadIdx.x == 0) {
        d.red[2 * blockIdx.x] = p[0];
        d.red[2 * blockIdx.x + 1] = p[1];
    }
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_amplitude(SfDev d, int buf) {
    __shared__ double sh[2][32];
    if (*d.status) return;
    const int n = d.n, r = d.meta[0];
    const size_t o = plan_am(n, W);
    uint64_t y[W], zm[W], ze[W];
#pragma unroll
    for (int w = 0; w < W; w++) { y[w] = d.plan[o + w]; zm[w] = d.plan[o + W + w]; ze[w] = d.plan[o + 2 * W + w]; }
    const unsigned long long k = d.kcnt[buf];
    double acc[2] = {0.0, 0.0};
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t s[W];
        load_sig<W>(d.sig[buf], d.cap, j, s);
        bool match = true;
#pragma unroll
        for (int w = 0; w < W; w++) match &= ((s[w] & zm[w]) == ze[w]);
        if (!match) continue;
        const int ip = elem_amp_phi<W>(d, s, y, r);
        if (ip < 0) continue;
        const double2 c = ipow_mul(d.amp[buf][j], ip);
        acc[0] += c.x;
        acc[1] += c.y;
    }
    block_sum<2>(acc, sh);
    if (threadIdx.x == 0) {
        d.red[2 * blockIdx.x] = acc[0];
        d.red[2 * blockIdx.x + 1] = acc[1];
    }
}

// fixed-order sum of the per-CTA partials.  what 0: probabilities -> out[0..1];
// what 1: amplitude -> out[2..3] scaled by g 2^{-r/2}.
__global__ void k_reduce_final(SfDev d, int what) {
    __shared__ double sh[2][32];
    double v[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < d.nblk; b += blockDim.x) {
        v[0] += d.red[2 * b];
        v[1] += d.red[2 * b + 1];
    }
    block_sum<2>(v, sh);
    if (threadIdx.x == 0) {
        if (what == 0) {
            d.out[0] = v[0];
            d.out[1] = v[1];
        } else {
            const double sc = exp2(-0.5 * (double)d.meta[0]);
            const double2 c = cmul(*d.g, make_double2(v[0] * sc, v[1] * sc));
            d.out[2] = c.x;
            d.out[3] = c.y;
        }
    }
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_export(SfDev d, int buf, int stage_buf) {
    if (*d.status) return;
    const int r = d.meta[0];
    const double2 g = *d.g;
    const unsigned long long k = d.kcnt[buf];
    uint64_t* xsig = d.sig[stage_buf];   // staging, row-major per element
    double2* xamp = d.amp[stage_buf];
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t s[W], b[W];
        load_sig<W>(d.sig[buf], d.cap, j, s);
        elem_anchor<W>(d, s, r, b);
        const int ip = elem_amp_phi<W>(d, s, b, r);
        if (ip < 0) {
            set_status(d.status, SF_ST_INTERNAL, buf, 22u);
            continue;
        }
        xamp[j] = ipow_mul(cmul(g, d.amp[buf][j]), ip);
#pragma unroll
        for (int w = 0; w < W; w++) xsig[(size_t)j * W + w] = s[w];
    }
}

}  // namespace

#define SF_DISPATCH(W_, ...)                                  \
    switch (W_) {                                             \
        case 1: { constexpr int WW = 1; __VA_ARGS__; } break; \
        case 2: { constexpr int WW = 2; __VA_ARGS__; } break; \
        case 4: { constexpr int WW = 4; __VA_ARGS__; } break; \
        case 8: { constexpr int WW = 8; __VA_ARGS__; } break; \
        default: { constexpr int WW = 16; __VA_ARGS__; } break; \
    }

size_t sf_affine_smem_bytes(int n, int W) { return (size_t)((n + 3) / 4) * W * 16 * 8; }

void sf_launch_affine(const SfDev& d, int buf, cudaStream_t s) {
    if (d.W == 16) {
        k_affine_cols<16><<<d.nblk, kThreads, 0, s>>>(d, buf);
        return;
    }
    const size_t sm = sf_affine_smem_bytes(d.n, d.W);
    SF_DISPATCH(d.W, {
        static bool attr = false;
        if (!attr && sm > 48 * 1024) {
            cudaFuncSetAttribute(k_affine<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr = true;
        }
        k_affine<WW><<<d.nblk, kThreads, sm, s>>>(d, buf);
    });
}

void sf_launch_branch(const SfDev& d, int in_buf, int out_buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_branch<WW><<<d.nblk, kThreads, 0, s>>>(d, in_buf, out_buf));
}

void sf_launch_coal_clear(const SfDev& d, int buf, cudaStream_t s) { k_coal_clear<<<d.nblk, kThreads, 0, s>>>(d, buf); }

void sf_launch_coal_insert(const SfDev& d, int buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_coal_insert<WW><<<d.nblk, kThreads, 0, s>>>(d, buf));
}

void sf_launch_coal_accum(const SfDev& d, int buf, cudaStream_t s) { k_coal_accum<<<d.nblk, kThreads, 0, s>>>(d, buf); }

void sf_launch_count(const SfDev& d, int buf, int mode, double eps2, int x, cudaStream_t s) {
    SF_DISPATCH(d.W, k_count<WW><<<d.nblk, kThreads, 0, s>>>(d, buf, mode, eps2, x));
}

void sf_launch_scan(const SfDev& d, int out_buf, cudaStream_t s) { k_scan<<<1, 1024, 0, s>>>(d, out_buf); }

void sf_launch_scatter(const SfDev& d, int in_buf, int out_buf, int mode, double eps2, int x, cudaStream_t s) {
    SF_DISPATCH(d.W, k_scatter<WW><<<d.nblk, kThreads, 0, s>>>(d, in_buf, out_buf, mode, eps2, x));
}

void sf_launch_cofactor_split(const SfDev& d, int in_buf, int out_buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_cof_split<WW><<<d.nblk, kThreads, 0, s>>>(d, in_buf, out_buf));
}

void sf_launch_prob(const SfDev& d, int buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_prob<WW><<<d.nblk, kThreads, 0, s>>>(d, buf));
}

void sf_launch_reduce_final(const SfDev& d, int what, cudaStream_t s) { k_reduce_final<<<1, 1024, 0, s>>>(d, what); }

void sf_launch_amplitude(const SfDev& d, int buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_amplitude<WW><<<d.nblk, kThreads, 0, s>>>(d, buf));
}

void sf_launch_export(const SfDev& d, int buf, int stage_buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_export<WW><<<d.nblk, kThreads, 0, s>>>(d, buf, stage_buf));
}
