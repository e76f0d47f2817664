// sf_frame.cu -- kernels that stream over the frame elements (phase vectors
// sigma, word-major [W][cap], and FP64 complex amplitudes):
//   k_affine      per-element Clifford update sigma' = A sigma ^ t (Sec. III,
//                 ROTATE: the memoised row operations of Invariant 1 applied
//                 to every phase vector), 4-bit table lookups in shared memory
//   k_branch      diagonal non-Clifford branching (Sec. IV), children unmerged
//   k_insert      children (of a branch, a cofactor split, or the frame itself)
//                 hashed into a slot table with FP64 amplitude accumulation
//   k_compact     COALESCE in the set sense of Def. 1: emit every slot with
//                 |a| >= eps and leave the table empty
//   k_filter      collapse after a measurement
//   k_cond        Toffoli / controlled-R(alpha) on the 11 cofactor (Eq. 2, Eq. 3)
//   k_prob        measurement probabilities (Sec. IV, measuring F)
//   k_amplitude   <y|Psi> (Observation 1)
//   k_export      canonical-convention amplitudes for export
// Per-element kernels use a fixed grid of d.nblk CTAs and read the element
// count from device memory, so no host synchronisation is needed between them.
#include <type_traits>

#include "sf_canon.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ unsigned long long table_size(unsigned long long k, unsigned long long cap) {
    unsigned long long t = 1024;
    while (t < 2 * k && t < cap) t <<= 1;
    return t < cap ? t : cap;
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

// Fixed-order sum of the per-CTA partials d.red[2b], d.red[2b + 1] over the
// grid, by the last CTA to finish (all its threads; every CTA wrote its
// partials before counting itself done).  what 0: probabilities -> out[0..1];
// what 1: amplitude -> out[2..3], scaled by g 2^{-r/2}.
__device__ void reduce_partials(const SfDev& d, int what, double (*sh)[32]) {
    double v[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        v[0] += __ldcg(&d.red[2 * b]);
        v[1] += __ldcg(&d.red[2 * b + 1]);
    }
    block_sum<2>(v, sh);
    if (threadIdx.x == 0) {
        if (what == 0) {
            d.out[0] = v[0];
            d.out[1] = v[1];
        } else {
            // 2^{-r/2} exactly: a power of two, times 1/sqrt(2) for odd r
            const int r = d.meta[0];
            const double sc = ldexp(1.0, -((r + 1) >> 1)) * ((r & 1) ? 1.41421356237309504880 : 1.0);
            const double2 c = cmul(*d.g, make_double2(v[0] * sc, v[1] * sc));
            d.out[2] = c.x;
            d.out[3] = c.y;
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
    if constexpr (W >= 8) {
        if (d.plan[plan_lr_aff(n, W)] <= SF_LR_MAX) return;  // k_affine_lr applies the map
    }
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

// W = 16 (n > 512): iterate over the set bits of sigma, XOR-ing columns of A;
// runs only when A ^ I has rank above SF_LR_MAX (k_affine_lr otherwise).
template <int W>
__global__ void __launch_bounds__(kThreads) k_affine_cols(SfDev d, int buf) {
    if (*d.status) return;
    const int n = d.n;
    if (d.plan[plan_lr_aff(n, W)] <= SF_LR_MAX) return;
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
// Low-rank form of a GF(2) map near a permutation (W >= 8).  One Clifford gate
// or one measurement changes the tableau by a few row operations and then
// sorts the rows by pivot, which moves the few rows whose pivot changed.  The
// phase-vector map R it induces is therefore the sort's permutation rho plus a
// matrix of small rank r: with Delta_h = R_h ^ e_{rho(h)} =
// sum_i C[h][i] B_i, a product sum_{h in sigma} R_h is
// rho(sigma) ^ sum_i parity(sigma & c_i) B_i -- a few bit moves and 2 r W
// word operations per element instead of one W-word row per set bit of sigma
// (n/2 on average).  The decomposition is exact for any rho; the sort's
// permutation only makes r small.

// the sort's permutation as bit moves, in shared memory (the plan's move list)
struct Moves {
    int m;
    int a[SF_MV_MAX], e[SF_MV_MAX], src[SF_MV_MAX], isrc[SF_MV_MAX];
};

// threads 0..4*SF_MV_MAX; a __syncthreads must follow
__device__ __forceinline__ void load_moves(const uint64_t* mv, Moves& M) {
    const int t = threadIdx.x;
    if (t == 0) M.m = (int)mv[0];
    if (t < 4 * SF_MV_MAX) {
        const int v = (int)mv[1 + t], k = t % SF_MV_MAX;
        int* dst = t < SF_MV_MAX ? M.a : t < 2 * SF_MV_MAX ? M.e : t < 3 * SF_MV_MAX ? M.src : M.isrc;
        dst[k] = v;
    }
}

// bit p of a W-word vector (p uniform or not; no indexed register access)
template <int W>
__device__ __forceinline__ uint32_t bit_at(const uint64_t* v, int p) {
    uint64_t r = 0;
#pragma unroll
    for (int w = 0; w < W; w++)
        if (w == (p >> 6)) r = (v[w] >> (p & 63)) & 1ull;
    return (uint32_t)r;
}

// delete bit position p: the bits above it move down one, a zero enters at the top
template <int W>
__device__ __forceinline__ void bits_delete(uint64_t* v, int p) {
    const int wp = p >> 6;
    const uint64_t low = (1ull << (p & 63)) - 1ull;
#pragma unroll
    for (int w = 0; w < W; w++) {
        const uint64_t nxt = (w + 1 < W) ? v[w + 1] : 0ull;
        const uint64_t sh = (v[w] >> 1) | (nxt << 63);
        if (w > wp) v[w] = sh;
        else if (w == wp) v[w] = (v[w] & low) | (sh & ~low);
    }
}

// insert bit x at position p: the bits at and above it move up one (the top
// bit of the vector, always zero here, leaves)
template <int W>
__device__ __forceinline__ void bits_insert(uint64_t* v, int p, uint32_t x) {
    const int wp = p >> 6;
    const uint64_t low = (1ull << (p & 63)) - 1ull, at = 1ull << (p & 63);
#pragma unroll
    for (int w = W - 1; w >= 0; w--) {
        const uint64_t prv = w > 0 ? v[w - 1] : 0ull;
        const uint64_t sh = (v[w] << 1) | (prv >> 63);
        if (w > wp) v[w] = sh;
        else if (w == wp) v[w] = (v[w] & low) | (sh & ~(low | at)) | ((uint64_t)x << (p & 63));
    }
}

// bits pos[0..m) of v, packed (bit k = bit pos[k] of v).  Words outside,
// positions inside: a word picked by a run-time position would take v out of
// registers.
template <int W>
__device__ __forceinline__ uint32_t bits_gather(const uint64_t* v, const int* pos, int m) {
    uint32_t bits = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        const uint64_t x = v[w];
#pragma unroll 1
        for (int k = 0; k < m; k++) {
            const int p = pos[k];
            if ((p >> 6) == w) bits |= (uint32_t)((x >> (p & 63)) & 1ull) << k;
        }
    }
    return bits;
}

// v <- rho(v): bit h moves to rho(h)
template <int W>
__device__ __forceinline__ void apply_moves(uint64_t* v, const Moves& M) {
    const int m = M.m;
    const uint32_t bits = bits_gather<W>(v, M.a, m);
#pragma unroll 1
    for (int k = m - 1; k >= 0; k--) bits_delete<W>(v, M.a[k]);
#pragma unroll 1
    for (int j = 0; j < m; j++) bits_insert<W>(v, M.e[j], (bits >> M.src[j]) & 1u);
}

// v <- rho^{-1}(v)
template <int W>
__device__ __forceinline__ void apply_moves_inv(uint64_t* v, const Moves& M) {
    const int m = M.m;
    const uint32_t bits = bits_gather<W>(v, M.e, m);
#pragma unroll 1
    for (int j = m - 1; j >= 0; j--) bits_delete<W>(v, M.e[j]);
#pragma unroll 1
    for (int k = 0; k < m; k++) bits_insert<W>(v, M.a[k], (bits >> M.isrc[k]) & 1u);
}

// Gaussian elimination over the n vectors Delta_h, one thread per vector
// (x: this thread's vector, zero for threads h >= n; consumed): each round the
// first vector not yet in the span of B_0..B_{m-1} becomes B_m (pivot: its
// lowest set bit), and every thread clears that pivot from its own remainder.
// B_m has the pivots of B_0..B_{m-1} clear, so clearing pivot m never sets an
// earlier one, and a remainder that reaches zero is the sum of the B_i it
// used.  blockDim.x >= n, a multiple of 32.  Writes the block at out (r, B,
// c) and returns r, or -1 when r would exceed SF_LR_MAX (the block then reads
// SF_LR_NONE).
template <int W>
__device__ int cta_lowrank(uint64_t* x, int n, uint64_t* out) {
    __shared__ uint64_t B[SF_LR_MAX][W];
    __shared__ int piv[SF_LR_MAX];
    __shared__ int first;
    __shared__ uint32_t cb[SF_LR_MAX][32];
    const int h = threadIdx.x;
    uint32_t used = 0;
    int r = 0;
    for (;;) {
        if (h == 0) first = 0x7fffffff;
        __syncthreads();
        bool nz = false;
#pragma unroll
        for (int w = 0; w < W; w++) nz |= x[w] != 0ull;
        if (nz) atomicMin(&first, h);
        __syncthreads();
        const int f = first;
        if (f == 0x7fffffff) break;
        if (r == SF_LR_MAX) {
            r = -1;
            break;
        }
        if (h == f) {
            int p = -1;
#pragma unroll
            for (int w = W - 1; w >= 0; w--)
                if (x[w]) p = 64 * w + __ffsll((long long)x[w]) - 1;
#pragma unroll
            for (int w = 0; w < W; w++) {
                B[r][w] = x[w];
                x[w] = 0ull;
            }
            piv[r] = p;
            used |= 1u << r;
        }
        __syncthreads();
        if (bit_at<W>(x, piv[r])) {
#pragma unroll
            for (int w = 0; w < W; w++) x[w] ^= B[r][w];
            used |= 1u << r;
        }
        r++;
    }
    if (r < 0) {
        if (h == 0) out[0] = SF_LR_NONE;
        __syncthreads();
        return -1;
    }
    for (int e = h; e < SF_LR_MAX * 32; e += blockDim.x) cb[e >> 5][e & 31] = 0u;
    __syncthreads();
    for (int i = 0; i < r; i++) {
        const unsigned bal = __ballot_sync(SF_FULL, (used >> i) & 1u);
        if ((h & 31) == 0) cb[i][h >> 5] = bal;
    }
    __syncthreads();
    if (h == 0) out[0] = (uint64_t)r;
    for (int e = h; e < r * W; e += blockDim.x) {
        const int i = e / W, w = e % W;
        out[lr_B(W) + (size_t)i * W + w] = B[i][w];
        out[lr_C(W) + (size_t)i * W + w] = (uint64_t)cb[i][2 * w] | ((uint64_t)cb[i][2 * w + 1] << 32);
    }
    __syncthreads();
    return r;
}

// factors of the Clifford batch's map (columns of A: sigma' = sum_{j in sigma}
// col_j ^ t), with Delta_j = col_j ^ e_{rho(j)}
template <int W>
__global__ void __launch_bounds__(1024) k_affine_lowrank(SfDev d) {
    if (*d.status) return;
    const int n = d.n, h = threadIdx.x;
    uint64_t* out = d.plan + plan_lr_aff(n, W);
    if (!d.lowrank || d.plan[plan_mv_aff(n, W)] > SF_MV_MAX) {
        if (h == 0) out[0] = SF_LR_NONE;
        return;
    }
    uint64_t x[W];
#pragma unroll
    for (int w = 0; w < W; w++) x[w] = h < n ? d.plan[plan_AT(n, W) + (size_t)h * W + w] : 0ull;
    if (h < n) {
        const int p = (int)reinterpret_cast<const uint32_t*>(d.plan + plan_rho_aff(n, W))[h];
#pragma unroll
        for (int w = 0; w < W; w++)
            if (w == (p >> 6)) x[w] ^= 1ull << (p & 63);
    }
    cta_lowrank<W>(x, n, out);
}

// sigma' = rho(sigma) ^ t ^ sum_i parity(sigma & c_i) B_i; does nothing when
// the low-rank form is not available (the dense kernel applies the map then)
template <int W>
__global__ void __launch_bounds__(kThreads) k_affine_lr(SfDev d, int buf) {
    __shared__ uint64_t B[SF_LR_MAX][W], C[SF_LR_MAX][W], t[W];
    __shared__ Moves M;
    if (*d.status) return;
    const int n = d.n;
    const uint64_t* L = d.plan + plan_lr_aff(n, W);
    const uint64_t rr = L[0];
    if (rr > SF_LR_MAX) return;
    const int r = (int)rr;
    for (int e = threadIdx.x; e < r * W; e += blockDim.x) {
        B[e / W][e % W] = L[lr_B(W) + e];
        C[e / W][e % W] = L[lr_C(W) + e];
    }
    if (threadIdx.x < W) t[threadIdx.x] = d.plan[plan_t(n, W) + threadIdx.x];
    load_moves(d.plan + plan_mv_aff(n, W), M);
    __syncthreads();
    const unsigned long long k = d.kcnt[buf];
    uint64_t* S = d.sig[buf];
    const uint64_t cap = d.cap;
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t s[W];
        load_sig<W>(S, cap, j, s);
        uint32_t sel = 0;
#pragma unroll 1
        for (int i = 0; i < r; i++) sel |= (uint32_t)(popc_and<W>(C[i], s) & 1) << i;
        apply_moves<W>(s, M);
#pragma unroll
        for (int w = 0; w < W; w++) s[w] ^= *(const volatile uint64_t*)&t[w];
#pragma unroll 1
        for (int i = 0; i < r; i++) {
            if ((sel >> i) & 1u) {
#pragma unroll
                for (int w = 0; w < W; w++) s[w] ^= B[i][w];
            }
        }
        store_sig<W>(S, cap, j, s);
    }
}

// ---------------------------------------------------------------------------
// Plan of a diagonal gate sum_j c_j Z^{w_j} (Sec. IV), computed by one warp of
// every CTA from the tableau: Z^w = eps D^u M^v with u_h = [Z^w anticommutes
// with M_h], v_h = [Z^w anticommutes with D_h], so that
// Z^w D^sigma phi_0 = eps (-1)^{v.sigma} D^{sigma ^ u} phi_0.  eps may be +-i.
// Terms with equal u form one group (one child per element).
template <int W>
struct BrPlan {
    int ng, bad;
    int nt[SF_BR_MAXG];
    uint64_t u[SF_BR_MAXG][W];
    uint64_t v[SF_BR_MAXG][SF_BR_MAXT][W];
    double2 c[SF_BR_MAXG][SF_BR_MAXT];
};


__device__ __forceinline__ uint64_t warp_or(uint64_t v) {
#pragma unroll
    for (int off = 16; off; off >>= 1) v |= __shfl_xor_sync(SF_FULL, v, off);
    return v;
}

// called by the 32 lanes of one warp; lane 0 writes P
template <int W>
// tm: the term coefficients of the gate (diag_terms)
__device__ void warp_branch_plan(const SfDev& d, uint32_t kind, uint32_t q0, uint32_t q1, const SfTerms& tm,
                                 BrPlan<W>& P) {
    const int lane = threadIdx.x & 31, n = d.n;
    const double2* cf = tm.c;
    int nt;
    int wq[SF_BR_MAXT][2];
    if (kind <= 2) {  // terms I, Z_q0
        nt = 2;
        wq[0][0] = -1; wq[0][1] = -1;
        wq[1][0] = (int)q0; wq[1][1] = -1;
    } else {  // terms I, Z_c, Z_t, Z_c Z_t
        nt = 4;
        wq[0][0] = -1; wq[0][1] = -1;
        wq[1][0] = (int)q0; wq[1][1] = -1;
        wq[2][0] = (int)q1; wq[2][1] = -1;
        wq[3][0] = (int)q0; wq[3][1] = (int)q1;
    }
    uint64_t um[SF_BR_MAXT][W], vm[SF_BR_MAXT][W], wz[SF_BR_MAXT][W], odd[W];
    int epsq[SF_BR_MAXT];
    int bad = 0;
    Pauli<W> p[SF_BR_MAXT];
    // the identity term needs no pass; for CR the Z_c Z_t term follows from the other two
    bool skip[SF_BR_MAXT];
    for (int j = 0; j < nt; j++) {
#pragma unroll
        for (int w = 0; w < W; w++) { wz[j][w] = 0; um[j][w] = 0; vm[j][w] = 0; }
        for (int a = 0; a < 2; a++)
            if (wq[j][a] >= 0) wz[j][wq[j][a] >> 6] ^= 1ull << (wq[j][a] & 63);
        pauli_id<W>(p[j]);
        skip[j] = wq[j][0] < 0 || (kind == 3 && j == 3);
    }
#pragma unroll
    for (int w = 0; w < W; w++) odd[w] = 0;
    // each row is read once for all terms: u_h = [Z^w anticommutes with M_h],
    // v_h = [Z^w anticommutes with D_h], contribution D_h^{u_h} M_h^{v_h}
    for (int h = lane; h < n; h += 32) {
        Pauli<W> dh, mh;
#pragma unroll
        for (int w = 0; w < W; w++) {
            mh.x[w] = __ldg(&d.mx[w * n + h]);
            mh.z[w] = __ldg(&d.mz[w * n + h]);
            dh.x[w] = __ldg(&d.dx[w * n + h]);
            dh.z[w] = __ldg(&d.dz[w * n + h]);
        }
        mh.e = 0;
        dh.e = (int)__ldg(&d.de[h]);
        if (dh.e & 1) odd[h >> 6] |= 1ull << (h & 63);
        for (int j = 0; j < nt; j++) {
            if (skip[j]) continue;
            const bool ub = popc_and<W>(mh.x, wz[j]) & 1;
            const bool vb = popc_and<W>(dh.x, wz[j]) & 1;
            if (ub) {
                um[j][h >> 6] |= 1ull << (h & 63);
                pauli_mul<W>(p[j], dh);
            }
            if (vb) {
                vm[j][h >> 6] |= 1ull << (h & 63);
                pauli_mul<W>(p[j], mh);
            }
        }
    }
    for (int j = 0; j < nt; j++) {
        if (skip[j]) continue;
        warp_pauli_product<W>(p[j]);
#pragma unroll
        for (int w = 0; w < W; w++) {
            um[j][w] = warp_or(um[j][w]);
            vm[j][w] = warp_or(vm[j][w]);
            if (p[j].x[w] != 0 || p[j].z[w] != wz[j][w]) bad = 1;
        }
        epsq[j] = (4 - p[j].e) & 3;
    }
    epsq[0] = 0;  // identity: u = v = 0 (zeroed above)
    if (kind == 3) {
        // Z^{w1} Z^{w2} = eps1 eps2 D^{u1} M^{v1} D^{u2} M^{v2}: moving M^{v1} past D^{u2}
        // gives (-1)^{|v1 & u2|}; D^{u1} D^{u2} = D^{u1^u2} times the squares of the
        // shared destabilizers (-1 for an odd i-power)
        int par = 0;
#pragma unroll
        for (int w = 0; w < W; w++) {
            odd[w] = warp_or(odd[w]);
            um[3][w] = um[1][w] ^ um[2][w];
            vm[3][w] = vm[1][w] ^ vm[2][w];
            par += __popcll(vm[1][w] & um[2][w]) + __popcll(um[1][w] & um[2][w] & odd[w]);
        }
        epsq[3] = (epsq[1] + epsq[2] + 2 * par) & 3;
    }
    if (lane != 0) return;
    int gid[SF_BR_MAXT];
    int ng = 0;
    for (int j = 0; j < nt; j++) {
        int found = -1;
        for (int j2 = 0; j2 < j; j2++) {
            bool same = true;
            for (int w = 0; w < W; w++) same &= um[j2][w] == um[j][w];
            if (same) { found = gid[j2]; break; }
        }
        gid[j] = found >= 0 ? found : ng++;
    }
    P.ng = ng;
    P.bad = bad;
    for (int g = 0; g < ng; g++) P.nt[g] = 0;
    for (int j = 0; j < nt; j++) {
        const int g = gid[j], t = P.nt[g]++;
        for (int w = 0; w < W; w++) {
            P.u[g][w] = um[j][w];
            P.v[g][t][w] = vm[j][w];
        }
        P.c[g][t] = ipow_mul(cf[j], epsq[j]);
    }
}

// The same plan computed once per gate by one CTA of kPlanThreads threads and
// written to the plan area (W >= 8, where the 16-word Pauli products would
// otherwise set the register count of every streaming kernel and each of
// their CTAs would read the whole tableau).  Thread t reads the rows
// h = t, t + kPlanThreads, ...; u_h reads only the words of the term's qubits.
// The partial products of distinct rows commute (D_h and M_k anticommute only
// for h = k, and both factors of one h stay in one thread, D_h first), so the
// warps' partials may be multiplied in any order.
constexpr int kPlanThreads = 256;

template <int W>
__global__ void __launch_bounds__(kPlanThreads) k_branch_plan(SfDev d, uint32_t kind, uint32_t q0, uint32_t q1,
                                                              SfTerms tm) {
    __shared__ uint64_t su[SF_BR_MAXT][W], sv[SF_BR_MAXT][W], sodd[W];
    __shared__ Pauli<W> part[kPlanThreads / 32];
    __shared__ int epsq[SF_BR_MAXT], sbad;
    __shared__ BrPlan<W> P;
    static_assert(sizeof(BrPlan<W>) <= 8 * SF_BR_WORDS(W), "branch plan area too small");
    if (*d.status) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, n = d.n;
    const int nt = kind <= 2 ? 2 : 4;
    const int qa[SF_BR_MAXT] = {-1, (int)q0, (int)q1, (int)q0};
    for (int e = tid; e < SF_BR_MAXT * W; e += blockDim.x) {
        su[e / W][e % W] = 0ull;
        sv[e / W][e % W] = 0ull;
    }
    if (tid < W) sodd[tid] = 0ull;
    if (tid == 0) {
        sbad = 0;
        for (int j = 0; j < SF_BR_MAXT; j++) epsq[j] = 0;
    }
    __syncthreads();
    for (int h = tid; h < n; h += blockDim.x)
        if (__ldg(&d.de[h]) & 1u) atomicOr(reinterpret_cast<unsigned long long*>(&sodd[h >> 6]), 1ull << (h & 63));
    // terms 1 (and 2 for the two-qubit gates); the identity needs no pass and the
    // Z_c Z_t term follows from the other two
    for (int j = 1; j < nt && j <= 2; j++) {
        uint64_t wz[W];
#pragma unroll
        for (int w = 0; w < W; w++) wz[w] = 0ull;
        wz[qa[j] >> 6] ^= 1ull << (qa[j] & 63);
        Pauli<W> p;
        pauli_id<W>(p);
        for (int h = tid; h < n; h += blockDim.x) {
            const int qw = qa[j] >> 6, qs = qa[j] & 63;
            const bool ub = (__ldg(&d.mx[qw * n + h]) >> qs) & 1ull;
            const bool vb = (__ldg(&d.dx[qw * n + h]) >> qs) & 1ull;
            if (ub) {
                Pauli<W> dh;
#pragma unroll
                for (int w = 0; w < W; w++) {
                    dh.x[w] = __ldg(&d.dx[w * n + h]);
                    dh.z[w] = __ldg(&d.dz[w * n + h]);
                }
                dh.e = (int)__ldg(&d.de[h]);
                pauli_mul<W>(p, dh);
                atomicOr(reinterpret_cast<unsigned long long*>(&su[j][h >> 6]), 1ull << (h & 63));
            }
            if (vb) {
                Pauli<W> mh;
#pragma unroll
                for (int w = 0; w < W; w++) {
                    mh.x[w] = __ldg(&d.mx[w * n + h]);
                    mh.z[w] = __ldg(&d.mz[w * n + h]);
                }
                mh.e = 0;
                pauli_mul<W>(p, mh);
                atomicOr(reinterpret_cast<unsigned long long*>(&sv[j][h >> 6]), 1ull << (h & 63));
            }
        }
        warp_pauli_product<W>(p);
        if (lane == 0) part[wid] = p;
        __syncthreads();
        if (tid == 0) {
            Pauli<W> t = part[0];
            for (int k = 1; k < (int)(blockDim.x >> 5); k++) pauli_mul<W>(t, part[k]);
            int bad = 0;
            for (int w = 0; w < W; w++)
                if (t.x[w] != 0ull || t.z[w] != wz[w]) bad = 1;
            sbad |= bad;
            epsq[j] = (4 - t.e) & 3;
        }
        __syncthreads();
    }
    if (tid != 0) return;
    if (kind == 3) {  // as in warp_branch_plan
        int par = 0;
        for (int w = 0; w < W; w++) {
            su[3][w] = su[1][w] ^ su[2][w];
            sv[3][w] = sv[1][w] ^ sv[2][w];
            par += __popcll(sv[1][w] & su[2][w]) + __popcll(su[1][w] & su[2][w] & sodd[w]);
        }
        epsq[3] = (epsq[1] + epsq[2] + 2 * par) & 3;
    }
    int gid[SF_BR_MAXT];
    int ng = 0;
    for (int j = 0; j < nt; j++) {
        int found = -1;
        for (int j2 = 0; j2 < j; j2++) {
            bool same = true;
            for (int w = 0; w < W; w++) same &= su[j2][w] == su[j][w];
            if (same) { found = gid[j2]; break; }
        }
        gid[j] = found >= 0 ? found : ng++;
    }
    P.ng = ng;
    P.bad = sbad;
    for (int g = 0; g < SF_BR_MAXG; g++) P.nt[g] = 0;
    for (int j = 0; j < nt; j++) {
        const int g = gid[j], t = P.nt[g]++;
        for (int w = 0; w < W; w++) {
            P.u[g][w] = su[j][w];
            P.v[g][t][w] = sv[j][w];
        }
        P.c[g][t] = ipow_mul(tm.c[j], epsq[j]);
    }
    const uint64_t* src = reinterpret_cast<const uint64_t*>(&P);
    uint64_t* dst = d.plan + plan_br(n, W);
    for (size_t e = 0; e < sizeof(BrPlan<W>) / 8; e++) dst[e] = src[e];
}

// the plan of the current diagonal gate in shared memory: computed in place by
// warp 0 (W <= 4) or copied from the planning kernel's output (W >= 8);
// followed by a __syncthreads
template <int W>
__device__ __forceinline__ void get_branch_plan(const SfDev& d, uint32_t kind, uint32_t q0, uint32_t q1,
                                                const SfTerms& tm, BrPlan<W>& P) {
    if constexpr (W >= 8) {
        const uint64_t* src = d.plan + plan_br(d.n, W);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&P);
        for (int e = threadIdx.x; e < (int)(sizeof(BrPlan<W>) / 8); e += blockDim.x) dst[e] = src[e];
    } else {
        if (threadIdx.x < 32) warp_branch_plan<W>(d, kind, q0, q1, tm, P);
    }
    __syncthreads();
}

// coefficient of group g for phase vector s
template <int W>
__device__ __forceinline__ double2 group_coef(const BrPlan<W>& P, int g, const uint64_t* s) {
    double2 cf = make_double2(0.0, 0.0);
    for (int t = 0; t < P.nt[g]; t++) {
        const double sg = (popc_and<W>(P.v[g][t], s) & 1) ? -1.0 : 1.0;
        cf.x += sg * P.c[g][t].x;
        cf.y += sg * P.c[g][t].y;
    }
    return cf;
}

// children of a diagonal gate written out unmerged: child g of element j at
// g * k + j
template <int W>
__global__ void __launch_bounds__(kThreads) k_branch(SfDev d, uint32_t kind, uint32_t q0, uint32_t q1, SfTerms tm,
                                                     int in_buf, int out_buf) {
    __shared__ BrPlan<W> P;
    if (*d.status) return;
    get_branch_plan<W>(d, kind, q0, q1, tm, P);
    if (P.bad) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, in_buf, 23u);
        return;
    }
    const int ng = P.ng;
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
            const double2 cf = group_coef<W>(P, g, s);
            const unsigned long long o = (unsigned long long)g * k + j;
            uint64_t c[W];
#pragma unroll
            for (int w = 0; w < W; w++) c[w] = s[w] ^ P.u[g][w];
            store_sig<W>(So, cap, o, c);
            Ao[o] = cmul(cf, a);
        }
    }
}

// ---------------------------------------------------------------------------
// Slot table.  W = 1: the key word itself is claimed by compare-and-swap
// (all ones = empty, never a phase vector).  W > 1: a state word is claimed
// (empty -> being written), the key is written, then published (ready);
// readers of a slot being written wait for it with a bounded spin.  Keys are
// slot-major (the W words of a slot contiguous): a random insert or compare
// touches one W * 8-byte run instead of W separate sectors.
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

template <int W>
__device__ __forceinline__ bool table_insert(const SfDev& d, unsigned long long T, const uint64_t* key, double2 c) {
    unsigned long long slot = hash_sig<W>(key) & (T - 1);
    for (unsigned long long probe = 0; probe < T; probe++) {
        if constexpr (W == 1) {
            unsigned long long* K = reinterpret_cast<unsigned long long*>(d.tkey);
            unsigned long long cur = *(volatile unsigned long long*)&K[slot];
            if (cur == SF_EMPTY_KEY) cur = atomicCAS(&K[slot], SF_EMPTY_KEY, (unsigned long long)key[0]);
            if (cur == SF_EMPTY_KEY || cur == key[0]) {
                atomicAdd(&d.tacc[slot].x, c.x);
                atomicAdd(&d.tacc[slot].y, c.y);
                return true;
            }
        } else {
            // the key is published by a release store of the state word and read
            // after an acquire load of it; keys are W / 2 16-byte words
            ulonglong2* kv = reinterpret_cast<ulonglong2*>(d.tkey + slot * W);
            uint32_t st = ld_acquire_u32(&d.tstate[slot]);
            if (st == 0) {
                st = atomicCAS(&d.tstate[slot], 0u, 1u);
                if (st == 0) {
#pragma unroll
                    for (int w = 0; w < W / 2; w++) kv[w] = make_ulonglong2(key[2 * w], key[2 * w + 1]);
                    st_release_u32(&d.tstate[slot], 2u);
                    atomicAdd(&d.tacc[slot].x, c.x);
                    atomicAdd(&d.tacc[slot].y, c.y);
                    return true;
                }
            }
            for (int spin = 0; st == 1u && spin < (1 << 22); spin++) st = ld_acquire_u32(&d.tstate[slot]);
            if (st != 2u) return false;
            bool eq = true;
#pragma unroll
            for (int w = 0; w < W / 2; w++) {
                const ulonglong2 v = __ldcg(kv + w);
                eq &= v.x == key[2 * w] && v.y == key[2 * w + 1];
            }
            if (eq) {
                atomicAdd(&d.tacc[slot].x, c.x);
                atomicAdd(&d.tacc[slot].y, c.y);
                return true;
            }
        }
        slot = (slot + 1) & (T - 1);
    }
    return false;
}

// Cofactor children (COFACTOR, Sec. III) of one element from the plan written
// by k_measure_prep: for outcome x, y = x ^ parity(v & sigma); the child starts
// at (tau_y, kappa_y) and the old destabilizers of sigma are applied one at a
// time in the new basis: D_h phi'(t) = eps_h (-1)^{v'_h . t} phi'(t ^ u'_h).
template <int W>
struct CofPlan {
    double2 kap[2];
    uint64_t vq[W], tau[2][W], eps0[W], eps1[W];
};

template <int W>
__device__ __forceinline__ void load_cof_plan(const SfDev& d, CofPlan<W>& C) {
    const int n = d.n;
    const uint64_t* pl = d.plan;
    const size_t ko = cf_kappa(n, W);
    C.kap[0] = make_double2(__longlong_as_double((long long)pl[ko]), __longlong_as_double((long long)pl[ko + 1]));
    C.kap[1] = make_double2(__longlong_as_double((long long)pl[ko + 2]), __longlong_as_double((long long)pl[ko + 3]));
    for (int w = 0; w < W; w++) {
        C.vq[w] = pl[cf_vq(n, W) + w];
        C.tau[0][w] = pl[cf_tau(n, W) + w];
        C.tau[1][w] = pl[cf_tau(n, W) + W + w];
        C.eps0[w] = pl[cf_eps(n, W) + w];
        C.eps1[w] = pl[cf_eps(n, W) + W + w];
    }
}

template <int W>
__device__ __forceinline__ double2 cof_child(const SfDev& d, const CofPlan<W>& C, const uint64_t* s, double2 a,
                                             int x, uint64_t* t) {
    const int n = d.n;
    const uint64_t* U = d.plan + cf_u(n, W);
    const uint64_t* V = d.plan + cf_v(n, W);
    const int y = x ^ (popc_and<W>(C.vq, s) & 1);
#pragma unroll
    for (int w = 0; w < W; w++) t[w] = C.tau[y][w];
    int ip = 0;
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
            ip += (int)((C.eps0[w] >> b) & 1) + 2 * (int)((C.eps1[w] >> b) & 1) + 2 * (popc_and<W>(vv, t) & 1);
#pragma unroll
            for (int u = 0; u < W; u++) t[u] ^= __ldg(&U[(size_t)h * W + u]);
        }
    }
    return ipow_mul(cmul(C.kap[y], a), ip & 3);
}

// Hash every element of in_buf into the slot table, accumulating the
// amplitudes of equal phase vectors (generic COALESCE of a frame that may hold
// repeated phase vectors).  Sets the table size for the compaction and zeroes
// the output count.
template <int W>
__global__ void __launch_bounds__(kThreads) k_insert(SfDev d, int in_buf, int out_buf) {
    if (*d.status) return;
    const unsigned long long k = d.kcnt[in_buf];
    const unsigned long long T = table_size(k, d.tcap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *d.tsize = T;
        d.kcnt[out_buf] = 0;
    }
    const uint64_t* Si = d.sig[in_buf];
    const double2* Ai = d.amp[in_buf];
    const uint64_t cap = d.cap;
    bool ok = true;
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t s[W];
        load_sig<W>(Si, cap, j, s);
        ok &= table_insert<W>(d, T, s, Ai[j]);
    }
    if (!ok) set_status(d.status, SF_ST_TIMEOUT, in_buf);
}

// Emit every occupied slot with |a| >= eps into out_buf (warp-aggregated
// output positions; the order of the frame is not meaningful) and empty the
// slot again, so the table is clean for the next merge.
template <int W>
__global__ void __launch_bounds__(kThreads) k_compact(SfDev d, int out_buf, double eps2) {
    if (*d.status) return;
    const unsigned long long T = *d.tsize;
    // outputs are at most the occupied slots, which are at most T / 2
    const unsigned long long TI = index_slots(T / 2, d.icap);
    const uint32_t tag = next_tag(d.itag[out_buf]);
    bool ok = true;
    const int lane = threadIdx.x & 31;
    const unsigned long long gw = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    uint64_t* So = d.sig[out_buf];
    double2* Ao = d.amp[out_buf];
    const uint64_t cap = d.cap;
    for (unsigned long long base = gw * 32; base < T; base += nw * 32) {
        const unsigned long long i = base + lane;
        bool keep = false;
        uint64_t key[W];
        double2 a = make_double2(0.0, 0.0);
        if (i < T) {
            bool occ;
            if constexpr (W == 1) {
                key[0] = d.tkey[i];
                occ = key[0] != SF_EMPTY_KEY;
            } else {
                occ = d.tstate[i] == 2u;
            }
            if (occ) {
                a = d.tacc[i];
                if constexpr (W > 1) {
                    const ulonglong2* kv = reinterpret_cast<const ulonglong2*>(d.tkey + i * W);
#pragma unroll
                    for (int w = 0; w < W / 2; w++) {
                        const ulonglong2 v = kv[w];
                        key[2 * w] = v.x;
                        key[2 * w + 1] = v.y;
                    }
                    d.tstate[i] = 0u;
                } else {
                    d.tkey[i] = SF_EMPTY_KEY;
                }
                d.tacc[i] = make_double2(0.0, 0.0);
                keep = amp_kept(a, keep_bits(eps2), eps2);
            }
        }
        const unsigned bal = __ballot_sync(SF_FULL, keep);
        if (bal) {
            const int leader = __ffs(bal) - 1;
            unsigned long long b = 0;
            if (lane == leader) b = atomicAdd(&d.kcnt[out_buf], (unsigned long long)__popc(bal));
            b = __shfl_sync(SF_FULL, b, leader);
            if (keep) {
                const unsigned long long o = b + __popc(bal & ((1u << lane) - 1u));
                store_sig<W>(So, cap, o, key);
                Ao[o] = a;
                if constexpr (sf_emit_index(W)) ok &= index_insert<W>(d, out_buf, TI, tag, key, (uint32_t)o);
            }
        }
    }
    if (!ok) set_status(d.status, SF_ST_TIMEOUT, out_buf);
    if (last_block(d.done) && threadIdx.x == 0 && sf_emit_index(W)) {
        d.itag[out_buf] = tag;
        d.isize[out_buf] = TI;
    }
}

// keep the elements whose sign of row meta[1] is x, scaled by 1/sqrt(p_x)
// (collapse after a measurement); kcnt[out_buf] must be zero on entry
// ---------------------------------------------------------------------------
// Toffoli and controlled-R(alpha) by cofactors (Eq. 2, Eq. 3), the step after
// COFACTOR on the two qubits: the rows of M equal to Z_c1 and Z_c2 select the
// elements of the 11 cofactor (sigma bit 1 at both).  kind 0: X_t = eps D^u M^v
// (u_h = [X_t anticommutes with M_h], v_h = [X_t anticommutes with D_h]) maps
// such an element in place to sigma ^ u with the factor eps (-1)^{v.sigma};
// the class maps onto itself, so no two elements meet.  kind 1: the amplitude
// takes e^{i alpha}.
template <int W>
__global__ void __launch_bounds__(kThreads) k_cond(SfDev d, int buf, int kind, int c1, int c2, int t,
                                                   double2 ealpha) {  // e^{i alpha} (kind 1)
    __shared__ int rows[2], epsq, bad;
    __shared__ uint64_t ux[W], vx[W];
    if (*d.status) return;
    const int n = d.n, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        rows[0] = rows[1] = 0x7fffffff;
        bad = 0;
    }
    __syncthreads();
    for (int h = threadIdx.x; h < n; h += blockDim.x) {
        for (int which = 0; which < 2; which++) {
            const int q = which ? c2 : c1;
            bool eq = true;
#pragma unroll
            for (int w = 0; w < W; w++) {
                eq &= d.mx[w * n + h] == 0ull;
                eq &= d.mz[w * n + h] == (((q >> 6) == w) ? (1ull << (q & 63)) : 0ull);
            }
            if (eq) atomicMin(&rows[which], h);
        }
    }
    if (kind == 0 && threadIdx.x < 32) {
        // X_t in the basis (M, D): one warp pass over the rows
        uint64_t um[W], vm[W];
        Pauli<W> p;
        pauli_id<W>(p);
#pragma unroll
        for (int w = 0; w < W; w++) um[w] = vm[w] = 0;
        const int tw = t >> 6;
        const uint64_t tb = 1ull << (t & 63);
        for (int h = lane; h < n; h += 32) {
            const bool ub = (d.mz[tw * n + h] & tb) != 0;
            const bool vb = (d.dz[tw * n + h] & tb) != 0;
            if (ub) {
                Pauli<W> dh;
#pragma unroll
                for (int w = 0; w < W; w++) { dh.x[w] = d.dx[w * n + h]; dh.z[w] = d.dz[w * n + h]; }
                dh.e = (int)d.de[h];
                pauli_mul<W>(p, dh);
                um[h >> 6] |= 1ull << (h & 63);
            }
            if (vb) {
                Pauli<W> mh;
#pragma unroll
                for (int w = 0; w < W; w++) { mh.x[w] = d.mx[w * n + h]; mh.z[w] = d.mz[w * n + h]; }
                mh.e = 0;
                pauli_mul<W>(p, mh);
                vm[h >> 6] |= 1ull << (h & 63);
            }
        }
        warp_pauli_product<W>(p);
        bool ok = true;
#pragma unroll
        for (int w = 0; w < W; w++) {
            um[w] = warp_or(um[w]);
            vm[w] = warp_or(vm[w]);
            ok &= p.x[w] == (w == tw ? tb : 0ull) && p.z[w] == 0ull;
        }
        if (lane == 0) {
#pragma unroll
            for (int w = 0; w < W; w++) { ux[w] = um[w]; vx[w] = vm[w]; }
            epsq = (4 - p.e) & 3;
            bad = ok ? 0 : 1;
        }
    }
    __syncthreads();
    if (rows[0] == 0x7fffffff || rows[1] == 0x7fffffff || bad) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, buf, 28u);
        return;
    }
    const int ru = rows[0], rv = rows[1];
    const double cs = ealpha.x, sn = ealpha.y;
    const unsigned long long k = d.kcnt[buf];
    const uint64_t cap = d.cap;
    uint64_t* S = d.sig[buf];
    double2* A = d.amp[buf];
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t s[W];
        load_sig<W>(S, cap, j, s);
        if (!((s[ru >> 6] >> (ru & 63)) & 1) || !((s[rv >> 6] >> (rv & 63)) & 1)) continue;
        double2 a = A[j];
        if (kind == 0) {
            uint64_t vv[W];
#pragma unroll
            for (int w = 0; w < W; w++) vv[w] = vx[w];
            a = ipow_mul(a, epsq + 2 * (popc_and<W>(vv, s) & 1));
#pragma unroll
            for (int w = 0; w < W; w++) s[w] ^= ux[w];
            store_sig<W>(S, cap, j, s);
        } else {
            a = cmul(a, make_double2(cs, sn));
        }
        A[j] = a;
    }
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_filter(SfDev d, int x, int in_buf, int out_buf) {
    if (*d.status) return;
    const int R = d.meta[1];
    if (R < 0 || R >= d.n) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, in_buf, 25u);
        return;
    }
    const double scale = 1.0 / sqrt(d.out[x]);
    const unsigned long long k = d.kcnt[in_buf];
    const unsigned long long TI = index_slots(k, d.icap);
    const uint32_t tag = next_tag(d.itag[out_buf]);
    bool ok = true;
    const int lane = threadIdx.x & 31;
    const unsigned long long gw = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const uint64_t* Si = d.sig[in_buf];
    uint64_t* So = d.sig[out_buf];
    const uint64_t cap = d.cap;
    for (unsigned long long base = gw * 32; base < k; base += nw * 32) {
        const unsigned long long j = base + lane;
        bool keep = false;
        uint64_t s[W];
        if (j < k) {
            load_sig<W>(Si, cap, j, s);
            // the word of row R loaded once more (an L1 hit): s[R >> 6] would put s
            // in local memory
            keep = (int)((Si[(size_t)(R >> 6) * cap + j] >> (R & 63)) & 1) == x;
        }
        const unsigned bal = __ballot_sync(SF_FULL, keep);
        if (bal) {
            const int leader = __ffs(bal) - 1;
            unsigned long long b = 0;
            if (lane == leader) b = atomicAdd(&d.kcnt[out_buf], (unsigned long long)__popc(bal));
            b = __shfl_sync(SF_FULL, b, leader);
            if (keep) {
                const unsigned long long o = b + __popc(bal & ((1u << lane) - 1u));
                store_sig<W>(So, cap, o, s);
                double2 a = d.amp[in_buf][j];
                a.x *= scale;
                a.y *= scale;
                d.amp[out_buf][o] = a;
                if constexpr (sf_emit_index(W)) ok &= index_insert<W>(d, out_buf, TI, tag, s, (uint32_t)o);
            }
        }
    }
    if (!ok) set_status(d.status, SF_ST_TIMEOUT, out_buf);
    if (last_block(d.done) && threadIdx.x == 0 && sf_emit_index(W)) {
        d.itag[out_buf] = tag;
        d.isize[out_buf] = TI;
    }
}

// ---------------------------------------------------------------------------
// (Re)build the index of buffer b.
template <int W>
__global__ void __launch_bounds__(kThreads) k_build_index(SfDev d, int b) {
    if (*d.status) return;
    const unsigned long long k = d.kcnt[b];
    const unsigned long long TI = index_slots(k, d.icap);
    const uint32_t tag = next_tag(d.itag[b]);
    bool ok = true;
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < k;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t s[W];
        load_sig<W>(d.sig[b], d.cap, j, s);
        ok &= index_insert<W>(d, b, TI, tag, s, (uint32_t)j);
    }
    if (!ok) set_status(d.status, SF_ST_TIMEOUT, b);
    if (last_block(d.done) && threadIdx.x == 0) {
        d.itag[b] = tag;
        d.isize[b] = TI;
    }
}

// Diagonal gate sum_g G_g (G_g the terms with anticommutation mask u_g) with
// merging: the masks form a group U (u_0 = 0), and the children of element s
// are s ^ u_g.  Output tau = s ^ u_g is produced only by its owner, the parent
// s such that no tau ^ u_g' with g' < g is in the frame; its amplitude sums the
// contributions of every parent tau ^ u_g'' found through the index of in_buf,
// in a fixed order.  No amplitude atomics; the output frame is indexed.
template <int W>
__global__ void __launch_bounds__(kThreads) k_branch_merge(SfDev d, uint32_t kind, uint32_t q0, uint32_t q1,
                                                           SfTerms tm, double eps2, int in_buf, int out_buf) {
    __shared__ BrPlan<W> P;
    __shared__ int xidx[SF_BR_MAXG][SF_BR_MAXG];
    __shared__ double2 ctab[SF_BR_MAXG][1 << SF_BR_MAXT];  // group coefficient per sign pattern
    __shared__ unsigned int wsum[kThreads / 32];
    __shared__ unsigned long long bbase;
    if (*d.status) return;
    const unsigned long long k = d.kcnt[in_buf];
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const uint32_t tag_out = next_tag(d.itag[out_buf]);
    // CTAs without elements skip the plan and only take part in the publication
    const bool idle = (unsigned long long)blockIdx.x * blockDim.x >= k && blockIdx.x != 0;
    if (idle) {
        if (last_block(d.done) && threadIdx.x == 0) {
            d.kcnt[out_buf] = *d.ocnt;
            *d.ocnt = 0;
            if (sf_emit_index(W)) {
                d.itag[out_buf] = tag_out;
                d.isize[out_buf] = *d.ipend;
            }
        }
        return;
    }
    get_branch_plan<W>(d, kind, q0, q1, tm, P);
    // xidx[g][g2]: the group whose u is u_g ^ u_g2 (threads 0-15, one entry
    // each); threads 32-95: the coefficient of each group per sign pattern
    int bad = 0;
    if (threadIdx.x < SF_BR_MAXG * SF_BR_MAXG) {
        const int g = threadIdx.x / SF_BR_MAXG, g2 = threadIdx.x % SF_BR_MAXG;
        if (g < P.ng && g2 < P.ng) {
            int m = -1;
            for (int g3 = 0; g3 < P.ng && m < 0; g3++) {
                bool eq = true;
                for (int w = 0; w < W; w++) eq &= (P.u[g][w] ^ P.u[g2][w]) == P.u[g3][w];
                if (eq) m = g3;
            }
            bad = m < 0;
            xidx[g][g2] = m < 0 ? 0 : m;
        }
        if (threadIdx.x == 0)
            for (int w = 0; w < W; w++) bad |= (P.u[0][w] != 0);
    } else if (threadIdx.x >= 32 && threadIdx.x < 32 + SF_BR_MAXG * (1 << SF_BR_MAXT)) {
        const int e = threadIdx.x - 32, g = e >> SF_BR_MAXT, p = e & ((1 << SF_BR_MAXT) - 1);
        if (!P.bad && g < P.ng && p < (1 << P.nt[g])) ctab[g][p] = coef_pattern(P.c[g], P.nt[g], p);
    }
    if (__syncthreads_or(bad) || P.bad) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, in_buf, 26u);
        return;
    }
    const int ng = P.ng;
    const unsigned long long nmax = (unsigned long long)ng * k;
    if (nmax > d.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_CAPACITY, in_buf);
        return;
    }
    const unsigned long long Tin = d.isize[in_buf];
    const uint32_t tag_in = d.itag[in_buf];
    const unsigned long long Tout = index_slots(nmax, d.icap);
    if (blockIdx.x == 0 && threadIdx.x == 0) *d.ipend = Tout;
    const uint64_t* Si = d.sig[in_buf];
    const double2* Ai = d.amp[in_buf];
    uint64_t* So = d.sig[out_buf];
    double2* Ao = d.amp[out_buf];
    const uint64_t cap = d.cap;
    const unsigned long long kb = keep_bits(eps2);
    bool ok = tag_in != 0;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < k; base += stride) {
        const unsigned long long j = base + threadIdx.x;
        const bool act = j < k;
        uint64_t s[W];
        double2 a = make_double2(0.0, 0.0);
        // the loops over groups are unrolled over SF_BR_MAXG with guards, and
        // idx is read through pick_grp, so that idx, amps and s stay in
        // registers (a run-time subscript would put them in local memory)
        long long idx[SF_BR_MAXG];
        idx[0] = act ? (long long)j : -1;
        if (act) {
            load_sig<W>(Si, cap, j, s);
            a = Ai[j];
        } else {
#pragma unroll
            for (int w = 0; w < W; w++) s[w] = 0;
        }
#pragma unroll
        for (int g = 1; g < SF_BR_MAXG; g++)
            idx[g] = (act && g < ng) ? index_find_xor<W>(d, in_buf, Tin, tag_in, s, P.u[g]) : -1;
        double2 amps[SF_BR_MAXG];
        unsigned keepm = 0;
#pragma unroll
        for (int g = 0; g < SF_BR_MAXG; g++) {
            amps[g] = make_double2(0.0, 0.0);
            if (g >= ng) continue;
            bool own = act;
#pragma unroll
            for (int g2 = 0; g2 < g; g2++) own &= pick_grp(idx, xidx[g][g2]) < 0;
            double2 amp = make_double2(0.0, 0.0);
            if (own) {
#pragma unroll
                for (int g2 = 0; g2 < SF_BR_MAXG; g2++) {
                    if (g2 >= ng) continue;
                    const int m = xidx[g][g2];
                    const long long im = pick_grp(idx, m);
                    if (im < 0) continue;
                    const double2 ap = m == 0 ? a : Ai[im];
                    int pat = 0;  // sign pattern of the parent tau ^ u_g2 = s ^ u_m
                    for (int t = 0; t < P.nt[g2]; t++) {
                        int c = 0;
#pragma unroll
                        for (int w = 0; w < W; w++) c += __popcll(P.v[g2][t][w] & (s[w] ^ P.u[m][w]));
                        pat |= (c & 1) << t;
                    }
                    cmul_acc(amp, ctab[g2][pat], ap);
                }
            }
            amps[g] = amp;
            if (own && amp_kept(amp, kb, eps2)) keepm |= 1u << g;
        }
        // one reservation per iteration for all kept outputs of the block
        unsigned long long o = block_out_range(d.ocnt, __popc(keepm), wsum, &bbase);
#pragma unroll
        for (int g = 0; g < SF_BR_MAXG; g++) {
            if (!((keepm >> g) & 1u)) continue;
            if constexpr (sf_emit_index(W)) {
                uint64_t tau[W];
#pragma unroll
                for (int w = 0; w < W; w++) tau[w] = s[w] ^ P.u[g][w];
                store_sig<W>(So, cap, o, tau);
                ok &= index_insert<W>(d, out_buf, Tout, tag_out, tau, (uint32_t)o);
            } else {
#pragma unroll
                for (int w = 0; w < W; w++) So[(size_t)w * cap + o] = s[w] ^ *(const volatile uint64_t*)&P.u[g][w];
            }
            Ao[o] = amps[g];
            o++;
        }
    }
    if (!ok) set_status(d.status, SF_ST_TIMEOUT, in_buf);
    if (last_block(d.done) && threadIdx.x == 0) {
        d.kcnt[out_buf] = *d.ocnt;
        *d.ocnt = 0;
        if (sf_emit_index(W)) {
            d.itag[out_buf] = tag_out;
            d.isize[out_buf] = *d.ipend;
        }
    }
}

// Cofactor split with merging (COFACTOR, Sec. III): elements s and s ^ uq
// (uq: rows of the old tableau anticommuting with Z_q) have the same two
// cofactor children; the one with the smaller phase vector emits both, summing
// the two contributions.
template <int W>
__device__ __forceinline__ bool sig_less(const uint64_t* a, const uint64_t* b) {
#pragma unroll
    for (int w = W - 1; w >= 0; w--)
        if (a[w] != b[w]) return a[w] < b[w];
    return false;
}

// Closed form of the cofactor children for W >= 8.  cof_child walks the set
// bits h of sigma in increasing order: t starts at tau_y, each h adds
// eps_h + 2 [V_h . t] to the i-power and then XORs U_h into t.  With the
// measurement's row sort rho split off, U_h = e_{rho(h)} ^ sum_i CU[h][i] B_i,
// and V'_h = rho^{-1}(V_h) = sum_j CV[h][j] F_j (cta_lowrank):
//   t = tau_y ^ t0,  t0 = rho(sigma) ^ sum_i parity(sigma & cu_i) B_i,
//   ip = |sigma & eps0| + 2 |sigma & eps1| + 2 (parity(sigma & omega_y) ^ Q),
// where omega_y[h] = V_h . tau_y = sum_j (rho(F_j) . tau_y) cv_j[h] and the
// ordered part Q = sum_{h in sigma} V_h . (sum_{h' in sigma, h' < h} U_h') is,
// with K_j = F_j ^ sum_i (rho(F_j) . B_i) cu_i (V_h . rho(x) = V'_h . x),
//   Q = sum_j parity(sigma & cv_j & xpp(sigma & K_j)),
// xpp(b)[h] the parity of the bits of b below h.  k_cof_lowrank writes K_j and
// omega_y; the U block's rank word reads SF_LR_NONE when the move list or
// either rank is over its limit (the dense kernel runs then).
template <int W>
__global__ void __launch_bounds__(1024) k_cof_lowrank(SfDev d) {
    __shared__ int G[SF_LR_MAX][SF_LR_MAX], ft[SF_LR_MAX][2];
    __shared__ uint64_t Fr[SF_LR_MAX][W];
    __shared__ Moves M;
    if (*d.status) return;
    if (!d.meta[2]) return;
    const int n = d.n, tid = threadIdx.x;
    uint64_t* pl = d.plan;
    uint64_t* LU = pl + plan_lr_u(n, W);
    uint64_t* LV = pl + plan_lr_v(n, W);
    if (!d.lowrank || pl[plan_mv_cf(n, W)] > SF_MV_MAX) {
        if (tid == 0) {
            LU[0] = SF_LR_NONE;
            LV[0] = SF_LR_NONE;
        }
        return;
    }
    load_moves(pl + plan_mv_cf(n, W), M);
    __syncthreads();
    uint64_t x[W];
#pragma unroll
    for (int w = 0; w < W; w++) x[w] = tid < n ? pl[cf_u(n, W) + (size_t)tid * W + w] : 0ull;
    if (tid < n) {
        const int p = (int)reinterpret_cast<const uint32_t*>(pl + plan_rho_cf(n, W))[tid];
#pragma unroll
        for (int w = 0; w < W; w++)
            if (w == (p >> 6)) x[w] ^= 1ull << (p & 63);
    }
    const int ru = cta_lowrank<W>(x, n, LU);
#pragma unroll
    for (int w = 0; w < W; w++) x[w] = tid < n ? pl[cf_v(n, W) + (size_t)tid * W + w] : 0ull;
    apply_moves_inv<W>(x, M);
    const int rv = cta_lowrank<W>(x, n, LV);
    if (ru < 0 || rv < 0) {
        if (tid == 0) LU[0] = SF_LR_NONE;
        return;
    }
    if (tid < rv) {  // rho(F_j)
        uint64_t f[W];
#pragma unroll
        for (int w = 0; w < W; w++) f[w] = LV[lr_B(W) + (size_t)tid * W + w];
        apply_moves<W>(f, M);
#pragma unroll
        for (int w = 0; w < W; w++) Fr[tid][w] = f[w];
    }
    __syncthreads();
    for (int e = tid; e < rv * ru; e += blockDim.x) {
        const int j = e / ru, i = e % ru;
        G[j][i] = popc_and<W>(Fr[j], LU + lr_B(W) + (size_t)i * W) & 1;
    }
    for (int e = tid; e < 2 * rv; e += blockDim.x) {
        const int j = e >> 1, y = e & 1;
        ft[j][y] = popc_and<W>(Fr[j], pl + cf_tau(n, W) + (size_t)y * W) & 1;
    }
    __syncthreads();
    for (int e = tid; e < rv * W; e += blockDim.x) {
        const int j = e / W, w = e % W;
        uint64_t k = LV[lr_B(W) + (size_t)j * W + w];
        for (int i = 0; i < ru; i++)
            if (G[j][i]) k ^= LU[lr_C(W) + (size_t)i * W + w];
        pl[plan_cf_k(n, W) + (size_t)j * W + w] = k;
    }
    for (int e = tid; e < 2 * W; e += blockDim.x) {
        const int y = e / W, w = e % W;
        uint64_t o = 0ull;
        for (int j = 0; j < rv; j++)
            if (ft[j][y]) o ^= LV[lr_C(W) + (size_t)j * W + w];
        pl[plan_cf_om(n, W) + (size_t)y * W + w] = o;
    }
    // An element s and its partner s ^ uq have the same children: child x of
    // the partner has y' = y ^ c (c = parity(vq & uq)) and t0 shifted by
    // U uq = rho(uq) ^ sum_i parity(uq & cu_i) B_i, so tau_{y^c} ^ tau_y must
    // equal U uq.  Checked once here; k_cof_merge then takes the element's
    // children for both.
    if (tid == 0) {
        const uint64_t* uq = pl + cf_uq(n, W);
        const uint64_t* vq = pl + cf_vq(n, W);
        const uint64_t* tau = pl + cf_tau(n, W);
        const int c = popc_and<W>(vq, uq) & 1;
        uint32_t sel = 0;
        for (int i = 0; i < ru; i++) sel |= (uint32_t)(popc_and<W>(LU + lr_C(W) + (size_t)i * W, uq) & 1) << i;
        uint64_t u[W];
        for (int w = 0; w < W; w++) u[w] = uq[w];
        apply_moves<W>(u, M);
        bool ok = true;
        for (int w = 0; w < W; w++) {
            for (int i = 0; i < ru; i++)
                if ((sel >> i) & 1u) u[w] ^= LU[lr_B(W) + (size_t)i * W + w];
            ok &= (c ? (tau[w] ^ tau[W + w]) : 0ull) == u[w];
        }
        if (!ok) set_status(d.status, SF_ST_INTERNAL, 0, 27u);
    }
}

template <int W>
struct CofLR {
    double2 kap[2];
    int ru, rv;
    Moves M;
    uint64_t vq[W], eps0[W], eps1[W], tau[2][W], om[2][W];
    uint64_t B[SF_LR_MAX][W], cu[SF_LR_MAX][W], cv[SF_LR_MAX][W], K[SF_LR_MAX][W];
};

template <int W>
__device__ void load_cof_lr(const SfDev& d, CofLR<W>& C) {
    const int n = d.n, tid = threadIdx.x;
    const uint64_t* pl = d.plan;
    const uint64_t* LU = pl + plan_lr_u(n, W);
    const uint64_t* LV = pl + plan_lr_v(n, W);
    const int ru = (int)LU[0], rv = (int)LV[0];
    if (tid == 0) {
        C.ru = ru;
        C.rv = rv;
        const size_t ko = cf_kappa(n, W);
        C.kap[0] = make_double2(__longlong_as_double((long long)pl[ko]), __longlong_as_double((long long)pl[ko + 1]));
        C.kap[1] = make_double2(__longlong_as_double((long long)pl[ko + 2]), __longlong_as_double((long long)pl[ko + 3]));
    }
    load_moves(pl + plan_mv_cf(n, W), C.M);
    if (tid < W) {
        C.vq[tid] = pl[cf_vq(n, W) + tid];
        C.eps0[tid] = pl[cf_eps(n, W) + tid];
        C.eps1[tid] = pl[cf_eps(n, W) + W + tid];
        for (int y = 0; y < 2; y++) {
            C.tau[y][tid] = pl[cf_tau(n, W) + y * W + tid];
            C.om[y][tid] = pl[plan_cf_om(n, W) + y * W + tid];
        }
    }
    for (int e = tid; e < ru * W; e += blockDim.x) {
        C.B[e / W][e % W] = LU[lr_B(W) + e];
        C.cu[e / W][e % W] = LU[lr_C(W) + e];
    }
    for (int e = tid; e < rv * W; e += blockDim.x) {
        C.cv[e / W][e % W] = LV[lr_C(W) + e];
        C.K[e / W][e % W] = pl[plan_cf_k(n, W) + e];
    }
}

// the y-independent scalars of the closed form for phase vector s ^ m
// (m = 0 for the element itself, uq for its partner)
struct CofScal {
    int pq, pe, pw[2], q;
};

// |a & b| with a read from shared memory at every use (volatile), so that the
// plan's loop-invariant vectors are not hoisted into registers across the
// element loop (seven of them would take 224 registers at W = 16)
template <int W>
__device__ __forceinline__ int popc_and_sh(const uint64_t* a, const uint64_t* b) {
    int c = 0;
#pragma unroll
    for (int w = 0; w < W; w++) c += __popcll(*(const volatile uint64_t*)&a[w] & b[w]);
    return c;
}

template <int W>
__device__ __forceinline__ void cof_scalars(const CofLR<W>& C, const uint64_t* s, const uint64_t* m, CofScal& E) {
    uint64_t v[W];
#pragma unroll
    for (int w = 0; w < W; w++) v[w] = m ? s[w] ^ *(const volatile uint64_t*)&m[w] : s[w];
    E.pq = popc_and_sh<W>(C.vq, v) & 1;
    E.pe = popc_and_sh<W>(C.eps0, v) + 2 * popc_and_sh<W>(C.eps1, v);
    E.pw[0] = popc_and_sh<W>(C.om[0], v) & 1;
    E.pw[1] = popc_and_sh<W>(C.om[1], v) & 1;
    int q = 0;
#pragma unroll 1
    for (int j = 0; j < C.rv; j++) {
        uint64_t carry = 0ull;  // all ones when the bits of v & K_j in lower words have odd parity
        int cnt = 0;
#pragma unroll
        for (int w = 0; w < W; w++) {
            const uint64_t b = v[w] & C.K[j][w];
            uint64_t x = b;  // inclusive prefix parity within the word
            x ^= x << 1;
            x ^= x << 2;
            x ^= x << 4;
            x ^= x << 8;
            x ^= x << 16;
            x ^= x << 32;
            cnt += __popcll(v[w] & C.cv[j][w] & ((x << 1) ^ carry));
            carry ^= (x >> 63) ? ~0ull : 0ull;
        }
        q ^= cnt & 1;
    }
    E.q = q;
}

// t0 = rho(s) ^ sum_i parity(s & cu_i) B_i, in place
template <int W>
__device__ __forceinline__ void cof_t0(const CofLR<W>& C, uint64_t* s) {
    uint32_t sel = 0;
#pragma unroll 1
    for (int i = 0; i < C.ru; i++) sel |= (uint32_t)(popc_and<W>(C.cu[i], s) & 1) << i;
    apply_moves<W>(s, C.M);
#pragma unroll 1
    for (int i = 0; i < C.ru; i++) {
        if ((sel >> i) & 1u) {
#pragma unroll
            for (int w = 0; w < W; w++) s[w] ^= C.B[i][w];
        }
    }
}

// amplitude of child x (y = x ^ pq) of an element with scalars E and amplitude a
template <int W>
__device__ __forceinline__ double2 cof_amp_lr(const CofLR<W>& C, const CofScal& E, double2 a, int x) {
    const int y = x ^ E.pq;
    const int ip = E.pe + 2 * (E.pw[y] ^ E.q);
    return ipow_mul(cmul(C.kap[y], a), ip & 3);
}

// The partner's scalars from the element's.  Every scalar of the closed form
// is linear in the phase vector v except the ordered part Q, which is a sum of
// bilinear forms f_j(a, b) = parity(a & cv_j & xpp(b & K_j)) at a = b = v, so
// for v = s ^ u
//   Q(s ^ u) = Q(s) ^ Q(u) ^ parity(s & Wu),
//   Wu = sum_j [cv_j & xpp(u & K_j)  ^  K_j & spp(u & cv_j)],
// with xpp (spp) the parity of the bits strictly below (above) each bit: the
// second term is f_j(u, s) rewritten by exchanging the two sums over bits.
// The count |(s ^ u) & eps0| is |s & eps0| + |u & eps0| - 2 |s & u & eps0|.
template <int W>
struct CofPart {
    uint64_t wu[W], ue0[W];
    int qu, pqu, peu, pwu[2];
};

// warp 0: the per-mask constants of the partner rule for u = uq
template <int W>
__device__ __noinline__ void cof_partner_setup(const CofLR<W>& C, const uint64_t* u, CofPart<W>& P) {
    const int lane = threadIdx.x & 31;
    uint64_t acc[W];
#pragma unroll
    for (int w = 0; w < W; w++) acc[w] = 0ull;
    int qj = 0;
    if (lane < C.rv) {
        const int j = lane;
        uint64_t carry = 0ull;  // parity of the lower words of u & K_j, as a full word
#pragma unroll
        for (int w = 0; w < W; w++) {
            uint64_t x = u[w] & C.K[j][w];  // inclusive prefix parity within the word
            x ^= x << 1;
            x ^= x << 2;
            x ^= x << 4;
            x ^= x << 8;
            x ^= x << 16;
            x ^= x << 32;
            const uint64_t xp = (x << 1) ^ carry;  // strictly below
            acc[w] ^= C.cv[j][w] & xp;
            qj ^= __popcll(u[w] & C.cv[j][w] & xp) & 1;
            carry ^= (x >> 63) ? ~0ull : 0ull;
        }
        carry = 0ull;  // parity of the higher words of u & cv_j
#pragma unroll
        for (int w = W - 1; w >= 0; w--) {
            uint64_t y = u[w] & C.cv[j][w];  // inclusive suffix parity within the word
            y ^= y >> 1;
            y ^= y >> 2;
            y ^= y >> 4;
            y ^= y >> 8;
            y ^= y >> 16;
            y ^= y >> 32;
            const uint64_t sp = (y >> 1) ^ carry;  // strictly above
            acc[w] ^= C.K[j][w] & sp;
            carry ^= (y & 1ull) ? ~0ull : 0ull;
        }
    }
#pragma unroll
    for (int w = 0; w < W; w++) {
        const unsigned lo = __reduce_xor_sync(SF_FULL, (unsigned)acc[w]);
        const unsigned hi = __reduce_xor_sync(SF_FULL, (unsigned)(acc[w] >> 32));
        if (lane == 0) {
            P.wu[w] = (uint64_t)lo | ((uint64_t)hi << 32);
            P.ue0[w] = u[w] & C.eps0[w];
        }
    }
    const int q = __reduce_xor_sync(SF_FULL, (unsigned)qj) & 1;
    if (lane == 0) {
        P.qu = q;
        P.pqu = popc_and<W>(C.vq, u) & 1;
        P.peu = (popc_and<W>(C.eps0, u) + 2 * popc_and<W>(C.eps1, u)) & 3;
        P.pwu[0] = popc_and<W>(C.om[0], u) & 1;
        P.pwu[1] = popc_and<W>(C.om[1], u) & 1;
    }
}

// the partner's scalars (v = s ^ u) from the element's (v = s)
template <int W>
__device__ __forceinline__ void cof_scalars_partner(const CofPart<W>& P, const uint64_t* s, const CofScal& es,
                                                    CofScal& ep) {
    ep.pq = es.pq ^ P.pqu;
    ep.pe = es.pe + P.peu + 2 * (popc_and_sh<W>(P.ue0, s) & 1);
    ep.pw[0] = es.pw[0] ^ P.pwu[0];
    ep.pw[1] = es.pw[1] ^ P.pwu[1];
    ep.q = es.q ^ P.qu ^ (popc_and_sh<W>(P.wu, s) & 1);
}

template <int W, bool LR>
__global__ void __launch_bounds__(kThreads, LR ? 2 : 1) k_cof_merge(SfDev d, double eps2, int in_buf, int out_buf) {
    using Plan = typename std::conditional<LR, CofLR<W>, CofPlan<W>>::type;
    __shared__ Plan CP;
    __shared__ uint64_t uq[W];
    __shared__ unsigned int wsum[kThreads / 32];
    __shared__ unsigned long long bbase;
    __shared__ CofPart<W> PP;  // LR: the partner rule's constants
    if (*d.status) return;
    if (!d.meta[2]) return;
    if constexpr (W >= 8) {
        // exactly one of the two variants runs
        if ((d.plan[plan_lr_u(d.n, W)] <= SF_LR_MAX) != LR) return;
    }
    if constexpr (LR) {
        load_cof_lr<W>(d, CP);
        if (threadIdx.x < W) uq[threadIdx.x] = d.plan[cf_uq(d.n, W) + threadIdx.x];
        __syncthreads();
        if (threadIdx.x < 32) cof_partner_setup<W>(CP, uq, PP);
    } else if (threadIdx.x == 0) {
        load_cof_plan<W>(d, CP);
        for (int w = 0; w < W; w++) uq[w] = d.plan[cf_uq(d.n, W) + w];
    }
    __syncthreads();
    const unsigned long long k = d.kcnt[in_buf];
    if (2 * k > d.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_CAPACITY, in_buf);
        return;
    }
    const unsigned long long Tin = d.isize[in_buf];
    const uint32_t tag_in = d.itag[in_buf];
    const unsigned long long Tout = index_slots(2 * k, d.icap);
    const uint32_t tag_out = next_tag(d.itag[out_buf]);
    const uint64_t* Si = d.sig[in_buf];
    const double2* Ai = d.amp[in_buf];
    uint64_t* So = d.sig[out_buf];
    double2* Ao = d.amp[out_buf];
    const uint64_t cap = d.cap;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long kb = keep_bits(eps2);
    bool ok = tag_in != 0;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < k; base += stride) {
        const unsigned long long j = base + threadIdx.x;
        const bool act = j < k;
        uint64_t s[W], p[W];
        double2 a = make_double2(0.0, 0.0), ap = make_double2(0.0, 0.0);
        long long l = -1;
        bool own = false;
        if (act) {
            load_sig<W>(Si, cap, j, s);
            a = Ai[j];
#pragma unroll
            for (int w = 0; w < W; w++) p[w] = s[w] ^ uq[w];
            l = index_find<W>(d, in_buf, Tin, tag_in, p);
            own = l < 0 || sig_less<W>(s, p);
            if (l >= 0) ap = Ai[l];
        }
        double2 cc[2];
        unsigned keepm = 0;
        if constexpr (LR) {
            // the partner's children are the element's (checked on the plan by
            // k_cof_lowrank); only their amplitudes differ
            CofScal es, ep;
            if (own) {
                cof_scalars<W>(CP, s, nullptr, es);
                if (l >= 0) cof_scalars_partner<W>(PP, s, es, ep);
                cof_t0<W>(CP, s);  // s now holds t0; the child x is tau_{x ^ pq} ^ t0
            }
            for (int x = 0; x < 2; x++) {
                double2 c = make_double2(0.0, 0.0);
                if (own) {
                    c = cof_amp_lr<W>(CP, es, a, x);
                    if (l >= 0) {
                        const double2 c2 = cof_amp_lr<W>(CP, ep, ap, x);
                        c.x += c2.x;
                        c.y += c2.y;
                    }
                }
                cc[x] = c;
                if (own && amp_kept(c, kb, eps2)) keepm |= 1u << x;
            }
            unsigned long long o = block_out_range(d.ocnt, __popc(keepm), wsum, &bbase);
#pragma unroll 1
            for (int x = 0; x < 2; x++) {
                if (!((keepm >> x) & 1u)) continue;
                const int y = x ^ es.pq;
                uint64_t t[W];
#pragma unroll
                for (int w = 0; w < W; w++) t[w] = *(const volatile uint64_t*)&CP.tau[y][w] ^ s[w];
                store_sig<W>(So, cap, o, t);
                Ao[o] = cc[x];
                if constexpr (sf_emit_index(W)) ok &= index_insert<W>(d, out_buf, Tout, tag_out, t, (uint32_t)o);
                o++;
            }
        } else {
        uint64_t t[2][W];
        for (int x = 0; x < 2; x++) {
            double2 c = make_double2(0.0, 0.0);
            if (own) {
                c = cof_child<W>(d, CP, s, a, x, t[x]);
                if (l >= 0) {
                    uint64_t t2[W];
                    const double2 c2 = cof_child<W>(d, CP, p, ap, x, t2);
                    bool same = true;
#pragma unroll
                    for (int w = 0; w < W; w++) same &= t2[w] == t[x][w];
                    if (!same) set_status(d.status, SF_ST_INTERNAL, in_buf, 27u);
                    c.x += c2.x;
                    c.y += c2.y;
                }
            }
            cc[x] = c;
            if (own && amp_kept(c, kb, eps2)) keepm |= 1u << x;
        }
        unsigned long long o = block_out_range(d.ocnt, __popc(keepm), wsum, &bbase);
        for (int x = 0; x < 2; x++) {
            if (!((keepm >> x) & 1u)) continue;
            store_sig<W>(So, cap, o, t[x]);
            Ao[o] = cc[x];
            if constexpr (sf_emit_index(W)) ok &= index_insert<W>(d, out_buf, Tout, tag_out, t[x], (uint32_t)o);
            o++;
        }
        }
    }    if (!ok) set_status(d.status, SF_ST_TIMEOUT, in_buf);
    if (last_block(d.done) && threadIdx.x == 0) {
        d.kcnt[out_buf] = *d.ocnt;
        *d.ocnt = 0;
        if (sf_emit_index(W)) {
            d.itag[out_buf] = tag_out;
            d.isize[out_buf] = Tout;
        }
    }
}

// Cofactor split with merging on a frame whose layout the grid program left
// known (n <= 63): element j is s_0 ^ (XOR of u[i] over the set bits of j), so
// the partner s ^ uq of element j sits at j ^ c when uq = XOR of u[i] over the
// set bits of c, and no element has a partner when uq lies outside the span of
// the u[i].  No index is read or written, and the work goes by pairs (one
// thread per pair, so no lane idles through the double-precision pipe).
// The children are those of cof_child, rewritten: with P the XOR of U_h over
// the set bits of sigma, t = tau_y ^ P, and the i-power
//   ip_y = |sigma & eps0| + 2 |sigma & eps1| + 2 (parity(sigma & omega_y) ^ Q),
// omega_y[h] = V_h . tau_y, Q = sum over set bits h of V_h . (XOR of U_h'
// over the set bits h' < h) -- one walk over the bits serves both outcomes.
// kappa_y = sc i^{e_y} (a real scale times an i-power, as the measurement
// prep builds it), so a child amplitude is sc i^{e_y + ip_y} a: an exact
// rotation, the partners' two summed, then one real scaling.  Does nothing
// when the layout is not known (the host checks that before it launches it).
// With prob set it also does what k_prob does: per CTA, the summed |a|^2 of
// the children it keeps, split by their bit on row meta[1] (the measured
// qubit's row), summed over the grid by the last CTA into d.out[0..1].
__global__ void __launch_bounds__(kThreads) k_cof_pos(SfDev d, double eps2, int in_buf, int out_buf, int prob) {
    __shared__ uint64_t sU[64], sV[64];
    __shared__ unsigned int wsum[kThreads / 32];
    __shared__ unsigned long long bbase, s_c, s_om[2];
    __shared__ int s_span, s_e[2];
    __shared__ double s_sc;
    __shared__ double shp[2][32];
    if (*d.status) return;
    if (!d.meta[2]) return;
    const GpLayout* L = reinterpret_cast<const GpLayout*>(d.gp);
    if (!L->ok) return;
    const int n = d.n;
    const int R = d.meta[1];
    if (prob && (R < 0 || R >= n)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, in_buf, 21u);
        return;
    }
    const uint64_t* pl = d.plan;
    const uint64_t uq = pl[cf_uq(n, 1)], vq = pl[cf_vq(n, 1)];
    const uint64_t eps0 = pl[cf_eps(n, 1)], eps1 = pl[cf_eps(n, 1) + 1];
    const uint64_t tau[2] = {pl[cf_tau(n, 1)], pl[cf_tau(n, 1) + 1]};
    if (threadIdx.x < 64) {
        const int h = threadIdx.x;
        sU[h] = h < n ? pl[cf_u(n, 1) + h] : 0ull;
        sV[h] = h < n ? pl[cf_v(n, 1) + h] : 0ull;
    }
    if (threadIdx.x == 33) s_om[0] = s_om[1] = 0ull;
    if (threadIdx.x == 32) {  // kappa_y = sc i^{e_y}
        bool ok = true;
        double sc = 0.0;
        for (int y = 0; y < 2; y++) {
            const size_t ko = cf_kappa(n, 1) + 2 * y;
            const double kx = __longlong_as_double((long long)pl[ko]), ky = __longlong_as_double((long long)pl[ko + 1]);
            ok &= (kx == 0.0) != (ky == 0.0);
            s_e[y] = kx > 0.0 ? 0 : (ky > 0.0 ? 1 : (kx < 0.0 ? 2 : 3));
            const double m = fabs(kx) + fabs(ky);
            ok &= y == 0 || m == sc;
            sc = m;
        }
        s_sc = sc;
        if (!ok) set_status(d.status, SF_ST_INTERNAL, in_buf, 29u);
    }
    __syncthreads();
    if (threadIdx.x < 64) {  // omega_y
        const int h = threadIdx.x;
        const bool o0 = (__popcll(sV[h] & tau[0]) & 1) != 0, o1 = (__popcll(sV[h] & tau[1]) & 1) != 0;
        const unsigned b0 = __ballot_sync(SF_FULL, o0), b1 = __ballot_sync(SF_FULL, o1);
        if ((h & 31) == 0) {
            atomicOr(&s_om[0], (unsigned long long)b0 << h);
            atomicOr(&s_om[1], (unsigned long long)b1 << h);
        }
    }
    if (threadIdx.x < 32) {
        // uq in the basis u[0..m): Gauss-Jordan over the bit columns (lane i
        // holds u[i] and u[i + 32] with their combinations), then uq reduced
        const int lane = threadIdx.x, m = (int)L->n;
        uint64_t v[2] = {lane < m ? L->u[lane] : 0ull, lane + 32 < m ? L->u[lane + 32] : 0ull};
        uint64_t cmb[2] = {lane < m ? 1ull << lane : 0ull, lane + 32 < m ? 1ull << (lane + 32) : 0ull};
        bool used[2] = {false, false};
        uint64_t x = uq, cx = 0;
        for (int b = 0; b < 64; b++) {
            const bool h0 = !used[0] && ((v[0] >> b) & 1), h1 = !used[1] && ((v[1] >> b) & 1);
            const unsigned b0 = __ballot_sync(SF_FULL, h0), b1 = __ballot_sync(SF_FULL, h1);
            if (!(b0 | b1)) continue;
            const int p = b0 ? __ffs(b0) - 1 : 32 + __ffs(b1) - 1;
            const uint64_t pv = __shfl_sync(SF_FULL, p < 32 ? v[0] : v[1], p & 31);
            const uint64_t pc = __shfl_sync(SF_FULL, p < 32 ? cmb[0] : cmb[1], p & 31);
            for (int hf = 0; hf < 2; hf++) {
                const int idx = lane + 32 * hf;
                if (idx == p) used[hf] = true;
                else if ((v[hf] >> b) & 1) {
                    v[hf] ^= pv;
                    cmb[hf] ^= pc;
                }
            }
            if ((x >> b) & 1) {
                x ^= pv;
                cx ^= pc;
            }
        }
        if (lane == 0) {
            s_span = x == 0 && cx != 0;
            s_c = cx;
        }
    }
    __syncthreads();
    const unsigned long long k = d.kcnt[in_buf];
    const bool span = s_span != 0 && (s_c >> L->n) == 0;
    const unsigned long long cmask = s_c;
    if (!span && 2 * k > d.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_CAPACITY, in_buf);
        return;
    }
    const int bl = span ? __ffsll((long long)cmask) - 1 : 0;  // pairs: the element with bit bl clear
    const unsigned long long units = span ? k / 2 : k;
    const uint64_t om0 = s_om[0], om1 = s_om[1];
    const int e0 = s_e[0], e1 = s_e[1];
    const double sc = s_sc;
    const uint64_t* Si = d.sig[in_buf];
    const double2* Ai = d.amp[in_buf];
    uint64_t* So = d.sig[out_buf];
    double2* Ao = d.amp[out_buf];
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long kb = keep_bits(eps2);
    // the walk over the set bits of an element: P and Q
    auto walk = [&](uint64_t x, uint64_t& P, int& Q) {
        P = 0;
        Q = 0;
        while (x) {
            const int h = __ffsll((long long)x) - 1;
            x &= x - 1;
            Q ^= __popcll(sV[h] & P) & 1;
            P ^= sU[h];
        }
    };
    // exponent of child x of element x_el (walk P, Q): y and e_y + ip_y
    auto expo = [&](uint64_t el, int Q, int x, int& y) {
        y = x ^ (__popcll(vq & el) & 1);
        const int pw = __popcll(el & (y ? om1 : om0)) & 1;
        return (y ? e1 : e0) + __popcll(el & eps0) + 2 * __popcll(el & eps1) + 2 * (pw ^ Q);
    };
    bool bad = false;
    double pr[2] = {0.0, 0.0};
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < units; base += stride) {
        const unsigned long long m = base + threadIdx.x;
        const bool act = m < units;
        unsigned keepm = 0;
        uint64_t t[2] = {0, 0};
        double2 cc[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
        if (act) {
            unsigned long long j = m, pj = 0;
            if (span) {
                j = ((m >> bl) << (bl + 1)) | (m & ((1ull << bl) - 1ull));
                pj = j ^ cmask;
            }
            uint64_t s0 = Si[j];
            double2 a0 = Ai[j];
            uint64_t s1 = 0;
            double2 a1 = make_double2(0.0, 0.0);
            if (span) {
                s1 = Si[pj];
                a1 = Ai[pj];
                bad |= s1 != (s0 ^ uq);  // the layout says the partner is there
                if (s1 < s0) {  // the owner (smaller phase vector) first, as in k_cof_merge
                    const uint64_t ts = s0; s0 = s1; s1 = ts;
                    const double2 ta = a0; a0 = a1; a1 = ta;
                }
            }
            uint64_t P0, P1 = 0;
            int Q0, Q1 = 0;
            walk(s0, P0, Q0);
            if (span) walk(s1, P1, Q1);
#pragma unroll
            for (int x = 0; x < 2; x++) {
                int y0, y1 = 0;
                const int m0 = expo(s0, Q0, x, y0);
                t[x] = tau[y0] ^ P0;
                double2 z = ipow_mul(a0, m0 & 3);
                if (span) {
                    const int m1 = expo(s1, Q1, x, y1);
                    bad |= (tau[y1] ^ P1) != t[x];
                    const double2 z1 = ipow_mul(a1, m1 & 3);
                    z.x += z1.x;
                    z.y += z1.y;
                }
                cc[x] = make_double2(sc * z.x, sc * z.y);
                if (amp_kept(cc[x], kb, eps2)) keepm |= 1u << x;
            }
        }
        unsigned long long o = block_out_range(d.ocnt, __popc(keepm), wsum, &bbase);
        for (int x = 0; x < 2; x++) {
            if (!((keepm >> x) & 1u)) continue;
            So[o] = t[x];
            Ao[o] = cc[x];
            o++;
            pr[(t[x] >> (R & 63)) & 1] += cc[x].x * cc[x].x + cc[x].y * cc[x].y;
        }
    }
    if (bad) set_status(d.status, SF_ST_INTERNAL, in_buf, 28u);
    if (prob) {
        block_sum<2>(pr, shp);
        if (threadIdx.x == 0) {
            d.red[2 * blockIdx.x] = pr[0];
            d.red[2 * blockIdx.x + 1] = pr[1];
        }
    }
    if (last_block(d.done)) {
        if (threadIdx.x == 0) {
            d.kcnt[out_buf] = *d.ocnt;
            *d.ocnt = 0;
        }
        if (prob) reduce_partials(d, 0, shp);
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
    // four elements of the thread's grid-stride sequence per round, their
    // loads in flight together (the sums keep the sequence's order)
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long j0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j0 < k;
         j0 += 4 * stride) {
        double2 av[4];
        uint64_t pw[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const unsigned long long j = j0 + u * stride;
            av[u] = j < k ? A[j] : make_double2(0.0, 0.0);
            pw[u] = j < k ? plane[j] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (j0 + u * stride >= k) break;
            const double m = av[u].x * av[u].x + av[u].y * av[u].y;
            if ((pw[u] >> (R & 63)) & 1) p[1] += m;
            else p[0] += m;
        }
    }
    block_sum<2>(p, sh);
    if (threadIdx.x == 0) {
        d.red[2 * blockIdx.x] = p[0];
        d.red[2 * blockIdx.x + 1] = p[1];
    }
    if (last_block(d.done)) reduce_partials(d, 0, sh);
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
    if constexpr (W == 1) {
        // The two Pauli products of elem_amp_phi by 4-bit chunks, tabulated once
        // per CTA: DT[c][v] = the product of D_h over the set bits h = 4c + b of v,
        // MT[c][v] = the product of M_R over the X-block rows R = 4c + b < r
        // selected by v (both in increasing index, as the per-bit loops multiply)
        __shared__ Pauli<1> DT[16][16], MT[16][16];
        __shared__ int pv[64];
        const int nc = (n + 3) >> 2, rc = (r + 3) >> 2;
        for (int e = threadIdx.x; e < 16 * 16; e += blockDim.x) {
            const int c = e >> 4, v = e & 15;
            Pauli<1> a, b;
            pauli_id<1>(a);
            pauli_id<1>(b);
            for (int bb = 0; bb < 4; bb++) {
                const int h = 4 * c + bb;
                if (!((v >> bb) & 1)) continue;
                if (h < n) {
                    Pauli<1> dh;
                    dh.x[0] = __ldg(&d.dx[h]);
                    dh.z[0] = __ldg(&d.dz[h]);
                    dh.e = (int)__ldg(&d.de[h]);
                    pauli_mul<1>(a, dh);
                }
                if (h < r) {
                    Pauli<1> m;
                    m.x[0] = __ldg(&d.mx[h]);
                    m.z[0] = __ldg(&d.mz[h]);
                    m.e = 0;
                    pauli_mul<1>(b, m);
                }
            }
            DT[c][v] = a;
            MT[c][v] = b;
        }
        for (int R = threadIdx.x; R < 64; R += blockDim.x) pv[R] = R < r ? (__ldg(&d.piv[R]) & 63) : 0;
        __syncthreads();
        // four elements of the thread's grid-stride sequence per round, their
        // loads in flight together (the sums keep the sequence's order)
        const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
        for (unsigned long long j0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j0 < k;
             j0 += 4 * stride) {
            uint64_t sv[4];
            double2 av[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const unsigned long long j = j0 + u * stride;
                sv[u] = j < k ? d.sig[buf][j] : 0ull;
                av[u] = j < k ? d.amp[buf][j] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (j0 + u * stride >= k) break;
                const uint64_t s = sv[u];
                if ((s & zm[0]) != ze[0]) continue;
                Pauli<1> q;
                pauli_id<1>(q);
                for (int c = 0; c < nc; c++) pauli_mul<1>(q, DT[c][(s >> (4 * c)) & 15]);
                const uint64_t wv = y[0] ^ q.x[0];
                Pauli<1> p;
                pauli_id<1>(p);
                for (int c = 0; c < rc; c++) {
                    int v = 0;
                    for (int bb = 0; bb < 4; bb++) {
                        const int R = 4 * c + bb;
                        if (R < r) v |= (int)((wv >> pv[R]) & 1) << bb;
                    }
                    pauli_mul<1>(p, MT[c][v]);
                }
                if (p.x[0] != wv) continue;
                const int ip = (q.e + __popcll(q.x[0] & q.z[0]) + 2 * __popcll(q.z[0] & wv) + p.e +
                                __popcll(p.x[0] & p.z[0])) & 3;
                const double2 c = ipow_mul(av[u], ip);
                acc[0] += c.x;
                acc[1] += c.y;
            }
        }
    } else {
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
    }
    block_sum<2>(acc, sh);
    if (threadIdx.x == 0) {
        d.red[2 * blockIdx.x] = acc[0];
        d.red[2 * blockIdx.x + 1] = acc[1];
    }
    if (last_block(d.done)) reduce_partials(d, 1, sh);
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
    // W >= 8: the map's low-rank form, then whichever of the low-rank and the
    // dense kernel the rank selects (the other returns at once)
    if (d.W >= 8) {
        const int nt = (d.n + 31) & ~31;
        if (d.W == 16) k_affine_lowrank<16><<<1, nt, 0, s>>>(d);
        else k_affine_lowrank<8><<<1, nt, 0, s>>>(d);
        if (d.W == 16) k_affine_lr<16><<<d.nblk, kThreads, 0, s>>>(d, buf);
        else k_affine_lr<8><<<d.nblk, kThreads, 0, s>>>(d, buf);
    }
    if (d.W == 16) {
        k_affine_cols<16><<<d.nblk, kThreads, 0, s>>>(d, buf);
        return;
    }
    const size_t sm = sf_affine_smem_bytes(d.n, d.W);
    SF_DISPATCH(d.W, {
        // once per kernel, thread-safe (handles may be driven from several host threads)
        static const bool attr = cudaFuncSetAttribute(k_affine<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      200 * 1024) == cudaSuccess;
        (void)attr;
        k_affine<WW><<<d.nblk, kThreads, sm, s>>>(d, buf);
    });
}

void sf_launch_branch(const SfDev& d, uint32_t kind, uint32_t q0, uint32_t q1, double theta, int in_buf,
                      int out_buf, cudaStream_t s) {
    const SfTerms tm = diag_terms_host(kind, theta);
    if (d.W == 16) k_branch_plan<16><<<1, kPlanThreads, 0, s>>>(d, kind, q0, q1, tm);
    if (d.W == 8) k_branch_plan<8><<<1, kPlanThreads, 0, s>>>(d, kind, q0, q1, tm);
    SF_DISPATCH(d.W, k_branch<WW><<<d.nblk, kThreads, 0, s>>>(d, kind, q0, q1, tm, in_buf, out_buf));
}

void sf_launch_insert(const SfDev& d, int in_buf, int out_buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_insert<WW><<<d.nblk, kThreads, 0, s>>>(d, in_buf, out_buf));
}

void sf_launch_branch_merge(const SfDev& d, uint32_t kind, uint32_t q0, uint32_t q1, double theta, double eps,
                            int in_buf, int out_buf, cudaStream_t s) {
    const SfTerms tm = diag_terms_host(kind, theta);
    if (d.W == 16) k_branch_plan<16><<<1, kPlanThreads, 0, s>>>(d, kind, q0, q1, tm);
    if (d.W == 8) k_branch_plan<8><<<1, kPlanThreads, 0, s>>>(d, kind, q0, q1, tm);
    SF_DISPATCH(d.W, k_branch_merge<WW><<<d.nblk, kThreads, 0, s>>>(d, kind, q0, q1, tm, eps * eps, in_buf, out_buf));
}

// the cofactor of a frame whose layout the grid program left known (n <= 63;
// the host has checked that no kernel moved the elements since)
void sf_launch_cof_pos(const SfDev& d, int in_buf, int out_buf, bool prob, cudaStream_t s) {
    k_cof_pos<<<d.nblk, kThreads, 0, s>>>(d, 1e-24, in_buf, out_buf, prob ? 1 : 0);
}

void sf_launch_cof_merge(const SfDev& d, int in_buf, int out_buf, cudaStream_t s) {
    // W >= 8: the closed form when U ^ I and V have low rank, else the per-bit
    // walk (each variant returns at once when the other one applies)
    if (d.W >= 8) {
        const int nt = (d.n + 31) & ~31;
        if (d.W == 16) {
            k_cof_lowrank<16><<<1, nt, 0, s>>>(d);
            k_cof_merge<16, true><<<d.nblk, kThreads, 0, s>>>(d, 1e-24, in_buf, out_buf);
        } else {
            k_cof_lowrank<8><<<1, nt, 0, s>>>(d);
            k_cof_merge<8, true><<<d.nblk, kThreads, 0, s>>>(d, 1e-24, in_buf, out_buf);
        }
    }
    SF_DISPATCH(d.W, k_cof_merge<WW, false><<<d.nblk, kThreads, 0, s>>>(d, 1e-24, in_buf, out_buf));
}

void sf_launch_build_index(const SfDev& d, int buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_build_index<WW><<<d.nblk, kThreads, 0, s>>>(d, buf));
}

void sf_launch_compact(const SfDev& d, double eps, int out_buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_compact<WW><<<d.nblk, kThreads, 0, s>>>(d, out_buf, eps * eps));
}

void sf_launch_cond(const SfDev& d, int buf, int kind, int c1, int c2, int t, double alpha, cudaStream_t s) {
    const double2 ea = kind == 1 ? make_double2(std::cos(alpha), std::sin(alpha)) : make_double2(1.0, 0.0);
    SF_DISPATCH(d.W, k_cond<WW><<<d.nblk, kThreads, 0, s>>>(d, buf, kind, c1, c2, t, ea));
}

void sf_launch_filter(const SfDev& d, int x, int in_buf, int out_buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_filter<WW><<<d.nblk, kThreads, 0, s>>>(d, x, in_buf, out_buf));
}

void sf_launch_prob(const SfDev& d, int buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_prob<WW><<<d.nblk, kThreads, 0, s>>>(d, buf));
}


void sf_launch_amplitude(const SfDev& d, int buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_amplitude<WW><<<d.nblk, kThreads, 0, s>>>(d, buf));
}

void sf_launch_export(const SfDev& d, int buf, int stage_buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_export<WW><<<d.nblk, kThreads, 0, s>>>(d, buf, stage_buf));
}
