// sf_tableau.cu -- single-CTA kernels that work on the shared tableau:
//   * k_clifford:      ROTATE(F, U) on M and D for a batch of Clifford gates
//                      (Table 2 conjugation, Invariant 1 repair by a row
//                      reduction that only works on dirty columns, global-phase
//                      update by the five-step rule of Sec. III once per gate),
//                      emitting the composed affine map sigma' = A sigma ^ t that
//                      k_affine applies to every phase vector.
//   * k_measure_prep:  deterministic/random test of a qubit and, if random, the
//                      COFACTOR update of M (Sec. III, measurement of Sec. II-B
//                      forced to both outcomes) with the tables that map old
//                      frame elements to their two cofactor children.
//   * k_amp_prep, k_reset.
// One thread owns one tableau row (blockDim = NT >= n).  The tableau lives in
// shared memory when it fits, else in a global workspace of the same layout.
#include "sf_device.cuh"

namespace {

constexpr int kMaxWarps = 32;
constexpr int kLeadSlots = 64;  // open-addressing table of lead columns in one repair step
constexpr int kLeadMax = 32;    // distinct leads counted by ballots; more: one full occupancy pass
constexpr int kDirtyMax = 32;   // changed columns listed for a repair; more: every row is examined
constexpr int kRunMax = 512;    // monomial gates held back before a repair is forced

template <int W>
struct Ws {
    uint64_t *mx, *mz, *dx, *dz, *A, *d0x, *d0z;  // word-major [W][NT]
    uint32_t *de, *d0e, *t0, *t1;                // [NT]
    int32_t* piv;                                // [NT]
};

template <int W>
__device__ Ws<W> carve(uint64_t* base, int NT) {
    Ws<W> T;
    size_t o = 0, s = (size_t)W * NT;
    T.mx = base + o; o += s;
    T.mz = base + o; o += s;
    T.dx = base + o; o += s;
    T.dz = base + o; o += s;
    T.A = base + o; o += s;
    T.d0x = base + o; o += s;
    T.d0z = base + o; o += s;
    uint32_t* u = reinterpret_cast<uint32_t*>(base + o);
    T.de = u; u += NT;
    T.d0e = u; u += NT;
    T.t0 = u; u += NT;
    T.t1 = u; u += NT;
    T.piv = reinterpret_cast<int32_t*>(u);
    return T;
}

template <int W>
struct Scratch {
    int wmin[2][kMaxWarps];
    uint64_t y[W], y2[W], words[5][W];
    uint64_t occ1[2 * W], occ2[2 * W];  // columns holding >= 1 / >= 2 ones (x words, then z words)
    uint64_t wx[kMaxWarps][W], wz[kMaxWarps][W];  // per-warp word totals of a product
    uint64_t px[W], pz[W], qx[W], qz[W], wv[W];  // product results, amplitude point
    int pe, qe, ired[kMaxWarps];
    int iv[8];
    double dv[8];
    // repair bookkeeping
    uint64_t pol[2 * W];    // columns not known to hold a single 1 (see cta_rref)
    uint64_t dmask[2 * W];  // columns changed by the gates since the last repair
    int dl[kDirtyMax], ndl;  // the same columns as a list (ndl > kDirtyMax: not listed)
    int lkey[kLeadSlots], lcnt[kLeadSlots], llist[kLeadMax], nlead;
    int wmin2[kMaxWarps];
    uint64_t prow[3 * W];  // the elimination pivot's x, z and A words
    int nlp;               // its next 1 after the eliminated column
};

template <int W>
__device__ __forceinline__ void load_m(const Ws<W>& T, int NT, int h, Pauli<W>& p) {
#pragma unroll
    for (int w = 0; w < W; w++) { p.x[w] = T.mx[w * NT + h]; p.z[w] = T.mz[w * NT + h]; }
    p.e = 0;
}
template <int W>
__device__ __forceinline__ void load_d(const Ws<W>& T, int NT, int h, Pauli<W>& p) {
#pragma unroll
    for (int w = 0; w < W; w++) { p.x[w] = T.dx[w * NT + h]; p.z[w] = T.dz[w * NT + h]; }
    p.e = (int)T.de[h];
}
template <int W>
__device__ __forceinline__ void store_d(const Ws<W>& T, int NT, int h, const Pauli<W>& p) {
#pragma unroll
    for (int w = 0; w < W; w++) { T.dx[w * NT + h] = p.x[w]; T.dz[w * NT + h] = p.z[w]; }
    T.de[h] = (uint32_t)p.e;
}

__device__ __forceinline__ uint64_t warp_xor64(uint64_t v) {
    const unsigned lo = __reduce_xor_sync(SF_FULL, (unsigned)v);
    const unsigned hi = __reduce_xor_sync(SF_FULL, (unsigned)(v >> 32));
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

// Ordered product, in row order, of the rows h with sel (Pauli i^{E_h} P(X_h,
// Z_h) from word-major planes; E null: phase 0) -- word by word, with no
// per-thread Pauli in registers.  The product P_1 ... P_m is
//   i^e P(X, Z),  X = xor x_i,  Z = xor z_i,
//   e = sum_i (e_i + |x_i & z_i|) + 2 sum_{i<j} |z_i & x_j| - |X & Z|  (mod 4)
// (Table 1 applied factor by factor).  Only the parity of the cross term
// matters, so it splits into an in-warp part (a shuffle scan of z along the
// lanes) and a cross-warp part: for warp v, the z total of the earlier warps
// against the xor of x over warp v.  Warps without a selected row skip the
// scan; one warp combines the per-warp totals.  Words are fetched four at a
// time so that their loads are in flight together.  Results in ox / oz / *oe
// (shared), visible to every thread on return.
template <int W>
__device__ void cta_rows_product(const uint64_t* X, const uint64_t* Z, const uint32_t* E, int NT, bool sel,
                                 Scratch<W>& S, uint64_t* ox, uint64_t* oz, int* oe) {
    const int h = threadIdx.x, lane = h & 31, wid = h >> 5, nw = blockDim.x >> 5;
    constexpr int CH = W < 4 ? W : 4;
    int tot = 0;
    if (__any_sync(SF_FULL, sel)) {
        int acc = (sel && E) ? (int)E[h] : 0;
        int par = 0;
#pragma unroll 1
        for (int b = 0; b < W; b += CH) {
            uint64_t xs[CH], zs[CH];
#pragma unroll
            for (int k = 0; k < CH; k++) {
                xs[k] = sel ? X[(b + k) * NT + h] : 0ull;
                zs[k] = sel ? Z[(b + k) * NT + h] : 0ull;
            }
#pragma unroll
            for (int k = 0; k < CH; k++) {
                const uint64_t x = xs[k], z = zs[k];
                acc += __popcll(x & z);
                uint64_t inc = z;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint64_t t = __shfl_up_sync(SF_FULL, inc, off);
                    if (lane >= off) inc ^= t;
                }
                par ^= __popcll((inc ^ z) & x) & 1;
                const uint64_t xt = warp_xor64(x);
                if (lane == 31) S.wz[wid][b + k] = inc;
                if (lane == 0) S.wx[wid][b + k] = xt;
            }
        }
        tot = __reduce_add_sync(SF_FULL, (acc + 2 * par) & 3);
    } else {
        for (int w = lane; w < W; w += 32) {
            S.wz[wid][w] = 0ull;
            S.wx[wid][w] = 0ull;
        }
    }
    if (lane == 0) S.ired[wid] = tot;
    __syncthreads();
    if (wid == 0) {  // lane w combines word w over the warps, in row order
        uint64_t zp = 0, xa = 0;
        int e = 0;
        if (lane < W) {
            for (int v = 0; v < nw; v++) {
                const uint64_t xv = S.wx[v][lane];
                e += 2 * __popcll(zp & xv);
                zp ^= S.wz[v][lane];
                xa ^= xv;
            }
            ox[lane] = xa;
            oz[lane] = zp;
            e -= __popcll(xa & zp);
        }
        if (lane < nw) e += S.ired[lane];
        e = __reduce_add_sync(SF_FULL, e);
        if (lane == 0) *oe = e & 3;
    }
    __syncthreads();
}

// OR a per-thread bit (thread h -> bit h) into words[W] (must be zeroed).
template <int W>
__device__ void cta_bits(bool b, uint64_t* words) {
    const int h = threadIdx.x;
    unsigned bal = __ballot_sync(SF_FULL, b);
    if ((h & 31) == 0 && bal) {
        atomicOr(reinterpret_cast<unsigned long long*>(&words[h >> 6]),
                 (unsigned long long)bal << (h & 32));
    }
}

// <y| D^tau phi_0(M)> * 2^{r/2} as an i-power (0..3), or -1 when it is zero.
// tau: per-row bits (nullptr = all zero).  y: W words in shared memory.
// With Q = prod_{tau_h} D_h = i^{q} P(qx, qz): D^tau phi_0 = Q phi_0, whose
// amplitude at y is the phi_0 amplitude at w = y ^ qx times i^{q + |qx qz| +
// 2 |qz w|}; phi_0 has support on the row span of the X block, and at w it is
// i^{|px pz|} 2^{-r/2} for the product P of the X-block rows picked by the
// pivot bits of w (zero unless px = w).  Stabilizer rows commute with each
// other, and so do destabilizer rows, so neither product depends on the order
// of the rows: the rows need not be sorted by pivot.
template <int W>
__device__ int cta_amp_phi(const Ws<W>& T, int n, int NT, int r, const uint32_t* tau, const uint64_t* y,
                           Scratch<W>& S) {
    const int h = threadIdx.x;
    if (tau) {
        cta_rows_product<W>(T.dx, T.dz, T.de, NT, h < n && tau[h], S, S.qx, S.qz, &S.qe);
    } else {  // Q = I
        if (h < W) S.qx[h] = S.qz[h] = 0ull;
        if (h == 0) S.qe = 0;
    }
    if (h < W) S.wv[h] = y[h] ^ S.qx[h];  // w
    __syncthreads();
    const uint64_t* wv = S.wv;
    bool sel = false;
    if (h < n) {  // X-block rows, wherever they sit (their products do not depend on the order)
        const int pv = T.piv[h];
        sel = pv < n && ((wv[pv >> 6] >> (pv & 63)) & 1);
    }
    cta_rows_product<W>(T.mx, T.mz, nullptr, NT, sel, S, S.px, S.pz, &S.pe);
    bool ok = true;
    int tot = S.qe + S.pe;
#pragma unroll 1
    for (int w = 0; w < W; w++) {
        ok &= (S.px[w] == wv[w]);
        tot += __popcll(S.qx[w] & S.qz[w]) + 2 * __popcll(S.qz[w] & wv[w]) + __popcll(S.px[w] & S.pz[w]);
    }
    __syncthreads();  // the scratch words are reused by the next call
    if (!ok) return -1;
    return tot & 3;
}

// Conjugate one row (x, z planes, word-major) by a Clifford gate; returns the
// sign flip.  Per qubit: H swaps x,z (flip on Y); S: z ^= x (flip on Y);
// S^dagger: z ^= x (flip on X); Paulis flip on anticommutation; CNOT(c,t):
// x_t ^= x_c, z_c ^= z_t, flip = x_c z_t (x_t ^ z_c ^ 1); CZ(a,b): z_b ^= x_a,
// z_a ^= x_b, flip = x_a x_b (z_a ^ z_b); SWAP exchanges the columns.
__device__ __forceinline__ int conj_row(int kind, int q0, int q1, uint64_t* X, uint64_t* Z, int NT, int h) {
    uint64_t* x0 = &X[(q0 >> 6) * NT + h];
    uint64_t* z0 = &Z[(q0 >> 6) * NT + h];
    const int b0 = q0 & 63;
    const uint64_t m0 = 1ull << b0;
    const int xa = (int)((*x0 >> b0) & 1), za = (int)((*z0 >> b0) & 1);
    int f = 0;
    switch (kind) {
        case 0: f = xa & za; if (xa != za) { *x0 ^= m0; *z0 ^= m0; } break;
        case 1: f = xa & za; if (xa) *z0 ^= m0; break;
        case 2: f = xa & (za ^ 1); if (xa) *z0 ^= m0; break;
        case 3: f = za; break;
        case 4: f = xa ^ za; break;
        case 5: f = xa; break;
        default: {
            uint64_t* x1 = &X[(q1 >> 6) * NT + h];
            uint64_t* z1 = &Z[(q1 >> 6) * NT + h];
            const int b1 = q1 & 63;
            const uint64_t m1 = 1ull << b1;
            const int xb = (int)((*x1 >> b1) & 1), zb = (int)((*z1 >> b1) & 1);
            if (kind == 6) {
                f = xa & zb & (xb ^ za ^ 1);
                if (xa) *x1 ^= m1;
                if (zb) *z0 ^= m0;
            } else if (kind == 7) {
                f = xa & xb & (za ^ zb);
                if (xa) *z1 ^= m1;
                if (xb) *z0 ^= m0;
            } else {
                if (xa != xb) { *x0 ^= m0; *x1 ^= m1; }
                if (za != zb) { *z0 ^= m0; *z1 ^= m1; }
            }
        }
    }
    return f;
}

// ---- Invariant 1 repair without row movement (CTA version) -----------------
// First set bit of plane P (row h) at or after word w0, word w0 masked by m0;
// -1 if none.  Words are fetched eight at a time so that their loads are in
// flight together.
template <int W>
__device__ __forceinline__ int plane_first(const uint64_t* P, int NT, int h, int w0, uint64_t m0) {
    constexpr int CH = W < 8 ? W : 8;
#pragma unroll 1
    for (int b = w0; b < W; b += CH) {
        uint64_t v[CH];
#pragma unroll
        for (int k = 0; k < CH; k++) v[k] = (b + k < W) ? P[(b + k) * NT + h] : 0ull;
        if (b == w0) v[0] &= m0;
#pragma unroll
        for (int k = 0; k < CH; k++)
            if (v[k]) return 64 * (b + k) + __ffsll((long long)v[k]) - 1;
    }
    return -1;
}

// leading column of row h (columns x_0..x_{n-1}, z_0..z_{n-1})
template <int W>
__device__ __forceinline__ int row_lead(const Ws<W>& T, int NT, int h, int n) {
    int b = plane_first<W>(T.mx, NT, h, 0, ~0ull);
    if (b >= 0) return b;
    b = plane_first<W>(T.mz, NT, h, 0, ~0ull);
    return b >= 0 ? n + b : 0x7fffffff;
}

// first 1 of row h after column c, for a row that leads at c
template <int W>
__device__ __forceinline__ int row_next_lead(const Ws<W>& T, int NT, int h, int n, int c) {
    if (c < n) {
        int b = plane_first<W>(T.mx, NT, h, c >> 6, ~((2ull << (c & 63)) - 1ull));
        if (b >= 0) return b;
        b = plane_first<W>(T.mz, NT, h, 0, ~0ull);
        return b >= 0 ? n + b : 0x7fffffff;
    }
    const int cz = c - n;
    const int b = plane_first<W>(T.mz, NT, h, cz >> 6, ~((2ull << (cz & 63)) - 1ull));
    return b >= 0 ? n + b : 0x7fffffff;
}

// bit of row h in column c
template <int W>
__device__ __forceinline__ bool row_bit(const Ws<W>& T, int NT, int h, int n, int c) {
    return c < n ? ((T.mx[(c >> 6) * NT + h] >> (c & 63)) & 1) : ((T.mz[((c - n) >> 6) * NT + h] >> ((c - n) & 63)) & 1);
}

__device__ __forceinline__ bool col_set(const uint64_t* occ, int W, int c, int n) {
    const int wi = c < n ? (c >> 6) : W + ((c - n) >> 6);
    const int b = c < n ? (c & 63) : ((c - n) & 63);
    return (occ[wi] >> b) & 1;
}

// S.occ1 / S.occ2: columns with at least one / at least two ones over all rows
template <int W>
__device__ void cta_occupancy(const Ws<W>& T, int NT, Scratch<W>& S) {
    const int h = threadIdx.x, lane = h & 31;
    constexpr int CH = W < 4 ? 2 * W : 4;  // words fetched together
    if (h < 2 * W) { S.occ1[h] = 0; S.occ2[h] = 0; }
    __syncthreads();
#pragma unroll 1
    for (int b = 0; b < 2 * W; b += CH) {
        uint64_t ov[CH];
#pragma unroll
        for (int k = 0; k < CH; k++) {
            const int w = b + k;
            ov[k] = w < W ? T.mx[w * NT + h] : T.mz[(w - W) * NT + h];
        }
#pragma unroll
        for (int k = 0; k < CH; k++) {
            uint64_t o = ov[k];
            if (!__any_sync(SF_FULL, o != 0)) continue;
            uint64_t m = 0;
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                const uint64_t oo = __shfl_xor_sync(SF_FULL, o, off);
                const uint64_t om = __shfl_xor_sync(SF_FULL, m, off);
                m |= om | (o & oo);
                o |= oo;
            }
            if (lane == 0 && o) {
                const unsigned long long prev = atomicOr(reinterpret_cast<unsigned long long*>(&S.occ1[b + k]), o);
                if (m | (prev & o)) atomicOr(reinterpret_cast<unsigned long long*>(&S.occ2[b + k]), m | (prev & o));
            }
        }
    }
    __syncthreads();
}

// move row fields so that row h goes to position dst (a permutation)
template <int W>
__device__ void cta_permute64(uint64_t* F, uint64_t* tmp, int NT, int h, int n, int dst) {
    if (h < n) {
#pragma unroll 1
        for (int w = 0; w < W; w++) tmp[w * NT + dst] = F[w * NT + h];
    }
    __syncthreads();
    if (h < n) {
#pragma unroll 1
        for (int w = 0; w < W; w++) F[w * NT + h] = tmp[w * NT + h];
    }
    __syncthreads();
}

__device__ void cta_permute32(uint32_t* F, uint32_t* tmp, int h, int n, int dst) {
    if (h < n) tmp[dst] = F[h];
    __syncthreads();
    if (h < n) F[h] = tmp[h];
    __syncthreads();
}

// where the sort records its permutation (W >= 8): the pivots before the
// kernel ran, the move list and rho in the plan (null: not recorded)
struct SortRec {
    const int32_t* old_piv;
    uint64_t* mv;
    uint32_t* rho;
};

template <int W, bool TRACK_A>
__device__ int cta_sort_rows(const Ws<W>& T, int n, int NT, Scratch<W>& S, SortRec rec = {nullptr, nullptr, nullptr});

// Record the lead column l of the calling lane in the lead table (lanes with
// l < 0 take no part); equal leads in a warp are inserted once.  Returns the
// slot, or -1 when the table is full (S.nlead is then pushed past kLeadMax).
template <int W>
__device__ __forceinline__ int lead_insert(Scratch<W>& S, int l) {
    const int lane = threadIdx.x & 31;
    const unsigned grp = __match_any_sync(SF_FULL, l);
    const int leader = __ffs(grp) - 1;
    int slot = -1;
    if (l >= 0 && lane == leader && *reinterpret_cast<volatile int*>(&S.nlead) <= kLeadMax) {
        int s = (int)(((unsigned)l * 0x9E3779B1u) >> 26);  // 64 slots
        for (int i = 0; i < 16; i++) {  // at most 16 probes (load factor <= 1/2)
            const int k = atomicCAS(&S.lkey[s], -1, l);
            if (k == -1) {
                const int idx = atomicAdd(&S.nlead, 1);
                if (idx < kLeadMax) S.llist[idx] = s;
                slot = s;
                break;
            }
            if (k == l) {
                slot = s;
                break;
            }
            s = (s + 1) & (kLeadSlots - 1);
        }
        if (slot < 0) atomicAdd(&S.nlead, kLeadMax + 1);
    }
    return __shfl_sync(SF_FULL, slot, leader);
}

// The repair.  Rows stay in place while pivots are chosen: every unassigned
// row whose leading column holds no other 1 in the tableau takes it as pivot
// at once (Gauss-Jordan would reach it with nothing to eliminate, in any
// order); otherwise the smallest leading column c among unassigned rows takes
// one elimination step, its pivot p being the unassigned row leading at c
// whose next 1 lies furthest right: every other row with bit c gets
// M_h <- M_h M_p, mirrored as D_p <- D_p D_h, A_h ^= A_p and t_h ^= t_p ^ c.
// The leading columns of unassigned rows are counted over all rows by
// ballots (one full occupancy pass only when more than kLeadMax distinct
// leads are open).  dirty: the tableau was in RREF with pivots T.piv before
// gates that changed only the columns S.dl / S.dmask.  Then a row is settled
// without a count while its lead is its old pivot column and that column is
// not "polluted" (S.pol: the changed columns and the old pivots of the rows
// used as elimination pivots), because such a column still holds its one 1:
// the gates did not touch it, and every elimination pivot other than its
// owner has a 0 there.  The decisions are those of the plain algorithm.
// Returns r (SORT: after sorting the rows by pivot), or -1 if a row has no
// bits (dependent rows).
template <int W, bool TRACK_A, bool SORT = true>
__device__ int cta_rref(const Ws<W>& T, int n, int NT, Scratch<W>& S, SortRec rec = {nullptr, nullptr, nullptr},
                        bool dirty = false) {
    const int h = threadIdx.x, lane = h & 31, wid = h >> 5, nw = NT >> 5;
    constexpr int INF = 0x7fffffff;
    const int pv0 = h < n ? T.piv[h] : INF;
    bool asg = false;
    if (h < 2 * W) S.pol[h] = dirty ? S.dmask[h] : ~0ull;
    if (h < kLeadSlots) {
        S.lkey[h] = -1;
        S.lcnt[h] = 0;
    }
    if (h == 0) S.nlead = 0;
    // l: the lead of an unassigned row, kept up to date across the steps (an
    // elimination changes only the rows that lead at its column)
    int l = INF;
    if (h < n) {
        if (dirty && pv0 < 2 * n) {
            // the row led at pv0 before the gates, which changed only the listed columns
            int dmin = INF;
            const int nd = S.ndl;
#pragma unroll 4
            for (int i = 0; i < nd; i++) {
                const int c = S.dl[i];
                if (c < pv0 && row_bit<W>(T, NT, h, n, c)) dmin = min(dmin, c);
            }
            if (dmin != INF)
                l = dmin;
            else if (!col_set(S.dmask, W, pv0, n))
                asg = true;  // settled: its lead and pivot column are untouched
            else
                l = row_bit<W>(T, NT, h, n, pv0) ? pv0 : row_next_lead<W>(T, NT, h, n, pv0);
        } else {
            l = row_lead<W>(T, NT, h, n);
        }
    }
    __syncthreads();
    for (int it = 0; it <= n; it++) {
        if (!asg && l != INF && l == pv0 && !col_set(S.pol, W, l, n)) asg = true;  // T.piv[h] == l already
        const bool need = h < n && !asg && l != INF;
        const int slot = lead_insert<W>(S, need ? l : -1);
        __syncthreads();
        bool uniq = false;
        if (S.nlead > kLeadMax) {  // many open leads: count every column once
            cta_occupancy<W>(T, NT, S);
            uniq = need && !col_set(S.occ2, W, l, n);
        } else if (S.nlead > 0) {
            const int K = S.nlead;
#pragma unroll 4
            for (int k = 0; k < K; k++) {
                const int sl = S.llist[k];
                const bool b = h < n && row_bit<W>(T, NT, h, n, S.lkey[sl]);
                const unsigned bal = __ballot_sync(SF_FULL, b);
                if (lane == 0 && bal) atomicAdd(&S.lcnt[sl], __popc(bal));
            }
            __syncthreads();
            uniq = need && S.lcnt[slot] < 2;
        }
        if (uniq) {
            asg = true;
            T.piv[h] = l;
        }
        // smallest leading column c of the unassigned rows, then the pivot among
        // the rows leading at c: the one whose next 1 lies furthest right (no
        // further 1: best), lowest row index on ties -- the other candidates then
        // keep their own next 1 as lead and no chain of steps follows
        const int lk = (h < n && !asg && l != INF) ? l : INF;
        const int wl = __reduce_min_sync(SF_FULL, lk);
        const bool wdone = __all_sync(SF_FULL, asg || h >= n);
        if (lane == 0) {
            S.wmin[0][wid] = wl;
            S.wmin2[wid] = wdone ? 1 : 0;
        }
        __syncthreads();
        int c = INF;
        bool none_left = true;
        for (int i = 0; i < nw; i++) {
            c = min(c, S.wmin[0][i]);
            none_left = none_left && S.wmin2[i];
        }
        if (h < kLeadSlots) {  // the table is read again only after the next barriers
            S.lkey[h] = -1;
            S.lcnt[h] = 0;
        }
        if (h == 0) S.nlead = 0;
        if (c == INF) {
            if (!none_left) return -1;  // an unassigned row without bits
            break;
        }
        unsigned pk = 0xffffffffu;
        int nl = INF;
        if (lk == c) {
            nl = row_next_lead<W>(T, NT, h, n, c);  // nl <= 2n - 1 <= 2047
            pk = ((nl == INF ? 0u : (unsigned)(2048 - nl)) << 10) | (unsigned)h;
        }
        const unsigned wp = __reduce_min_sync(SF_FULL, pk);
        if (lane == 0) S.wmin[1][wid] = (int)wp;
        __syncthreads();
        unsigned pmin = 0xffffffffu;
        for (int i = 0; i < nw; i++) pmin = min(pmin, (unsigned)S.wmin[1][i]);
        const int p = (int)(pmin & 1023u);
        // the pivot row (and its A row) in shared memory, with its next 1
        for (int e = h; e < (TRACK_A ? 3 : 2) * W; e += NT) {
            const int w = e % W, pl = e / W;
            S.prow[e] = (pl == 0 ? T.mx : pl == 1 ? T.mz : T.A)[w * NT + p];
        }
        if (h == p) S.nlp = nl;
        // elimination step at column c with pivot row p
        const uint64_t* plane = c < n ? T.mx : T.mz;
        const int cc = c < n ? c : c - n;
        const bool el = (h < n) && (h != p) && ((plane[(cc >> 6) * NT + h] >> (cc & 63)) & 1);
        __syncthreads();
        if (el) {
            // sign bit of the row product and the row update, four words at a time
            constexpr int CH = W < 4 ? W : 4;
            int lam = 0;
#pragma unroll 1
            for (int b = 0; b < W; b += CH) {
                uint64_t xh[CH], zh[CH];
#pragma unroll
                for (int k = 0; k < CH; k++) {
                    xh[k] = T.mx[(b + k) * NT + h];
                    zh[k] = T.mz[(b + k) * NT + h];
                }
#pragma unroll
                for (int k = 0; k < CH; k++) {
                    const int o = (b + k) * NT;
                    const uint64_t xi = S.prow[b + k], zi = S.prow[W + b + k];
                    lam += __popcll(xh[k] & zh[k]) + __popcll(xi & zi) + 2 * __popcll(zh[k] & xi) -
                           __popcll((xh[k] ^ xi) & (zh[k] ^ zi));
                    T.mx[o + h] = xh[k] ^ xi;
                    T.mz[o + h] = zh[k] ^ zi;
                }
            }
            if (TRACK_A) {
#pragma unroll 1
                for (int b = 0; b < W; b += CH) {
                    uint64_t ah[CH];
#pragma unroll
                    for (int k = 0; k < CH; k++) ah[k] = T.A[(b + k) * NT + h];
#pragma unroll
                    for (int k = 0; k < CH; k++) T.A[(b + k) * NT + h] = ah[k] ^ S.prow[2 * W + b + k];
                }
            }
            const uint32_t cbit = (uint32_t)((lam & 3) >> 1) & 1u;
            T.t0[h] ^= T.t0[p] ^ cbit;
            T.t1[h] ^= T.t1[p] ^ cbit;
        }
        if (__syncthreads_or(el)) {
            // D_p <- D_p * prod_{eliminated h} D_h, one lane of warp 0 per word
            cta_rows_product<W>(T.dx, T.dz, T.de, NT, el, S, S.qx, S.qz, &S.qe);
            if (wid == 0) {
                int lam = 0;
                for (int w = lane; w < W; w += 32) {
                    const uint64_t ax = T.dx[w * NT + p], az = T.dz[w * NT + p];
                    const uint64_t bx = S.qx[w], bz = S.qz[w];
                    lam += __popcll(ax & az) + __popcll(bx & bz) + 2 * __popcll(az & bx) -
                           __popcll((ax ^ bx) & (az ^ bz));
                    T.dx[w * NT + p] = ax ^ bx;
                    T.dz[w * NT + p] = az ^ bz;
                }
                lam = __reduce_add_sync(SF_FULL, lam);
                if (lane == 0) T.de[p] = (T.de[p] + (uint32_t)S.qe + (uint32_t)lam) & 3u;
            }
        }
        if (el && lk == c) {
            // a candidate other than p: its bits up to its own next 1 are p's zeros,
            // so that is its new lead, unless p's next 1 is the same column
            const int nlp = S.nlp;
            l = nl < nlp ? nl : (nl == INF ? INF : row_next_lead<W>(T, NT, h, n, nl));
        }
        if (h == p) {
            asg = true;
            T.piv[p] = c;
            if (pv0 < 2 * n) {  // p's old pivot column now holds p's 1 in the eliminated rows
                const int wi = pv0 < n ? (pv0 >> 6) : W + ((pv0 - n) >> 6);
                const int bb = pv0 < n ? (pv0 & 63) : ((pv0 - n) & 63);
                atomicOr(reinterpret_cast<unsigned long long*>(&S.pol[wi]), 1ull << bb);
            }
        }
        __syncthreads();
    }
    if (!SORT) {  // the caller sorts later (cta_sort_rows); r = rows with an x pivot
        const int xr = __syncthreads_count(h < n && T.piv[h] < n);
        return xr;
    }
    return cta_sort_rows<W, TRACK_A>(T, n, NT, S, rec);
}

// The sort's permutation as bit moves (the plan's move list): rows whose
// pivot differs from old_piv moved; the others keep their relative order, so
// deleting the moved rows' bits and inserting them at their new positions
// maps a phase vector like the sort maps the rows.  Called by every thread
// with its row's pre-sort pivot and new position.
__device__ void cta_record_moves(const SortRec& rec, int n, int h, int pv, int rank) {
    __shared__ int cnt;
    __shared__ int la[SF_MV_MAX], le[SF_MV_MAX];
    if (h == 0) cnt = 0;
    __syncthreads();
    if (h < n) {
        rec.rho[h] = (uint32_t)rank;
        if (pv != rec.old_piv[h]) {
            const int k = atomicAdd(&cnt, 1);
            if (k < SF_MV_MAX) {
                la[k] = h;
                le[k] = rank;
            }
        }
    }
    __syncthreads();
    if (h == 0) {
        const int m = cnt;
        if (m > SF_MV_MAX) {
            rec.mv[0] = SF_LR_NONE;
        } else {
            int a[SF_MV_MAX], e[SF_MV_MAX], ord[SF_MV_MAX];
            for (int k = 0; k < m; k++) { a[k] = la[k]; e[k] = le[k]; }
            for (int k = 1; k < m; k++)  // by old position
                for (int i = k; i > 0 && a[i - 1] > a[i]; i--) {
                    const int ta = a[i]; a[i] = a[i - 1]; a[i - 1] = ta;
                    const int te = e[i]; e[i] = e[i - 1]; e[i - 1] = te;
                }
            for (int k = 0; k < m; k++) ord[k] = k;
            for (int k = 1; k < m; k++)  // insertion order: by new position
                for (int i = k; i > 0 && e[ord[i - 1]] > e[ord[i]]; i--) {
                    const int t = ord[i]; ord[i] = ord[i - 1]; ord[i - 1] = t;
                }
            rec.mv[0] = (uint64_t)m;
            for (int k = 0; k < SF_MV_MAX; k++) {
                const bool in = k < m;
                rec.mv[1 + k] = in ? (uint64_t)a[k] : 0ull;
                rec.mv[1 + SF_MV_MAX + k] = in ? (uint64_t)e[ord[k]] : 0ull;
                rec.mv[1 + 2 * SF_MV_MAX + k] = in ? (uint64_t)ord[k] : 0ull;
                rec.mv[1 + 3 * SF_MV_MAX + (in ? ord[k] : k)] = in ? (uint64_t)k : 0ull;
            }
        }
    }
    __syncthreads();
}

// Rows sorted by pivot (rank = number of pivots in smaller columns), carrying
// every per-row field along; returns r, the X-block size.
template <int W, bool TRACK_A>
__device__ int cta_sort_rows(const Ws<W>& T, int n, int NT, Scratch<W>& S, SortRec rec) {
    const int h = threadIdx.x;
    constexpr int INF = 0x7fffffff;
    if (h < 2 * W) S.occ1[h] = 0;
    __syncthreads();
    const int pv = h < n ? T.piv[h] : INF;
    if (h < n) {
        const int wi = pv < n ? (pv >> 6) : W + ((pv - n) >> 6);
        const int b = pv < n ? (pv & 63) : ((pv - n) & 63);
        atomicOr(reinterpret_cast<unsigned long long*>(&S.occ1[wi]), 1ull << b);
    }
    __syncthreads();
    int rank = h, rx = 0;
#pragma unroll 1
    for (int w = 0; w < W; w++) rx += __popcll(S.occ1[w]);
    if (h < n) {
        const int wi = pv < n ? (pv >> 6) : W + ((pv - n) >> 6);
        const int b = pv < n ? (pv & 63) : ((pv - n) & 63);
        rank = __popcll(S.occ1[wi] & ((1ull << b) - 1));
#pragma unroll 1
        for (int w = 0; w < wi; w++) rank += __popcll(S.occ1[w]);
    }
    if (rec.mv) cta_record_moves(rec, n, h, pv, rank);
    if (__syncthreads_or(rank != h)) {
        // scratch: the Clifford kernel has d0x/d0e free, the measurement kernel
        // (which keeps the old destabilizers there) has A free
        uint64_t* t64 = TRACK_A ? T.d0x : T.A;
        uint32_t* t32 = TRACK_A ? T.d0e : reinterpret_cast<uint32_t*>(T.A);
        cta_permute64<W>(T.mx, t64, NT, h, n, rank);
        cta_permute64<W>(T.mz, t64, NT, h, n, rank);
        cta_permute64<W>(T.dx, t64, NT, h, n, rank);
        cta_permute64<W>(T.dz, t64, NT, h, n, rank);
        if (TRACK_A) cta_permute64<W>(T.A, t64, NT, h, n, rank);
        cta_permute32(T.de, t32, h, n, rank);
        cta_permute32(T.t0, t32, h, n, rank);
        cta_permute32(T.t1, t32, h, n, rank);
        cta_permute32(reinterpret_cast<uint32_t*>(T.piv), t32, h, n, rank);
    }
    return rx;
}

template <int W>
__device__ void load_tableau(const SfDev& d, const Ws<W>& T) {
    const int h = threadIdx.x, n = d.n, NT = d.NT;
#pragma unroll
    for (int w = 0; w < W; w++) {
        T.mx[w * NT + h] = h < n ? d.mx[w * n + h] : 0;
        T.mz[w * NT + h] = h < n ? d.mz[w * n + h] : 0;
        T.dx[w * NT + h] = h < n ? d.dx[w * n + h] : 0;
        T.dz[w * NT + h] = h < n ? d.dz[w * n + h] : 0;
    }
    T.de[h] = h < n ? d.de[h] : 0;
    T.piv[h] = h < n ? d.piv[h] : 0x7fffffff;
    T.t0[h] = 0;
    T.t1[h] = 0;
}

template <int W>
__device__ void store_tableau(const SfDev& d, const Ws<W>& T, int r) {
    const int h = threadIdx.x, n = d.n, NT = d.NT;
    if (h < n) {
#pragma unroll
        for (int w = 0; w < W; w++) {
            d.mx[w * n + h] = T.mx[w * NT + h];
            d.mz[w * n + h] = T.mz[w * NT + h];
            d.dx[w * n + h] = T.dx[w * NT + h];
            d.dz[w * n + h] = T.dz[w * NT + h];
        }
        d.de[h] = T.de[h];
        d.piv[h] = T.piv[h];
    }
    if (h == 0) d.meta[0] = r;
}

// ---------------------------------------------------------------------------
// Basis-point bookkeeping of a run of monomial gates (one thread, bits in
// shared words).
__device__ __forceinline__ int bit_of(const uint64_t* v, int q) { return (int)((v[q >> 6] >> (q & 63)) & 1); }
__device__ __forceinline__ void flip_bit(uint64_t* v, int q) { v[q >> 6] ^= 1ull << (q & 63); }

// U|v> = i^k |v'> for a monomial gate U: moves v to v', returns k
__device__ __forceinline__ int mono_step(int kind, int q0, int q1, uint64_t* v) {
    const int b0 = bit_of(v, q0), b1 = kind >= 6 ? bit_of(v, q1) : 0;
    switch (kind) {
        case 1: return b0;                          // S
        case 2: return 3 * b0;                      // S-dagger
        case 3: flip_bit(v, q0); return 0;          // X
        case 4: flip_bit(v, q0); return 1 + 2 * b0; // Y
        case 5: return 2 * b0;                      // Z
        case 6: if (b0) flip_bit(v, q1); return 0;  // CNOT
        case 7: return 2 * (b0 & b1);               // CZ
        default:                                    // SWAP
            if (b0 != b1) {
                flip_bit(v, q0);
                flip_bit(v, q1);
            }
            return 0;
    }
}

__device__ __forceinline__ uint32_t pack_gate(uint32_t kind, uint32_t q0, uint32_t q1) {
    return kind | (q0 << 4) | (q1 << 18);
}

// record a changed column (thread 0)
template <int W>
__device__ __forceinline__ void mark_col(Scratch<W>& S, int n, int c) {
    const int wi = c < n ? (c >> 6) : W + ((c - n) >> 6);
    const uint64_t m = 1ull << (c < n ? (c & 63) : ((c - n) & 63));
    if (S.dmask[wi] & m) return;
    S.dmask[wi] |= m;
    if (S.ndl < kDirtyMax) S.dl[S.ndl] = c;
    S.ndl++;
}

// the columns a gate changes (x_q: q, z_q: n + q); Paulis change signs only
template <int W>
__device__ __forceinline__ void mark_gate(Scratch<W>& S, int n, int kind, int q0, int q1) {
    switch (kind) {
        case 0: mark_col(S, n, q0); mark_col(S, n, n + q0); break;         // H swaps x_q and z_q
        case 1: case 2: mark_col(S, n, n + q0); break;                     // S: z_q ^= x_q
        case 6: mark_col(S, n, q1); mark_col(S, n, n + q0); break;         // CNOT: x_t ^= x_c, z_c ^= z_t
        case 7: mark_col(S, n, n + q0); mark_col(S, n, n + q1); break;     // CZ
        case 8:                                                            // SWAP
            mark_col(S, n, q0); mark_col(S, n, q1);
            mark_col(S, n, n + q0); mark_col(S, n, n + q1);
            break;
        default: break;
    }
}

// ---------------------------------------------------------------------------
// ROTATE for a batch.  A run of monomial gates (S, S-dagger, X, Y, Z, CNOT,
// CZ, SWAP: each maps a basis state to one basis state times a power of i) is
// held back and applied to the rows together with the H gate that ends it,
// followed by one repair.  Its effect on the global factor comes from basis
// points: the run maps b to pi(b) with U|b> = i^{kappa(b)} |pi(b)>; thread 0
// carries b0 = pi(0) and kappa(0) along (<0|phi_0(M)> = 2^{-r/2}), and for the
// H on q the other point of the pair, pi^{-1}(b0 ^ e_q) = L^{-1} e_q (L the
// run's linear part, walked backwards), whose amplitude on the representation
// before the run gives
//   psi(b0 ^ e_q) / psi(b0) = i^{kappa(v) - kappa(0)} phi_0(v) / phi_0(0).
// The numerator of the phase rule at y = b0 with bit q cleared (or set, when
// the two terms cancel) then follows as for a lone H, and the denominator is
// the new representation's amplitude at y.  A run longer than kRunMax, and
// the run at the end of the batch, are applied and repaired by themselves.
template <int W>
__global__ void __launch_bounds__(1024) k_clifford(SfDev d, const sf_gate_rec* gates, int ng, int buf,
                                                   uint64_t* gws) {
    extern __shared__ uint64_t smem[];
    __shared__ Scratch<W> S;
    __shared__ uint32_t run[kRunMax];
    __shared__ uint32_t gbuf[1024];
    if (*d.status) return;
    const int n = d.n, NT = d.NT, h = threadIdx.x;
    const Ws<W> T = carve<W>(gws ? gws : smem, NT);
    load_tableau<W>(d, T);
#pragma unroll
    for (int w = 0; w < W; w++) T.A[w * NT + h] = (h < n && (h >> 6) == w) ? (1ull << (h & 63)) : 0ull;
    int r = d.meta[0];
    int ga = 0, gb = 0;  // the batch's phase factor omega^ga sqrt(2)^gb
    if (h < W) S.y2[h] = 0;
    if (h < 2 * W) S.dmask[h] = 0;
    if (h == 0) {
        S.iv[0] = 0;
        S.ndl = 0;
    }
    if (h < n) T.t1[h] = 0;
    int nrun = 0;  // monomial gates held back (the same count in every thread)

    // Apply the held-back gates (and the H on hq, if hq >= 0), repair, and
    // update the global factor.  Returns false after setting the status.
    auto flush = [&](int hq) -> bool {
        int na = 0, nb = 0, cq = 0;
        if (hq >= 0) {
            if (h == 0) {
                uint64_t* v = S.y;
                for (int w = 0; w < W; w++) v[w] = 0ull;
                flip_bit(v, hq);
                for (int i = nrun - 1; i >= 0; i--) {  // L^{-1} e_q
                    const uint32_t g = run[i];
                    const int kind = (int)(g & 15u), a = (int)((g >> 4) & 0x3fffu), b = (int)(g >> 18);
                    if (kind == 6) {
                        if (bit_of(v, a)) flip_bit(v, b);
                    } else if (kind == 8 && bit_of(v, a) != bit_of(v, b)) {
                        flip_bit(v, a);
                        flip_bit(v, b);
                    }
                }
                uint64_t* u = S.words[1];
                for (int w = 0; w < W; w++) u[w] = v[w];
                int kv = 0;
                for (int i = 0; i < nrun; i++) {
                    const uint32_t g = run[i];
                    kv += mono_step((int)(g & 15u), (int)((g >> 4) & 0x3fffu), (int)(g >> 18), u);
                }
                S.iv[1] = kv & 3;
                mark_gate(S, n, 0, hq, 0);
            }
            __syncthreads();
            const int cv = cta_amp_phi<W>(T, n, NT, r, nullptr, S.y, S);
            cq = cv < 0 ? -1 : (S.iv[1] - S.iv[0] + cv) & 3;
            cliff_num_exp(0, cq, na, nb);
            if (cq == 2 && bit_of(S.y2, hq)) na += 4;
        } else {
            __syncthreads();
        }
        na += 2 * S.iv[0];
        // conjugate every row by the held-back gates; sign flips of M go to t0
        // (composed over the batch) and t1 (since the last repair)
        if (h < n) {
            uint32_t f = 0;
            int fd = 0;
#pragma unroll 1
            for (int i = 0; i < nrun; i++) {
                const uint32_t g = run[i];
                const int kind = (int)(g & 15u), a = (int)((g >> 4) & 0x3fffu), b = (int)(g >> 18);
                f ^= (uint32_t)conj_row(kind, a, b, T.mx, T.mz, NT, h);
                fd += conj_row(kind, a, b, T.dx, T.dz, NT, h);
            }
            if (hq >= 0) {
                f ^= (uint32_t)conj_row(0, hq, 0, T.mx, T.mz, NT, h);
                fd += conj_row(0, hq, 0, T.dx, T.dz, NT, h);
            }
            T.t0[h] ^= f;
            T.t1[h] ^= f;
            T.de[h] = (T.de[h] + 2u * (uint32_t)fd) & 3u;
        }
        __syncthreads();
        const int r_new = cta_rref<W, true, false>(T, n, NT, S, {nullptr, nullptr, nullptr}, S.ndl <= kDirtyMax);
        if (r_new < 0) {
            if (h == 0) set_status(d.status, SF_ST_INTERNAL, buf, 9u);
            return false;
        }
        // denominator: <y| D'^{t1} phi_0(M')>
        if (h < W) {
            uint64_t v = S.y2[h];
            if (hq >= 0 && (hq >> 6) == h) {
                v &= ~(1ull << (hq & 63));
                if (cq == 2) v |= 1ull << (hq & 63);
            }
            S.y[h] = v;
        }
        __syncthreads();
        const int dq = cta_amp_phi<W>(T, n, NT, r_new, T.t1, S.y, S);
        if (dq < 0) {
            if (h == 0) set_status(d.status, SF_ST_INTERNAL, buf, hq >= 0 ? 1u : 2u);
            return false;
        }
        ga = (ga + na + 2 * ((4 - dq) & 3)) & 7;
        gb += nb + r_new - r;
        r = r_new;
        nrun = 0;
        if (h < n) T.t1[h] = 0;
        if (h < W) S.y2[h] = 0;
        if (h < 2 * W) S.dmask[h] = 0;
        if (h == 0) {
            S.iv[0] = 0;
            S.ndl = 0;
        }
        __syncthreads();
        return true;
    };

    for (int base = 0; base < ng; base += NT) {
        const int cnt = min(NT, ng - base);
        __syncthreads();  // the previous chunk is no longer read
        bool bad = false;
        if (h < cnt) {
            const sf_gate_rec g = gates[base + h];
            const bool two = g.kind >= 6;
            bad = g.kind > 8 || g.q0 >= (uint32_t)n || (two && (g.q1 >= (uint32_t)n || g.q1 == g.q0));
            gbuf[h] = pack_gate(g.kind & 15u, g.q0 & 0x3fffu, two ? (g.q1 & 0x3fffu) : 0u);
        }
        if (__syncthreads_or(bad)) {
            if (h == 0) set_status(d.status, 1u, buf);  // SF_EINVAL: bad gate in a device list
            return;
        }
        for (int k = 0; k < cnt; k++) {
            const uint32_t g = gbuf[k];
            const int kind = (int)(g & 15u), q0 = (int)((g >> 4) & 0x3fffu), q1 = (int)(g >> 18);
            if (kind != 0) {
                if (h == 0) {
                    S.iv[0] = (S.iv[0] + mono_step(kind, q0, q1, S.y2)) & 3;
                    run[nrun] = g;
                    mark_gate(S, n, kind, q0, q1);
                }
                if (++nrun == kRunMax && !flush(-1)) return;
                continue;
            }
            if (!flush(q0)) return;
        }
    }
    if (nrun > 0 && !flush(-1)) return;
    SortRec rec = {nullptr, nullptr, nullptr};
    if constexpr (W >= 8)
        rec = {d.piv, d.plan + plan_mv_aff(n, W), reinterpret_cast<uint32_t*>(d.plan + plan_rho_aff(n, W))};
    const int rs = cta_sort_rows<W, true>(T, n, NT, S, rec);
    store_tableau<W>(d, T, rs);
    if (h == 0) *d.g = cmul(*d.g, cliff_factor(ga, gb));
    // emit the affine map: columns of A (column j = image of e_j) and t as bit words
    uint64_t* AT = T.d0x;  // free in this kernel; W*NT >= n*W words
    for (int e = h; e < n * W; e += NT) AT[e] = 0;
    if (h < W) S.words[0][h] = 0;
    __syncthreads();
    for (int j = 0; j < n; j++) {
        const bool b = (h < n) && ((T.A[(j >> 6) * NT + h] >> (j & 63)) & 1);
        const unsigned bal = __ballot_sync(SF_FULL, b);
        if ((h & 31) == 0 && bal)
            atomicOr(reinterpret_cast<unsigned long long*>(&AT[(size_t)j * W + (h >> 6)]),
                     (unsigned long long)bal << (h & 32));
    }
    __syncthreads();
    uint64_t* pa = d.plan + plan_AT(n, W);
    for (int e = h; e < n * W; e += NT) pa[e] = AT[e];
    cta_bits<W>(h < n && T.t0[h], S.words[0]);
    __syncthreads();
    if (h < W) d.plan[plan_t(n, W) + h] = S.words[0][h];
}

// ---------------------------------------------------------------------------
// COFACTOR(F, q) planning.  If q is random in M (some row has x_q = 1):
//   pick the first such row i; multiply every other anticommuting row by M_i
//   (dual: D_i <- D_i D_h); D_h <- D_h M_i for rows whose destabilizer
//   anticommutes with Z_q; D_i <- M_i, M_i <- Z_q; Gauss-Jordan to RREF.
//   For outcome y, P_y phi_0(M) = kappa_y D'^{tau_y} phi_0(M'); each old
//   destabilizer is D_h = eps_h D'^{u'_h} M'^{v'_h}.  An element sigma then has
//   children P_x D^sigma phi_0 = D^sigma P_{x ^ v.sigma} phi_0, expanded by
//   applying the old D_h of sigma one at a time in the new basis.
template <int W>
__global__ void __launch_bounds__(1024) k_measure_prep(SfDev d, uint32_t q, int buf, uint64_t* gws) {
    extern __shared__ uint64_t smem[];
    __shared__ Scratch<W> S;
    if (*d.status) return;
    const int n = d.n, NT = d.NT, h = threadIdx.x, lane = h & 31, wid = h >> 5, nw = NT >> 5;
    const Ws<W> T = carve<W>(gws ? gws : smem, NT);
    load_tableau<W>(d, T);
    const int r0 = d.meta[0];
    const int qw = q >> 6;
    const uint64_t qm = 1ull << (q & 63);
    __syncthreads();
    const bool uh = (h < n) && (T.mx[qw * NT + h] & qm);
    const unsigned bal = __ballot_sync(SF_FULL, uh);
    if (lane == 0) S.wmin[0][wid] = bal ? (wid * 32 + __ffs(bal) - 1) : 0x7fffffff;
    __syncthreads();
    int i = 0x7fffffff;
    for (int a = 0; a < nw; a++) i = min(i, S.wmin[0][a]);
    if (i == 0x7fffffff) {
        // deterministic: Z_q is a canonical Z-block row
        if (h == 0) d.meta[1] = -1;
        __syncthreads();
        bool isrow = (h < n) && (h >= r0) && (T.piv[h] == n + (int)q);
        if (isrow) {
#pragma unroll
            for (int w = 0; w < W; w++)
                isrow &= (T.mx[w * NT + h] == 0) && (T.mz[w * NT + h] == (w == qw ? qm : 0ull));
            d.meta[1] = isrow ? h : -1;
            if (!isrow) set_status(d.status, SF_ST_INTERNAL, buf, 3u);
        }
        if (h == 0) d.meta[2] = 0;
        return;
    }
    // numerators: <0|phi_0> = 1 and <x_i|phi_0> = i^{popc(x_i & z_i)} (units 2^{-r/2})
    if (h < W) {
        S.y[h] = 0;
        S.y2[h] = T.mx[h * NT + i];
        S.words[0][h] = 0;
        S.words[1][h] = 0;
        S.words[2][h] = 0;
        S.words[4][h] = 0;
    }
    __syncthreads();
    // rows anticommuting with Z_q: elements sigma and sigma ^ uq share their cofactors
    cta_bits<W>(uh, S.words[4]);
    int num1 = 0;
    {
        uint64_t xi[W], zi[W];
#pragma unroll
        for (int w = 0; w < W; w++) { xi[w] = T.mx[w * NT + i]; zi[w] = T.mz[w * NT + i]; }
        num1 = popc_and<W>(xi, zi) & 3;
    }
    // v = destabilizers anticommuting with Z_q (before any change)
    cta_bits<W>((h < n) && (T.dx[qw * NT + h] & qm), S.words[0]);
    // keep a copy of the old destabilizers
#pragma unroll
    for (int w = 0; w < W; w++) { T.d0x[w * NT + h] = T.dx[w * NT + h]; T.d0z[w * NT + h] = T.dz[w * NT + h]; }
    T.d0e[h] = T.de[h];
    __syncthreads();
    // rows anticommuting with Z_q (other than i) <- row * M_i
    const bool el = uh && h != i;
    if (el) {
        uint64_t xh[W], zh[W], xi[W], zi[W];
#pragma unroll
        for (int w = 0; w < W; w++) {
            xh[w] = T.mx[w * NT + h]; zh[w] = T.mz[w * NT + h];
            xi[w] = T.mx[w * NT + i]; zi[w] = T.mz[w * NT + i];
        }
        const uint32_t cbit = (uint32_t)(pauli_lambda<W>(xh, zh, xi, zi) >> 1) & 1u;
#pragma unroll
        for (int w = 0; w < W; w++) { T.mx[w * NT + h] = xh[w] ^ xi[w]; T.mz[w * NT + h] = zh[w] ^ zi[w]; }
        T.t0[h] = cbit;
        T.t1[h] = cbit;
    }
    if (__syncthreads_or(el)) {
        // D_i <- D_i * prod_{el} D_h
        cta_rows_product<W>(T.dx, T.dz, T.de, NT, el, S, S.qx, S.qz, &S.qe);
        if (h == 0) {
            int lam = 0;
#pragma unroll 1
            for (int w = 0; w < W; w++) {
                const uint64_t ax = T.dx[w * NT + i], az = T.dz[w * NT + i];
                const uint64_t bx = S.qx[w], bz = S.qz[w];
                lam += __popcll(ax & az) + __popcll(bx & bz) + 2 * __popcll(az & bx) - __popcll((ax ^ bx) & (az ^ bz));
                T.dx[w * NT + i] = ax ^ bx;
                T.dz[w * NT + i] = az ^ bz;
            }
            T.de[i] = (T.de[i] + (uint32_t)S.qe + (uint32_t)lam) & 3u;
        }
        __syncthreads();
    }
    Pauli<W> mi;
    load_m<W>(T, NT, i, mi);
    __syncthreads();
    if (h < n && h != i && (T.dx[qw * NT + h] & qm)) {
        Pauli<W> dh;
        load_d<W>(T, NT, h, dh);
        pauli_mul<W>(dh, mi);
        store_d<W>(T, NT, h, dh);
    }
    __syncthreads();
    if (h == i) {
        store_d<W>(T, NT, i, mi);
#pragma unroll
        for (int w = 0; w < W; w++) { T.mx[w * NT + i] = 0; T.mz[w * NT + i] = (w == qw) ? qm : 0ull; }
        T.t0[i] = 0;
        T.t1[i] = 1;
    }
    T.piv[h] = 0x7fffffff;
    __syncthreads();
    SortRec rec = {nullptr, nullptr, nullptr};
    if constexpr (W >= 8)
        rec = {d.piv, d.plan + plan_mv_cf(n, W), reinterpret_cast<uint32_t*>(d.plan + plan_rho_cf(n, W))};
    const int r = cta_rref<W, false>(T, n, NT, S, rec);
    if (r < 0) {
        if (h == 0) set_status(d.status, SF_ST_INTERNAL, buf, 10u);
        return;
    }
    const int den0 = cta_amp_phi<W>(T, n, NT, r, T.t0, S.y, S);
    const int den1 = cta_amp_phi<W>(T, n, NT, r, T.t1, S.y2, S);
    if (den0 < 0 || den1 < 0) {
        if (h == 0) set_status(d.status, SF_ST_INTERNAL, buf, 4u);
        return;
    }
    const double sc = (r == r0) ? 1.0 : (r > r0 ? 1.41421356237309504880 : 0.70710678118654752440);
    uint64_t* pl = d.plan;
    cta_bits<W>(h < n && T.t0[h], S.words[1]);
    cta_bits<W>(h < n && T.t1[h], S.words[2]);
    __syncthreads();
    if (h == 0) {
        const double2 k0 = ipow_mul(make_double2(sc, 0.0), (4 - den0) & 3);
        const double2 k1 = ipow_mul(make_double2(sc, 0.0), (num1 + 4 - den1) & 3);
        const size_t ko = cf_kappa(n, W);
        pl[ko + 0] = (uint64_t)__double_as_longlong(k0.x);
        pl[ko + 1] = (uint64_t)__double_as_longlong(k0.y);
        pl[ko + 2] = (uint64_t)__double_as_longlong(k1.x);
        pl[ko + 3] = (uint64_t)__double_as_longlong(k1.y);
    }
    if (h < W) {
        pl[cf_uq(n, W) + h] = S.words[4][h];
        pl[cf_vq(n, W) + h] = S.words[0][h];
        pl[cf_tau(n, W) + h] = S.words[1][h];
        pl[cf_tau(n, W) + W + h] = S.words[2][h];
    }
    // the tables (old D_hh = eps D'^{u'} M'^{v'}) are k_measure_tables' work:
    // keep the old destabilizers for it and clear the eps bit planes
    if (h < n) {
        uint64_t* d0 = pl + plan_d0(n, W);
#pragma unroll
        for (int w = 0; w < W; w++) {
            d0[(size_t)w * n + h] = T.d0x[w * NT + h];
            d0[(size_t)(W + w) * n + h] = T.d0z[w * NT + h];
        }
        d0[(size_t)2 * W * n + h] = T.d0e[h];
    }
    if (h < 2 * W) pl[cf_eps(n, W) + h] = 0ull;
    // the Z_q row of the new tableau
    if (h == 0) d.meta[1] = -1;
    __syncthreads();
    bool isrow = (h < n) && (h >= r) && (T.piv[h] == n + (int)q);
    if (isrow) d.meta[1] = h;
    if (h == 0) d.meta[2] = 1;
    store_tableau<W>(d, T, r);
}

// The cofactor tables of a random measurement (COFACTOR, Sec. III), one warp
// per old destabilizer hh: D_hh = eps_hh D'^{u'} M'^{v'} with
// u'_h = [D_hh anticommutes with M'_h], v'_h = [D_hh anticommutes with D'_h]
// over the new tableau (stored by k_measure_prep).  The D' rows commute with
// one another, and so do the M' rows, so each lane multiplies its own rows
// and the warp combines the lanes' partial products in any order; the D' part
// then multiplies the M' part (a D'_h and an M'_k anticommute only for h = k,
// and no such pair is swapped).  eps_hh is the i-power that makes the product
// equal to D_hh, written as two bit planes.
// a <- a * i^be P(x, z), the words of (x, z) read from word-major planes
// (word w at x[w * n]) as they are used
template <int W>
__device__ __forceinline__ void pauli_mul_planes(Pauli<W>& a, const uint64_t* x, const uint64_t* z, int n, int be) {
    int l = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        const uint64_t bx = __ldg(&x[w * n]), bz = __ldg(&z[w * n]);
        l += __popcll(a.x[w] & a.z[w]) + __popcll(bx & bz) + 2 * __popcll(a.z[w] & bx) -
             __popcll((a.x[w] ^ bx) & (a.z[w] ^ bz));
        a.x[w] ^= bx;
        a.z[w] ^= bz;
    }
    a.e = (a.e + be + l) & 3;
}

template <int W>
__global__ void __launch_bounds__(256) k_measure_tables(SfDev d, int buf) {
    if (*d.status) return;
    if (!d.meta[2]) return;
    const int n = d.n, lane = threadIdx.x & 31;
    const int hh = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (hh >= n) return;  // the whole warp
    uint64_t* pl = d.plan;
    const uint64_t* d0 = pl + plan_d0(n, W);
    uint64_t ox[W], oz[W];
#pragma unroll
    for (int w = 0; w < W; w++) {
        ox[w] = d0[(size_t)w * n + hh];
        oz[w] = d0[(size_t)(W + w) * n + hh];
    }
    const int oe = (int)d0[(size_t)2 * W * n + hh];
    Pauli<W> pd, pm;
    pauli_id<W>(pd);
    pauli_id<W>(pm);
#pragma unroll 1
    for (int wb = 0; wb < W; wb++) {
        uint64_t ubits = 0, vbits = 0;
#pragma unroll 1
        for (int half = 0; half < 2; half++) {
            const int h = 64 * wb + 32 * half + lane;
            bool ub = false, vb = false;
            if (h < n) {
                int cu = 0, cv = 0;
#pragma unroll
                for (int w = 0; w < W; w++) {
                    cu += __popcll(ox[w] & __ldg(&d.mz[w * n + h])) + __popcll(oz[w] & __ldg(&d.mx[w * n + h]));
                    cv += __popcll(ox[w] & __ldg(&d.dz[w * n + h])) + __popcll(oz[w] & __ldg(&d.dx[w * n + h]));
                }
                ub = cu & 1;
                vb = cv & 1;
                if (ub) pauli_mul_planes<W>(pd, d.dx + h, d.dz + h, n, (int)__ldg(&d.de[h]));
                if (vb) pauli_mul_planes<W>(pm, d.mx + h, d.mz + h, n, 0);
            }
            ubits |= (uint64_t)__ballot_sync(SF_FULL, ub) << (32 * half);
            vbits |= (uint64_t)__ballot_sync(SF_FULL, vb) << (32 * half);
        }
        if (lane == 0) {
            pl[cf_u(n, W) + (size_t)hh * W + wb] = ubits;
            pl[cf_v(n, W) + (size_t)hh * W + wb] = vbits;
        }
    }
    warp_pauli_product<W>(pd);
    warp_pauli_product<W>(pm);
    if (lane != 0) return;
    pauli_mul<W>(pd, pm);
    bool ok = true;
#pragma unroll
    for (int w = 0; w < W; w++) ok &= pd.x[w] == ox[w] && pd.z[w] == oz[w];
    if (!ok) set_status(d.status, SF_ST_INTERNAL, buf, 5u);
    const int epsq = (oe - pd.e + 4) & 3;
    unsigned long long* eps = reinterpret_cast<unsigned long long*>(pl + cf_eps(n, W));
    if (epsq & 1) atomicOr(&eps[hh >> 6], 1ull << (hh & 63));
    if (epsq & 2) atomicOr(&eps[W + (hh >> 6)], 1ull << (hh & 63));
}

// ---------------------------------------------------------------------------
// amplitude query: only elements whose Z-block signs match the parities of y
// against the Z-block rows contribute (their support must contain y).
template <int W>
__global__ void k_amp_prep(SfDev d, const uint64_t* y) {
    __shared__ uint64_t zm[W], ze[W];
    const int n = d.n, h = threadIdx.x, r = d.meta[0];
    if (h < W) { zm[h] = 0; ze[h] = 0; }
    __syncthreads();
    bool inz = false, par = false;
    if (h < n && h >= r) {
        uint64_t zr[W], yy[W];
#pragma unroll
        for (int w = 0; w < W; w++) { zr[w] = d.mz[w * n + h]; yy[w] = y[w]; }
        inz = true;
        par = popc_and<W>(zr, yy) & 1;
    }
    cta_bits<W>(inz, zm);
    cta_bits<W>(par, ze);
    __syncthreads();
    if (h < W) {
        const size_t o = plan_am(n, W);
        d.plan[o + h] = y[h];
        d.plan[o + W + h] = zm[h];
        d.plan[o + 2 * W + h] = ze[h];
    }
}

template <int W>
__global__ void k_reset(SfDev d, int buf) {
    const int n = d.n, h = threadIdx.x;
    if (h < n) {
        for (int w = 0; w < W; w++) {
            const uint64_t e = (w == (h >> 6)) ? (1ull << (h & 63)) : 0ull;
            d.mx[w * n + h] = 0;
            d.mz[w * n + h] = e;
            d.dx[w * n + h] = e;
            d.dz[w * n + h] = 0;
        }
        d.de[h] = 0;
        d.piv[h] = n + h;
    }
    if (h < W) d.sig[buf][(size_t)h * d.cap] = 0;
    if (h == 0) {
        d.meta[0] = 0;
        d.meta[1] = -1;
        d.meta[2] = 0;
        *d.g = make_double2(1.0, 0.0);
        d.amp[buf][0] = make_double2(1.0, 0.0);
        d.kcnt[buf] = 1;
        d.kcnt[buf ^ 1] = 0;
        *d.status = 0;
        *d.done = 0u;
        *d.ocnt = 0ull;
        // index of the one-element frame
        const uint32_t tag = next_tag(d.itag[buf]);
        uint64_t zero[W];
        for (int w = 0; w < W; w++) zero[w] = 0;
        index_insert<W>(d, buf, 64, tag, zero, 0u);
        d.itag[buf] = tag;
        d.isize[buf] = 64;
    }
}

template <int W>
size_t ws_bytes(int NT) {
    return (size_t)7 * W * NT * 8 + (size_t)5 * NT * 4 + 16;
}

template <int W, typename K>
uint64_t* pick_ws(const SfDev& d, K kern, size_t& smem, uint64_t* gws, int which) {
    const size_t need = ws_bytes<W>(d.NT);
    if (need <= 200 * 1024) {
        smem = need;
        // once per kernel, thread-safe (handles may be driven from several host threads)
        static const bool attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      200 * 1024) == cudaSuccess;
        (void)attr;
        return nullptr;
    }
    smem = 0;
    return gws;
}

}  // namespace

size_t sf_tableau_smem_bytes(int n, int W, int NT) {
    switch (W) {
        case 1: return ws_bytes<1>(NT);
        case 2: return ws_bytes<2>(NT);
        case 4: return ws_bytes<4>(NT);
        case 8: return ws_bytes<8>(NT);
        default: return ws_bytes<16>(NT);
    }
}

#define SF_DISPATCH(W_, ...)                                  \
    switch (W_) {                                             \
        case 1: { constexpr int WW = 1; __VA_ARGS__; } break; \
        case 2: { constexpr int WW = 2; __VA_ARGS__; } break; \
        case 4: { constexpr int WW = 4; __VA_ARGS__; } break; \
        case 8: { constexpr int WW = 8; __VA_ARGS__; } break; \
        default: { constexpr int WW = 16; __VA_ARGS__; } break; \
    }

void sf_launch_reset(const SfDev& d, int buf, cudaStream_t s) {
    SF_DISPATCH(d.W, k_reset<WW><<<1, d.NT, 0, s>>>(d, buf));
}

void sf_launch_clifford(const SfDev& d, const void* dev_gates, int ngates, int buf, uint64_t* gws, cudaStream_t s) {
    if (d.W == 1) {  // n <= 63: one warp, rows in registers
        sf_launch_clifford_warp(d, dev_gates, ngates, buf, s);
        return;
    }
    SF_DISPATCH(d.W, {
        size_t sm;
        uint64_t* ws = pick_ws<WW>(d, k_clifford<WW>, sm, gws, 0);
        k_clifford<WW><<<1, d.NT, sm, s>>>(d, reinterpret_cast<const sf_gate_rec*>(dev_gates), ngates, buf, ws);
    });
}

void sf_launch_measure_prep(const SfDev& d, uint32_t q, int buf, uint64_t* gws, cudaStream_t s) {
    if (d.W == 1) {  // n <= 63: one warp with the rows in registers
        sf_launch_measure_prep_warp(d, q, buf, s);
        return;
    }
    SF_DISPATCH(d.W, {
        size_t sm;
        uint64_t* ws = pick_ws<WW>(d, k_measure_prep<WW>, sm, gws, 1);
        k_measure_prep<WW><<<1, d.NT, sm, s>>>(d, q, buf, ws);
        k_measure_tables<WW><<<(d.n + 7) / 8, 256, 0, s>>>(d, buf);
    });
}

void sf_launch_amp_prep(const SfDev& d, const uint64_t* dev_y, cudaStream_t s) {
    SF_DISPATCH(d.W, k_amp_prep<WW><<<1, d.NT, 0, s>>>(d, dev_y));
}
