// sf_warp.cuh -- single-warp tableau primitives for n <= 63 (one 64-bit word
// per row half): lane L holds tableau rows L and L + 32 in registers.  Used by
// the single-warp Clifford kernel and by the batched campaign engine.
#pragma once
#include "sf_device.cuh"

namespace sfw {

struct Row {
    uint64_t mx, mz, dx, dz, A;
    uint32_t de, t0, t1;
    int piv;
};

__device__ __forceinline__ int lam1(uint64_t x1, uint64_t z1, uint64_t x2, uint64_t z2) {
    return (__popcll(x1 & z1) + __popcll(x2 & z2) + 2 * __popcll(z1 & x2) - __popcll((x1 ^ x2) & (z1 ^ z2))) & 3;
}

// (x, z, e) <- (x, z, e) * (x2, z2, e2)
__device__ __forceinline__ void pmul1(uint64_t& x, uint64_t& z, int& e, uint64_t x2, uint64_t z2, int e2) {
    const int l = lam1(x, z, x2, z2);
    x ^= x2;
    z ^= z2;
    e = (e + e2 + l) & 3;
}

// product of commuting Pauli operators over the warp, result in every lane
__device__ __forceinline__ void warp_prod(uint64_t& x, uint64_t& z, int& e) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const uint64_t ox = __shfl_xor_sync(SF_FULL, x, off);
        const uint64_t oz = __shfl_xor_sync(SF_FULL, z, off);
        const int oe = __shfl_xor_sync(SF_FULL, e, off);
        pmul1(x, z, e, ox, oz, oe);
    }
}

// Table 2 conjugation of one row held in registers; returns the sign flip
__device__ __forceinline__ int conj1(int kind, int q0, int q1, uint64_t& x, uint64_t& z) {
    const uint64_t m0 = 1ull << q0;
    const int xa = (int)((x >> q0) & 1), za = (int)((z >> q0) & 1);
    int f = 0;
    switch (kind) {
        case 0: f = xa & za; if (xa != za) { x ^= m0; z ^= m0; } break;
        case 1: f = xa & za; if (xa) z ^= m0; break;
        case 2: f = xa & (za ^ 1); if (xa) z ^= m0; break;
        case 3: f = za; break;
        case 4: f = xa ^ za; break;
        case 5: f = xa; break;
        default: {
            const uint64_t m1 = 1ull << q1;
            const int xb = (int)((x >> q1) & 1), zb = (int)((z >> q1) & 1);
            if (kind == 6) {
                f = xa & zb & (xb ^ za ^ 1);
                if (xa) x ^= m1;
                if (zb) z ^= m0;
            } else if (kind == 7) {
                f = xa & xb & (za ^ zb);
                if (xa) z ^= m1;
                if (xb) z ^= m0;
            } else {
                if (xa != xb) { x ^= m0 | m1; }
                if (za != zb) { z ^= m0 | m1; }
            }
        }
    }
    return f;
}

// every field of row `row` (held by lane row & 31, half row >> 5) in every lane
__device__ __forceinline__ Row fetch_row(const Row* r, int row) {
    const int src = row & 31, half = row >> 5;
    Row o;
    o.mx = __shfl_sync(SF_FULL, half ? r[1].mx : r[0].mx, src);
    o.mz = __shfl_sync(SF_FULL, half ? r[1].mz : r[0].mz, src);
    o.dx = __shfl_sync(SF_FULL, half ? r[1].dx : r[0].dx, src);
    o.dz = __shfl_sync(SF_FULL, half ? r[1].dz : r[0].dz, src);
    o.A = __shfl_sync(SF_FULL, half ? r[1].A : r[0].A, src);
    o.de = __shfl_sync(SF_FULL, half ? r[1].de : r[0].de, src);
    o.t0 = __shfl_sync(SF_FULL, half ? r[1].t0 : r[0].t0, src);
    o.t1 = __shfl_sync(SF_FULL, half ? r[1].t1 : r[0].t1, src);
    o.piv = __shfl_sync(SF_FULL, half ? r[1].piv : r[0].piv, src);
    return o;
}

__device__ __forceinline__ int colbit(const Row& a, int c, int n) {
    return c < n ? (int)((a.mx >> c) & 1) : (int)((a.mz >> (c - n)) & 1);
}

// <y| D^tau phi_0(M)> 2^{r/2} as an i-power, -1 if zero (tau = t1 bits, or none)
__device__ __forceinline__ int warp_amp_phi_sel(const Row* r, int n, int rx, int tau_sel, uint64_t y);
__device__ __forceinline__ int warp_amp_phi(const Row* r, int n, int rx, bool use_tau, uint64_t y) {
    return warp_amp_phi_sel(r, n, rx, use_tau ? 2 : 0, y);
}
// tau_sel: 0 none, 1 the t0 bits, 2 the t1 bits
__device__ __forceinline__ int warp_amp_phi_sel(const Row* r, int n, int rx, int tau_sel, uint64_t y) {
    const int lane = threadIdx.x & 31;
    uint64_t qx = 0, qz = 0;
    int qe = 0;
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        const uint32_t tb = tau_sel == 1 ? r[hf].t0 : (tau_sel == 2 ? r[hf].t1 : 0u);
        if (row < n && tb) pmul1(qx, qz, qe, r[hf].dx, r[hf].dz, (int)r[hf].de);
    }
    warp_prod(qx, qz, qe);
    const uint64_t w = y ^ qx;
    uint64_t px = 0, pz = 0;
    int pe = 0;
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        if (row < rx && ((w >> r[hf].piv) & 1)) pmul1(px, pz, pe, r[hf].mx, r[hf].mz, 0);
    }
    warp_prod(px, pz, pe);
    if (px != w) return -1;
    return (qe + __popcll(qx & qz) + 2 * __popcll(qz & w) + pe + __popcll(px & pz)) & 3;
}

// ---- Invariant 1 repair without row movement --------------------------------
// The same row reduction with the rows left in place while pivots are chosen:
// every unassigned row whose leading column holds no other 1 in the whole
// tableau becomes that column's pivot at once (Gauss-Jordan would reach it
// with nothing to eliminate, whatever the order), and only columns that hold
// several 1s take an elimination step (pivot = lowest-index unassigned row
// leading there; every other row with that bit gets M_h <- M_h M_p, the dual
// D_p <- D_p D_h, and the affine / sign tracking).  A final permutation sorts
// the rows by pivot.  The canonical M is the unique RREF of the row space;
// the destabilizers may differ from a reduction that swaps rows, which
// changes the internal labels but not the state any element stands for.  The
// block kernel of sf_tableau.cu runs the same algorithm.
// `stage` is 64 rows of shared memory owned by the calling warp.  Returns r,
// or -1 if a row has no bits left (dependent rows: a broken tableau).
__device__ __forceinline__ int lead_col(uint64_t mx, uint64_t mz, int n) {
    if (mx) return __ffsll((long long)mx) - 1;
    if (mz) return n + __ffsll((long long)mz) - 1;
    return 0x7fffffff;
}

__device__ __forceinline__ uint64_t warp_or64(uint64_t v) {
    const unsigned lo = __reduce_or_sync(SF_FULL, (unsigned)v);
    const unsigned hi = __reduce_or_sync(SF_FULL, (unsigned)(v >> 32));
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

// column c as a bit of the (x part, z part) pair
__device__ __forceinline__ void col_bit(int c, int n, uint64_t& bx, uint64_t& bz) {
    bx = c < n ? 1ull << c : 0ull;
    bz = (c >= n && c < 2 * n) ? 1ull << (c - n) : 0ull;
}

__device__ __forceinline__ bool col_in(int c, int n, uint64_t sx, uint64_t sz) {
    return c < n ? ((sx >> c) & 1) : ((sz >> (c - n)) & 1);
}

__device__ __forceinline__ void elim_row(Row& a, const Row& pv, int c, int n, uint64_t& dx, uint64_t& dz, int& de,
                                         bool& any) {
    if (!col_in(c, n, a.mx, a.mz)) return;
    const uint32_t cb = (uint32_t)(lam1(a.mx, a.mz, pv.mx, pv.mz) >> 1) & 1u;
    a.mx ^= pv.mx;
    a.mz ^= pv.mz;
    a.A ^= pv.A;
    a.t0 ^= pv.t0 ^ cb;
    a.t1 ^= pv.t1 ^ cb;
    pmul1(dx, dz, de, a.dx, a.dz, (int)a.de);
    any = true;
}

__device__ __forceinline__ void take_pivot(Row& t, int c, bool with_d, uint64_t dx, uint64_t dz, int de) {
    if (with_d) {
        uint64_t x = t.dx, z = t.dz;
        int e = (int)t.de;
        pmul1(x, z, e, dx, dz, de);
        t.dx = x;
        t.dz = z;
        t.de = (uint32_t)e;
    }
    t.piv = c;
}

// pivot preference among the rows leading at column c: the next 1 after c
// furthest right first (no further 1: best), then the lowest row index
__device__ __forceinline__ unsigned pivot_key(const Row& a, int c, int n, int row) {
    uint64_t bx, bz;
    col_bit(c, n, bx, bz);
    const int nl = lead_col(a.mx & ~bx, a.mz & ~bz, n);
    const unsigned rank = nl == 0x7fffffff ? 0u : (unsigned)(2047 - nl);
    return (rank << 6) | (unsigned)row;
}

// Optionally (C, cstage non-null) the rows of C = A^-T ride along, two per
// lane like the rows: a step A_a ^= A_p over the eliminated rows a is
// C_p ^= XOR of their C_a (A' = E A with E = I + s e_p^T, E^-1 = E, so
// A'^-T = E^T A^-T), and the sort moves C with its row (cstage: 64 words of
// shared memory owned by the warp).  The rows of A^-1 are then C's columns.
__device__ __forceinline__ int warp_rref(Row* r, int n, Row* stage, uint64_t* C = nullptr,
                                         uint64_t* cstage = nullptr) {
    const int lane = threadIdx.x & 31;
    constexpr int INF = 0x7fffffff;
    const bool v0 = lane < n, v1 = lane + 32 < n;
    bool asg0 = false, asg1 = false;
    for (int it = 0; it < 64; it++) {
        const int l0 = v0 ? (asg0 ? r[0].piv : lead_col(r[0].mx, r[0].mz, n)) : INF;
        const int l1 = v1 ? (asg1 ? r[1].piv : lead_col(r[1].mx, r[1].mz, n)) : INF;
        // bits other than each row's lead, and the leads of each half
        uint64_t b0x, b0z, b1x, b1z;
        col_bit(l0, n, b0x, b0z);
        col_bit(l1, n, b1x, b1z);
        const uint64_t nx = (v0 ? r[0].mx & ~b0x : 0ull) | (v1 ? r[1].mx & ~b1x : 0ull);
        const uint64_t nz = (v0 ? r[0].mz & ~b0z : 0ull) | (v1 ? r[1].mz & ~b1z : 0ull);
        const uint64_t dirty_x = warp_or64(nx), dirty_z = warp_or64(nz);
        const uint64_t cross_x = warp_or64(b0x) & warp_or64(b1x);
        const uint64_t cross_z = warp_or64(b0z) & warp_or64(b1z);
        const unsigned m0 = __match_any_sync(SF_FULL, l0), m1 = __match_any_sync(SF_FULL, l1);
        const bool c0 = v0 && !asg0 && l0 != INF && __popc(m0) == 1 &&
                        !col_in(l0, n, dirty_x | cross_x, dirty_z | cross_z);
        const bool c1 = v1 && !asg1 && l1 != INF && __popc(m1) == 1 &&
                        !col_in(l1, n, dirty_x | cross_x, dirty_z | cross_z);
        if (c0) { asg0 = true; r[0].piv = l0; }
        if (c1) { asg1 = true; r[1].piv = l1; }
        const int u0 = (v0 && !asg0) ? l0 : INF, u1 = (v1 && !asg1) ? l1 : INF;
        const int c = __reduce_min_sync(SF_FULL, min(u0, u1));
        if (c == INF) break;
        // one elimination step at column c; pivot: the candidate whose next 1
        // after c lies furthest right (lowest row index on ties), so that the
        // other candidates keep their own next 1 as lead and no chain of steps
        // follows
        const unsigned k0 = u0 == c ? pivot_key(r[0], c, n, lane) : 0xffffffffu;
        const unsigned k1 = u1 == c ? pivot_key(r[1], c, n, lane + 32) : 0xffffffffu;
        const int p = (int)(__reduce_min_sync(SF_FULL, min(k0, k1)) & 63u);
        const Row pv = fetch_row(r, p);
        uint64_t dx = 0, dz = 0;
        int de = 0;
        bool any = false;
        const bool e0 = v0 && lane != p && col_in(c, n, r[0].mx, r[0].mz);
        const bool e1 = v1 && lane + 32 != p && col_in(c, n, r[1].mx, r[1].mz);
        if (v0 && lane != p) elim_row(r[0], pv, c, n, dx, dz, de, any);
        if (v1 && lane + 32 != p) elim_row(r[1], pv, c, n, dx, dz, de, any);
        const bool with_d = __any_sync(SF_FULL, any);
        if (with_d) warp_prod(dx, dz, de);
        if (C) {
            uint64_t cs = (e0 ? C[0] : 0ull) ^ (e1 ? C[1] : 0ull);
#pragma unroll
            for (int off = 16; off; off >>= 1) cs ^= __shfl_xor_sync(SF_FULL, cs, off);
            if (lane == (p & 31)) C[p >> 5] ^= cs;
        }
        if (lane == (p & 31)) {
            if (p < 32) { take_pivot(r[0], c, with_d, dx, dz, de); asg0 = true; }
            else { take_pivot(r[1], c, with_d, dx, dz, de); asg1 = true; }
        }
    }
    if (__any_sync(SF_FULL, (v0 && !asg0) || (v1 && !asg1))) return -1;
    // sort by pivot: rank = number of pivots in smaller columns
    uint64_t p0x, p0z, p1x, p1z;
    col_bit(v0 ? r[0].piv : INF, n, p0x, p0z);
    col_bit(v1 ? r[1].piv : INF, n, p1x, p1z);
    const uint64_t PX = warp_or64(p0x | p1x), PZ = warp_or64(p0z | p1z);
    const int rx = __popcll(PX);
    auto rank = [&](int pc) {
        return pc < n ? __popcll(PX & ((1ull << pc) - 1)) : rx + __popcll(PZ & ((1ull << (pc - n)) - 1));
    };
    const int k0 = v0 ? rank(r[0].piv) : lane, k1 = v1 ? rank(r[1].piv) : lane + 32;
    if (__any_sync(SF_FULL, k0 != lane || k1 != lane + 32)) {
        if (v0) stage[k0] = r[0];
        if (v1) stage[k1] = r[1];
        if (C) {
            if (v0) cstage[k0] = C[0];
            if (v1) cstage[k1] = C[1];
        }
        __syncwarp();
        if (v0) r[0] = stage[lane];
        if (v1) r[1] = stage[lane + 32];
        if (C) {
            if (v0) C[0] = cstage[lane];
            if (v1) C[1] = cstage[lane + 32];
        }
        __syncwarp();
    }
    return rx;
}

// ---- cofactor planning (COFACTOR, Sec. III) with the rows in registers -------
// The same construction as the block kernel k_measure_prep: if q is random,
// rows anticommuting with Z_q are multiplied by the first such row i (dual
// D_i <- D_i D_h), destabilizers anticommuting with Z_q take a factor M_i,
// D_i <- M_i, M_i <- Z_q, Gauss-Jordan; then kappa_y, tau_y and, for every old
// destabilizer, D_h = eps_h D'^{u'_h} M'^{v'_h}.
struct CofTab {
    uint64_t u[64], v[64];
    uint64_t eps0, eps1, tau0, tau1, vq, uq;
    double2 kap[2];
    int rq, random, bad;
};

__device__ __forceinline__ int symp1(uint64_t ax, uint64_t az, uint64_t bx, uint64_t bz) {
    return (__popcll(ax & bz) + __popcll(az & bx)) & 1;
}

// lane 0 writes C; returns the new X-block size
__device__ __forceinline__ int warp_measure_prep(Row* r, int n, int rx, int q, CofTab& C, Row* stage) {
    const int lane = threadIdx.x & 31;
    const uint64_t qm = 1ull << q;
    bool uh[2];
    for (int hf = 0; hf < 2; hf++) uh[hf] = (lane + 32 * hf < n) && (r[hf].mx & qm);
    const uint64_t umask = (uint64_t)__ballot_sync(SF_FULL, uh[0]) | ((uint64_t)__ballot_sync(SF_FULL, uh[1]) << 32);
    if (!umask) {
        // deterministic: Z_q is a canonical Z-block row
        int rq = -1;
        for (int hf = 0; hf < 2; hf++) {
            const int row = lane + 32 * hf;
            if (row < n && row >= rx && r[hf].piv == n + q && r[hf].mx == 0 && r[hf].mz == qm) rq = row;
        }
        for (int off = 16; off; off >>= 1) rq = max(rq, __shfl_xor_sync(SF_FULL, rq, off));
        if (lane == 0) { C.random = 0; C.rq = rq; C.bad = rq < 0; }
        return rx;
    }
    const int i = __ffsll((long long)umask) - 1;
    const Row ri = fetch_row(r, i);
    const int num1 = __popcll(ri.mx & ri.mz) & 3;
    const uint64_t w1 = ri.mx;
    const uint64_t vq = (uint64_t)__ballot_sync(SF_FULL, lane < n && (r[0].dx & qm)) |
                        ((uint64_t)__ballot_sync(SF_FULL, lane + 32 < n && (r[1].dx & qm)) << 32);
    uint64_t d0x[2], d0z[2];
    uint32_t d0e[2];
    for (int hf = 0; hf < 2; hf++) {
        d0x[hf] = r[hf].dx;
        d0z[hf] = r[hf].dz;
        d0e[hf] = r[hf].de;
        r[hf].t0 = 0;
        r[hf].t1 = 0;
    }
    // rows anticommuting with Z_q (other than i) <- row * M_i; dual on D_i
    uint64_t px = 0, pz = 0;
    int pe = 0;
    bool any = false;
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        if (uh[hf] && row != i) {
            const uint32_t cb = (uint32_t)(lam1(r[hf].mx, r[hf].mz, ri.mx, ri.mz) >> 1) & 1u;
            r[hf].mx ^= ri.mx;
            r[hf].mz ^= ri.mz;
            r[hf].t0 = cb;
            r[hf].t1 = cb;
            pmul1(px, pz, pe, r[hf].dx, r[hf].dz, (int)r[hf].de);
            any = true;
        }
    }
    if (__any_sync(SF_FULL, any)) {
        warp_prod(px, pz, pe);
        if (lane == (i & 31)) {
            if (i < 32) take_pivot(r[0], r[0].piv, true, px, pz, pe);
            else take_pivot(r[1], r[1].piv, true, px, pz, pe);
        }
    }
    // destabilizers anticommuting with Z_q take a factor M_i (commutes with them)
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        if (row < n && row != i && (r[hf].dx & qm)) {
            uint64_t x = r[hf].dx, z = r[hf].dz;
            int e = (int)r[hf].de;
            pmul1(x, z, e, ri.mx, ri.mz, 0);
            r[hf].dx = x;
            r[hf].dz = z;
            r[hf].de = (uint32_t)e;
        }
    }
#pragma unroll
    for (int hf = 0; hf < 2; hf++) {
        if (lane + 32 * hf == i) {
            r[hf].dx = ri.mx;
            r[hf].dz = ri.mz;
            r[hf].de = 0;
            r[hf].mx = 0;
            r[hf].mz = qm;
            r[hf].t0 = 0;
            r[hf].t1 = 1;
        }
        r[hf].piv = 0x7fffffff;
    }
    const int rx2 = warp_rref(r, n, stage);
    const int den0 = warp_amp_phi_sel(r, n, rx2, 1, 0ull);
    const int den1 = warp_amp_phi_sel(r, n, rx2, 2, w1);
    const uint64_t tau0 = (uint64_t)__ballot_sync(SF_FULL, lane < n && r[0].t0) |
                          ((uint64_t)__ballot_sync(SF_FULL, lane + 32 < n && r[1].t0) << 32);
    const uint64_t tau1 = (uint64_t)__ballot_sync(SF_FULL, lane < n && r[0].t1) |
                          ((uint64_t)__ballot_sync(SF_FULL, lane + 32 < n && r[1].t1) << 32);
    const double sc = rx2 == rx ? 1.0 : (rx2 > rx ? 1.41421356237309504880 : 0.70710678118654752440);
    // tables of the old destabilizers in the new basis
    uint64_t eps0 = 0, eps1 = 0;
    int bad = (den0 < 0 || den1 < 0 || rx2 < 0) ? 1 : 0;
    for (int hh = 0; hh < n; hh++) {
        const int src = hh & 31, half = hh >> 5;
        const uint64_t ox = __shfl_sync(SF_FULL, half ? d0x[1] : d0x[0], src);
        const uint64_t oz = __shfl_sync(SF_FULL, half ? d0z[1] : d0z[0], src);
        const int oe = (int)__shfl_sync(SF_FULL, half ? d0e[1] : d0e[0], src);
        bool ub[2], vb[2];
        uint64_t cx = 0, cz = 0;
        int ce = 0;
        for (int hf = 0; hf < 2; hf++) {
            const int row = lane + 32 * hf;
            ub[hf] = row < n && symp1(ox, oz, r[hf].mx, r[hf].mz);
            vb[hf] = row < n && symp1(ox, oz, r[hf].dx, r[hf].dz);
            if (ub[hf]) pmul1(cx, cz, ce, r[hf].dx, r[hf].dz, (int)r[hf].de);
            if (vb[hf]) pmul1(cx, cz, ce, r[hf].mx, r[hf].mz, 0);
        }
        const uint64_t um = (uint64_t)__ballot_sync(SF_FULL, ub[0]) | ((uint64_t)__ballot_sync(SF_FULL, ub[1]) << 32);
        const uint64_t vm = (uint64_t)__ballot_sync(SF_FULL, vb[0]) | ((uint64_t)__ballot_sync(SF_FULL, vb[1]) << 32);
        warp_prod(cx, cz, ce);
        if (cx != ox || cz != oz) bad = 1;
        const int epsq = (oe - ce + 4) & 3;
        if (epsq & 1) eps0 |= 1ull << hh;
        if (epsq & 2) eps1 |= 1ull << hh;
        if (lane == 0) {
            C.u[hh] = um;
            C.v[hh] = vm;
        }
    }
    int rq = -1;
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        if (row < n && row >= rx2 && r[hf].piv == n + q) rq = row;
    }
    for (int off = 16; off; off >>= 1) rq = max(rq, __shfl_xor_sync(SF_FULL, rq, off));
    if (lane == 0) {
        C.random = 1;
        C.rq = rq;
        C.bad = bad | (rq < 0);
        C.eps0 = eps0;
        C.eps1 = eps1;
        C.tau0 = tau0;
        C.tau1 = tau1;
        C.vq = vq;
        C.uq = umask;
        C.kap[0] = ipow_mul(make_double2(sc, 0.0), (4 - den0) & 3);
        C.kap[1] = ipow_mul(make_double2(sc, 0.0), (num1 + 4 - den1) & 3);
    }
    return rx2;
}

// A run of Pauli gates as one Pauli P = i^e X^a Z^b (ROTATE, Sec. III): the
// rows that anticommute with P change sign (M's to t0, composed, and t1; D's
// to de), M keeps its bits and stays in RREF, and the phase rule takes one
// point: <a|P phi_0> = i^e <0|phi_0> (0 lies in the support of phi_0), over
// <a|D^{t1} phi_0>.  The product of the gates' own factors is the same number.
__device__ __forceinline__ bool warp_pauli_run(Row* r, int n, int rx, uint64_t a, uint64_t b, int e, int& ga) {
    const int lane = threadIdx.x & 31;
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        if (row < n) {
            const uint32_t f = (uint32_t)((__popcll(r[hf].mx & b) + __popcll(r[hf].mz & a)) & 1);
            r[hf].t0 ^= f;
            r[hf].t1 = f;
            const uint32_t fd = (uint32_t)((__popcll(r[hf].dx & b) + __popcll(r[hf].dz & a)) & 1);
            r[hf].de = (r[hf].de + 2u * fd) & 3u;
        } else {
            r[hf].t1 = 0;
        }
    }
    const int dq = warp_amp_phi(r, n, rx, true, a);
    if (dq < 0) return false;
    ga = (ga + 2 * e + 2 * ((4 - dq) & 3)) & 7;
    return true;
}

// One Clifford gate on the rows in registers (ROTATE, Sec. III, Table 2):
// conjugate M and D (sign flips of M to t0, composed, and t1, this gate),
// restore Invariant 1, and multiply the run's phase factor omega^ga sqrt(2)^gb
// by the gate's.  rx is the X-block size.  Returns false if the phase rule
// finds no point (an internal error).
__device__ __forceinline__ bool warp_clifford_gate(Row* r, int n, int& rx, int kind, int q0, int q1, Row* stage,
                                                   int& ga, int& gb, uint64_t* C = nullptr, uint64_t* cstage = nullptr) {
    const int lane = threadIdx.x & 31;
    // numerator of the phase rule: a point y with <y|U phi_0(M)> != 0
    int yq = -1, cq = -1;
    if (kind == 0) {
        cq = warp_amp_phi(r, n, rx, false, 1ull << q0);
        if (cq == 2) yq = q0;
    } else if (kind == 3 || kind == 4) {
        yq = q0;
    }
    int na, nb;
    cliff_num_exp(kind, cq, na, nb);
    const int r_old = rx;
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        if (row < n) {
            const uint32_t f = (uint32_t)conj1(kind, q0, q1, r[hf].mx, r[hf].mz);
            r[hf].t0 ^= f;
            r[hf].t1 = f;
            const int fd = conj1(kind, q0, q1, r[hf].dx, r[hf].dz);
            r[hf].de = (r[hf].de + 2u * (uint32_t)fd) & 3u;
        } else {
            r[hf].t1 = 0;
        }
    }
    // Pauli gates flip signs only: M keeps its bits and stays in RREF
    if (kind < 3 || kind > 5) rx = warp_rref(r, n, stage, C, cstage);
    // denominator: <y| D'^{t1} phi_0(M')>
    const int dq = rx < 0 ? -1 : warp_amp_phi(r, n, rx, true, yq >= 0 ? (1ull << yq) : 0ull);
    if (dq < 0) return false;
    const int dr = rx - r_old;
    ga = (ga + na + 2 * ((4 - dq) & 3)) & 7;
    gb += nb + (dr > 0) - (dr < 0);
    return true;
}

// ---- plan of a diagonal gate (Sec. IV) with the rows in registers ---------------
// Terms c_j Z^{w_j}; Z^w = eps D^u M^v; terms grouped by u (group 0: u = 0).
struct BrTab {
    int ng, bad;
    int nt[4];
    int fl[4];  // sign-pattern bits flipped for every element (0 unless the plan was moved to other coordinates)
    uint64_t u[4];
    uint64_t v[4][4];
    double2 c[4][4];
    int xidx[4][4];
};

// coefficient of group g of a plan for parent phase vector x: the sign
// pattern of the group's terms, looked up in the half table (patterns with
// the last term's bit set are the negations of their complements)
__device__ __forceinline__ double2 half_coef(const BrTab& P, const double2 (*ctab)[16], int g, uint64_t x) {
    const int ntg = P.nt[g];
    int pat = P.fl[g];
    for (int t = 0; t < ntg; t++) pat ^= (__popcll(P.v[g][t] & x) & 1) << t;
    const bool neg = (pat >> (ntg - 1)) & 1;
    const double2 cc = ctab[g][neg ? pat ^ ((1 << ntg) - 1) : pat];
    return make_double2(dneg_if(cc.x, neg), dneg_if(cc.y, neg));
}

// One warp's share of an in-place run of diagonal gates (plan(r) for r in
// [r0, r1) gives the gate's BrTab and half table) on the elements [base,
// base + 64) of a frame of hi elements: with pairs, each pair {s, s ^ cu}
// is carried by its element with the smaller phase vector, and those owners
// are packed onto consecutive lanes first, so no lane idles through the FP64
// pipe (a double-precision instruction costs the same for 1 lane as for 32).
// A window can hold up to 64 owners (the partners of its elements may sit in
// other windows), so the owners are taken 32 at a time.
// find(key) is the position of a phase vector, kL2: the frame is read through
// L2 (written by other CTAs of the launch).  Sets drop if a result is below
// the threshold, miss if a partner is absent.
template <bool kL2, class Plan, class Find>
__device__ __forceinline__ void inplace_run_warp(const uint64_t* S, double2* A, unsigned long long base,
                                                 unsigned long long hi, bool pairs, uint64_t cu, int r0, int r1,
                                                 Plan plan, Find find, unsigned long long kb, double eps2, bool& drop,
                                                 bool& miss) {
    const int lane = threadIdx.x & 31;
    const unsigned long long ja = base + lane, jb = base + 32 + lane;
    uint64_t sa = 0, sb = 0;
    if (ja < hi) sa = kL2 ? __ldcg(&S[ja]) : S[ja];
    if (jb < hi) sb = kL2 ? __ldcg(&S[jb]) : S[jb];
    const bool oa = ja < hi && (!pairs || (sa ^ cu) > sa), ob = jb < hi && (!pairs || (sb ^ cu) > sb);
    const unsigned ma = __ballot_sync(SF_FULL, oa), mb = __ballot_sync(SF_FULL, ob);
    const int na = __popc(ma), cnt = na + __popc(mb);
    for (int first = 0; first < cnt; first += 32) {
        // lane l takes owner first + l of the 64 elements
        const int l = first + lane;
        unsigned m = l < na ? ma : mb;
        for (int i = l < na ? l : l - na; i > 0 && m; i--) m &= m - 1;
        const int src = m ? __ffs(m) - 1 : 0;
        const uint64_t s_a = __shfl_sync(SF_FULL, sa, src), s_b = __shfl_sync(SF_FULL, sb, src);
        if (l >= cnt) continue;
        const bool second = l >= na;
        const uint64_t s0 = second ? s_b : s_a, s1 = s0 ^ cu;
        const unsigned long long j = base + (second ? 32 : 0) + src;
        long long q = -1;
        if (pairs) {
            q = find(s1);
            if (q < 0) {
                miss = true;
                continue;
            }
        }
        double2 a0 = kL2 ? __ldcg(&A[j]) : A[j];
        double2 a1 = make_double2(0.0, 0.0);
        if (q >= 0) a1 = kL2 ? __ldcg(&A[q]) : A[q];
        for (int r = r0; r < r1; r++) {
            const BrTab& Q = *plan(r).P;
            const double2(*ct)[16] = plan(r).ctab;
            double2 n0 = make_double2(0.0, 0.0), n1 = make_double2(0.0, 0.0);
            cmul_acc(n0, half_coef(Q, ct, 0, s0), a0);
            if (pairs) {
                if (Q.ng == 2) cmul_acc(n0, half_coef(Q, ct, 1, s1), a1);
                cmul_acc(n1, half_coef(Q, ct, 0, s1), a1);
                if (Q.ng == 2) cmul_acc(n1, half_coef(Q, ct, 1, s0), a0);
            }
            a0 = n0;
            a1 = n1;
        }
        A[j] = a0;
        if (q >= 0) A[q] = a1;
        drop |= !amp_kept(a0, kb, eps2) || (q >= 0 && !amp_kept(a1, kb, eps2));
    }
}

struct PlanRef {
    const BrTab* P;
    const double2 (*ctab)[16];
};

// cf: the nt term coefficients of the gate (diag_terms).  Every lane derives
// the groups from warp-uniform values; the lanes split the writes of P and of
// the coefficient table.  ctab[g][p] holds sum_t (-1)^{bit t of p} c_t for
// the patterns p of group g whose last-term bit is clear (terms in order); the
// other half are their negations.  A double-precision instruction costs the
// same pipe time for one lane as for 32, so the table takes one add per extra
// term of the largest group, all lanes at once.
__device__ __forceinline__ void warp_branch_plan_regs(const Row* r, int n, uint32_t kind, int q0, int q1,
                                                      const double2* cf, BrTab& P, double2 (*ctab)[16]) {
    const int lane = threadIdx.x & 31;
    const int nt = kind <= 2 ? 2 : 4;
    uint64_t wz[4];
    wz[0] = 0;
    wz[1] = 1ull << q0;
    wz[2] = kind == 3 ? 1ull << q1 : 0;
    wz[3] = wz[1] | wz[2];
    // Z^{w_j} = eps_j D^{u_j} M^{v_j} for the one-qubit terms j = 1, 2, both
    // decompositions interleaved (u_h = [Z^w anticommutes with M_h],
    // v_h = [Z^w anticommutes with D_h], product of D_h^{u_h} M_h^{v_h})
    uint64_t cx[2] = {0, 0}, cz[2] = {0, 0};
    int ce[2] = {0, 0};
    bool ub[2][2], vb[2][2];
#pragma unroll
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        const uint64_t mx = r[hf].mx, mz = r[hf].mz, dx = r[hf].dx, dz = r[hf].dz;
        const int de = (int)r[hf].de;
#pragma unroll
        for (int a = 0; a < 2; a++) {
            const uint64_t w = wz[1 + a];
            ub[a][hf] = row < n && (__popcll(mx & w) & 1);
            vb[a][hf] = row < n && (__popcll(dx & w) & 1);
            if (ub[a][hf]) pmul1(cx[a], cz[a], ce[a], dx, dz, de);
            if (vb[a][hf]) pmul1(cx[a], cz[a], ce[a], mx, mz, 0);
        }
    }
    uint64_t um[4], vm[4];
    int epsq[4], bad = 0;
    um[0] = vm[0] = 0;
    epsq[0] = 0;  // the identity term: u = v = 0, eps = 1
#pragma unroll
    for (int a = 0; a < 2; a++) {
        um[1 + a] = (uint64_t)__ballot_sync(SF_FULL, ub[a][0]) | ((uint64_t)__ballot_sync(SF_FULL, ub[a][1]) << 32);
        vm[1 + a] = (uint64_t)__ballot_sync(SF_FULL, vb[a][0]) | ((uint64_t)__ballot_sync(SF_FULL, vb[a][1]) << 32);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        uint64_t ox[2], oz[2];
        int oe[2];
#pragma unroll
        for (int a = 0; a < 2; a++) {
            ox[a] = __shfl_xor_sync(SF_FULL, cx[a], off);
            oz[a] = __shfl_xor_sync(SF_FULL, cz[a], off);
            oe[a] = __shfl_xor_sync(SF_FULL, ce[a], off);
        }
#pragma unroll
        for (int a = 0; a < 2; a++) pmul1(cx[a], cz[a], ce[a], ox[a], oz[a], oe[a]);
    }
#pragma unroll
    for (int a = 0; a < 2; a++) {
        if (cx[a] != 0 || cz[a] != wz[1 + a]) bad = 1;
        epsq[1 + a] = (4 - ce[a]) & 3;
    }
    if (kind == 3) {
        // Z_c Z_t from the two one-qubit terms: Z^{w1} Z^{w2} = eps1 eps2 D^{u1} M^{v1} D^{u2} M^{v2};
        // moving M^{v1} past D^{u2} gives (-1)^{|v1 & u2|}, D^{u1} D^{u2} = D^{u1^u2} up to the
        // squares of the shared destabilizers (-1 for an odd i-power)
        const unsigned o0 = __ballot_sync(SF_FULL, lane < n && (r[0].de & 1u));
        const unsigned o1 = __ballot_sync(SF_FULL, lane + 32 < n && (r[1].de & 1u));
        const uint64_t odd = (uint64_t)o0 | ((uint64_t)o1 << 32);
        um[3] = um[1] ^ um[2];
        vm[3] = vm[1] ^ vm[2];
        epsq[3] = (epsq[1] + epsq[2] + 2 * (__popcll(vm[1] & um[2]) + __popcll(um[1] & um[2] & odd))) & 3;
    } else {  // one-qubit gate: terms 0 and 1 only
        um[2] = um[3] = vm[2] = vm[3] = 0;
        epsq[2] = epsq[3] = 0;
    }
    // groups by u in order of first appearance (group 0: the identity term)
    int gid[4], tpos[4], gnt[4] = {0, 0, 0, 0}, ng = 0;
    uint64_t gu[4] = {0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < 4; j++) {
        gid[j] = -1;
        tpos[j] = 0;
        if (j >= nt) continue;
        int found = -1;
#pragma unroll
        for (int j2 = 0; j2 < j; j2++)
            if (found < 0 && um[j2] == um[j]) found = gid[j2];
        if (found < 0) {
            found = ng;
#pragma unroll
            for (int g = 0; g < 4; g++)
                if (g == ng) gu[g] = um[j];
            ng++;
        }
        gid[j] = found;
#pragma unroll
        for (int g = 0; g < 4; g++)
            if (g == found) tpos[j] = gnt[g]++;
    }
    // P.xidx[g][g2] = the group whose u is u_g ^ u_g2 (lanes 0-15)
    {
        const int g = lane >> 2, g2 = lane & 3;
        uint64_t ug = 0, ug2 = 0;
#pragma unroll
        for (int x = 0; x < 4; x++) {
            if (x == g) ug = gu[x];
            if (x == g2) ug2 = gu[x];
        }
        bool miss = false;
        if (lane < 16 && g < ng && g2 < ng) {
            int m = -1;
#pragma unroll
            for (int g3 = 3; g3 >= 0; g3--)
                if (g3 < ng && (ug ^ ug2) == gu[g3]) m = g3;
            miss = m < 0;
            P.xidx[g][g2] = m < 0 ? 0 : m;
        }
        if (__any_sync(SF_FULL, miss)) bad = 1;
    }
    // term coefficients c_j i^{eps_j} (sign flips and swaps only)
    double2 ct[4];
#pragma unroll
    for (int j = 0; j < 4; j++) ct[j] = j < nt ? ipow_mul(cf[j], epsq[j]) : make_double2(0.0, 0.0);
    // table: lane 2q + comp takes component comp of the q-th half-table entry
    // (groups in order, 2^{nt_g - 1} entries each)
    {
        const int q = lane >> 1;
        const bool comp = lane & 1;
        int g = -1, pp = 0, base = 0, gn = 0;
#pragma unroll
        for (int x = 0; x < 4; x++) {
            const int sz = x < ng ? 1 << (gnt[x] - 1) : 0;
            if (g < 0 && q < base + sz) {
                g = x;
                pp = q - base;
                gn = gnt[x];
            }
            base += sz;
        }
        // the terms of group g in order, signed by pattern pp
        double val[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (gid[j] != g || g < 0) continue;
            const double x = comp ? ct[j].y : ct[j].x;
#pragma unroll
            for (int t = 0; t < 4; t++)
                if (t == tpos[j]) val[t] = dneg_if(x, (pp >> t) & 1);
        }
        int maxn = 0;
#pragma unroll
        for (int x = 0; x < 4; x++) maxn = gnt[x] > maxn ? gnt[x] : maxn;
        double acc = val[0];
        if (maxn > 1) acc += gn > 1 ? val[1] : 0.0;
        if (maxn > 2) acc += gn > 2 ? val[2] : 0.0;
        if (maxn > 3) acc += gn > 3 ? val[3] : 0.0;
        if (g >= 0) reinterpret_cast<double*>(&ctab[g][pp])[comp] = acc;
    }
    // the rest of P, one field per lane
    if (lane < 4) {
        P.nt[lane] = gnt[lane];
        P.fl[lane] = 0;
        P.u[lane] = gu[lane];
    } else if (lane < 20) {
        const int g = (lane - 4) >> 2, t = (lane - 4) & 3;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (gid[j] == g && tpos[j] == t) {
                P.v[g][t] = vm[j];
                P.c[g][t] = ct[j];
            }
    } else if (lane == 20) {
        P.ng = ng;
        P.bad = bad | (gu[0] != 0);
    }
}
}  // namespace sfw
