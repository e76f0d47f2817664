// sf_tableau_warp.cu -- the Clifford tableau kernel (ROTATE(F, U) on M and D,
// Invariant 1 repair, global-phase update; Sec. III, Table 2) for n <= 63,
// run by a single warp.  Lane L keeps tableau rows L and L + 32 in registers;
// the pivot search is two ballots, row swaps and the pivot broadcast are
// shuffles, and the destabilizer products of the dual row operations are warp
// butterflies -- no shared memory and no block barrier.  Same results, bit for
// bit, as the block kernel of sf_tableau.cu.
#include "sf_device.cuh"

namespace {

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
__device__ int warp_amp_phi(const Row* r, int n, int rx, bool use_tau, uint64_t y) {
    const int lane = threadIdx.x & 31;
    uint64_t qx = 0, qz = 0;
    int qe = 0;
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        if (use_tau && row < n && r[hf].t1) pmul1(qx, qz, qe, r[hf].dx, r[hf].dz, (int)r[hf].de);
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

// Gauss-Jordan from column `start` (rows with pivot < start keep theirs), with
// the dual destabilizer updates and the affine-map / sign-vector tracking of
// the block version.  Returns r.
__device__ int warp_gj(Row* r, int n, int start) {
    const int lane = threadIdx.x & 31;
    int nxt = __popc(__ballot_sync(SF_FULL, lane < n && r[0].piv < start)) +
              __popc(__ballot_sync(SF_FULL, lane + 32 < n && r[1].piv < start));
    for (int c = start; c < 2 * n && nxt < n; c++) {
        const unsigned a0 = __ballot_sync(SF_FULL, lane < n && colbit(r[0], c, n));
        const unsigned a1 = __ballot_sync(SF_FULL, lane + 32 < n && colbit(r[1], c, n));
        const uint64_t all = (uint64_t)a0 | ((uint64_t)a1 << 32);
        const uint64_t mask = all & (~0ull << nxt);  // candidate rows: not yet pivots
        if (!mask) continue;
        const int p = __ffsll((long long)mask) - 1;
        if (p == nxt && all == (1ull << nxt)) {  // already reduced: the row keeps its pivot
            if (lane == (nxt & 31)) r[nxt >> 5].piv = c;
            nxt++;
            continue;
        }
        if (p != nxt) {
            const Row rp = fetch_row(r, p), rn = fetch_row(r, nxt);
            if (lane == (p & 31)) r[p >> 5] = rn;
            if (lane == (nxt & 31)) r[nxt >> 5] = rp;
        }
        const Row pv = fetch_row(r, nxt);
        uint64_t dx = 0, dz = 0;
        int de = 0;
        bool any = false;
        for (int hf = 0; hf < 2; hf++) {
            const int row = lane + 32 * hf;
            if (row < n && row != nxt && colbit(r[hf], c, n)) {
                const uint32_t cb = (uint32_t)(lam1(r[hf].mx, r[hf].mz, pv.mx, pv.mz) >> 1) & 1u;
                r[hf].mx ^= pv.mx;
                r[hf].mz ^= pv.mz;
                r[hf].A ^= pv.A;
                r[hf].t0 ^= pv.t0 ^ cb;
                r[hf].t1 ^= pv.t1 ^ cb;
                pmul1(dx, dz, de, r[hf].dx, r[hf].dz, (int)r[hf].de);
                any = true;
            }
        }
        if (__any_sync(SF_FULL, any)) {
            warp_prod(dx, dz, de);
            if (lane == (nxt & 31)) {
                Row& t = r[nxt >> 5];
                uint64_t x = t.dx, z = t.dz;
                int e = (int)t.de;
                pmul1(x, z, e, dx, dz, de);
                t.dx = x;
                t.dz = z;
                t.de = (uint32_t)e;
            }
        }
        if (lane == (nxt & 31)) r[nxt >> 5].piv = c;
        nxt++;
    }
    return __popc(__ballot_sync(SF_FULL, lane < n && r[0].piv < n)) +
           __popc(__ballot_sync(SF_FULL, lane + 32 < n && r[1].piv < n));
}

__global__ void __launch_bounds__(32) k_clifford_warp(SfDev d, const sf_gate_rec* gates, int ng, int buf) {
    if (*d.status) return;
    const int n = d.n, lane = threadIdx.x;
    Row r[2];
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        const bool in = row < n;
        r[hf].mx = in ? d.mx[row] : 0;
        r[hf].mz = in ? d.mz[row] : 0;
        r[hf].dx = in ? d.dx[row] : 0;
        r[hf].dz = in ? d.dz[row] : 0;
        r[hf].de = in ? d.de[row] : 0;
        r[hf].piv = in ? d.piv[row] : 0x7fffffff;
        r[hf].A = in ? (1ull << row) : 0;
        r[hf].t0 = 0;
        r[hf].t1 = 0;
    }
    int rx = d.meta[0];
    double2 g = *d.g;
    const double rs2 = 0.70710678118654752440;
    for (int gi = 0; gi < ng; gi++) {
        const uint32_t ukind = gates[gi].kind, uq0 = gates[gi].q0, uq1 = gates[gi].q1;
        const bool two = ukind >= 6;
        if (ukind > 8 || uq0 >= (uint32_t)n || (two && (uq1 >= (uint32_t)n || uq1 == uq0))) {
            if (lane == 0) set_status(d.status, 1u, buf);  // SF_EINVAL: bad gate in a device list
            return;
        }
        const int kind = (int)ukind, q0 = (int)uq0, q1 = two ? (int)uq1 : 0;
        // numerator of the phase rule (see the block kernel)
        int yq = -1;
        double2 num = make_double2(1.0, 0.0);
        if (kind == 0) {
            const int cq = warp_amp_phi(r, n, rx, false, 1ull << q0);
            if (cq != 2) {
                const double2 cv = cq < 0 ? make_double2(0.0, 0.0) : ipow_mul(make_double2(1.0, 0.0), cq);
                num = make_double2((1.0 + cv.x) * rs2, cv.y * rs2);
            } else {
                yq = q0;
                num = make_double2(2.0 * rs2, 0.0);
            }
        } else if (kind == 3) {
            yq = q0;
        } else if (kind == 4) {
            yq = q0;
            num = make_double2(0.0, 1.0);
        }
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
        rx = warp_gj(r, n, two ? min(q0, q1) : q0);
        const int dq = warp_amp_phi(r, n, rx, true, yq >= 0 ? (1ull << yq) : 0ull);
        if (dq < 0) {
            if (lane == 0) set_status(d.status, SF_ST_INTERNAL, buf, 8u);
            return;
        }
        double2 om = ipow_mul(num, (4 - dq) & 3);
        const int dr = rx - r_old;
        const double sc = dr == 0 ? 1.0 : (dr > 0 ? 1.41421356237309504880 : rs2);
        om.x *= sc;
        om.y *= sc;
        g = cmul(g, om);
    }
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        if (row < n) {
            d.mx[row] = r[hf].mx;
            d.mz[row] = r[hf].mz;
            d.dx[row] = r[hf].dx;
            d.dz[row] = r[hf].dz;
            d.de[row] = r[hf].de;
            d.piv[row] = r[hf].piv;
        }
    }
    if (lane == 0) {
        d.meta[0] = rx;
        *d.g = g;
    }
    // affine map: column j of A (image of e_j) and the sign word t
    uint64_t* AT = d.plan + plan_AT(n, 1);
    for (int j = 0; j < n; j++) {
        const unsigned b0 = __ballot_sync(SF_FULL, lane < n && ((r[0].A >> j) & 1));
        const unsigned b1 = __ballot_sync(SF_FULL, lane + 32 < n && ((r[1].A >> j) & 1));
        if (lane == 0) AT[j] = (uint64_t)b0 | ((uint64_t)b1 << 32);
    }
    const unsigned t0 = __ballot_sync(SF_FULL, lane < n && r[0].t0);
    const unsigned t1 = __ballot_sync(SF_FULL, lane + 32 < n && r[1].t0);
    if (lane == 0) d.plan[plan_t(n, 1)] = (uint64_t)t0 | ((uint64_t)t1 << 32);
}

}  // namespace

void sf_launch_clifford_warp(const SfDev& d, const void* dev_gates, int ngates, int buf, cudaStream_t s) {
    k_clifford_warp<<<1, 32, 0, s>>>(d, reinterpret_cast<const sf_gate_rec*>(dev_gates), ngates, buf);
}
