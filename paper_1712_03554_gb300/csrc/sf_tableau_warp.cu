// sf_tableau_warp.cu -- the Clifford tableau kernel (ROTATE(F, U) on M and D,
// Invariant 1 repair, global-phase update; Sec. III, Table 2) for n <= 63,
// run by a single warp.  Lane L keeps tableau rows L and L + 32 in registers;
// the reduction (sfw::warp_rref) accepts clean leading columns with warp
// reductions, pivots are broadcast by shuffles, the destabilizer products of
// the dual row operations are warp butterflies, and one shared-memory
// permutation sorts the rows.  Same algorithm, and the same results bit for
// bit, as the block kernel of sf_tableau.cu.
#include "sf_warp.cuh"

namespace {
using namespace sfw;

__global__ void __launch_bounds__(32) k_clifford_warp(SfDev d, const sf_gate_rec* gates, int ng, int buf) {
    __shared__ Row stage[64];
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
    int ga = 0, gb = 0;  // the run's phase factor omega^ga sqrt(2)^gb
    for (int gi = 0; gi < ng; gi++) {
        const uint32_t ukind = gates[gi].kind, uq0 = gates[gi].q0, uq1 = gates[gi].q1;
        const bool two = ukind >= 6;
        if (ukind > 8 || uq0 >= (uint32_t)n || (two && (uq1 >= (uint32_t)n || uq1 == uq0))) {
            if (lane == 0) set_status(d.status, 1u, buf);  // SF_EINVAL: bad gate in a device list
            return;
        }
        const int kind = (int)ukind, q0 = (int)uq0, q1 = two ? (int)uq1 : 0;
        if (!warp_clifford_gate(r, n, rx, kind, q0, q1, stage, ga, gb)) {
            if (lane == 0) set_status(d.status, SF_ST_INTERNAL, buf, 8u);
            return;
        }
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
        *d.g = cmul(*d.g, cliff_factor(ga, gb));
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

// COFACTOR's tableau step for n <= 63 (Sec. III; the deterministic/random test
// of Z_q, the update of M and D, Invariant 1 repair, the five-step phase rule
// for both cofactors, and the tables of the old destabilizers in the new
// basis), run by one warp with the rows in registers: the same routine as the
// campaign engine, writing the same plan words and meta entries as the block
// kernel of sf_tableau.cu.
__global__ void __launch_bounds__(32) k_measure_prep_warp(SfDev d, uint32_t q, int buf) {
    __shared__ Row stage[64];
    __shared__ CofTab C;
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
    const int rx = warp_measure_prep(r, n, d.meta[0], (int)q, C, stage);
    __syncwarp();
    if (!C.random) {
        if (lane == 0) {
            d.meta[1] = C.rq;
            d.meta[2] = 0;
            if (C.bad) set_status(d.status, SF_ST_INTERNAL, buf, 3u);
        }
        return;
    }
    if (C.bad) {
        if (lane == 0) set_status(d.status, SF_ST_INTERNAL, buf, 5u);
        return;
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
            d.plan[cf_u(n, 1) + row] = C.u[row];
            d.plan[cf_v(n, 1) + row] = C.v[row];
        }
    }
    if (lane == 0) {
        uint64_t* pl = d.plan;
        pl[cf_eps(n, 1)] = C.eps0;
        pl[cf_eps(n, 1) + 1] = C.eps1;
        const size_t ko = cf_kappa(n, 1);
        pl[ko + 0] = (uint64_t)__double_as_longlong(C.kap[0].x);
        pl[ko + 1] = (uint64_t)__double_as_longlong(C.kap[0].y);
        pl[ko + 2] = (uint64_t)__double_as_longlong(C.kap[1].x);
        pl[ko + 3] = (uint64_t)__double_as_longlong(C.kap[1].y);
        pl[cf_uq(n, 1)] = C.uq;
        pl[cf_vq(n, 1)] = C.vq;
        pl[cf_tau(n, 1)] = C.tau0;
        pl[cf_tau(n, 1) + 1] = C.tau1;
        d.meta[0] = rx;
        d.meta[1] = C.rq;
        d.meta[2] = 1;
    }
}

}  // namespace

void sf_launch_measure_prep_warp(const SfDev& d, uint32_t q, int buf, cudaStream_t s) {
    k_measure_prep_warp<<<1, 32, 0, s>>>(d, q, buf);
}

void sf_launch_clifford_warp(const SfDev& d, const void* dev_gates, int ngates, int buf, cudaStream_t s) {
    k_clifford_warp<<<1, 32, 0, s>>>(d, reinterpret_cast<const sf_gate_rec*>(dev_gates), ngates, buf);
}
