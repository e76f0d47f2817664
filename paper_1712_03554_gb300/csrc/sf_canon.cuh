// sf_canon.cuh -- the canonical amplitude convention of a frame element.
// An element (sigma, a) of a frame stands for g * a * D^sigma phi_0(M); the
// exported (canonical) amplitude refers instead to psi_can(M, sigma), whose
// amplitude at its anchor basis state b*(sigma) is 2^{-r/2}, real and positive
// (Sec. III, global phases of the states of a frame).  The two differ by the
// i-power that elem_amp_phi returns at the anchor.
#pragma once
#include "sf_device.cuh"

namespace {

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
        uint64_t wpv = 0;  // wv[pv >> 6] by masks: a run-time subscript would put wv in local memory
#pragma unroll
        for (int u = 0; u < W; u++) wpv |= wv[u] & (0ull - (uint64_t)(u == (pv >> 6)));
        if ((wpv >> (pv & 63)) & 1) {
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

}  // namespace
