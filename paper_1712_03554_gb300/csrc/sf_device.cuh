// sf_device.cuh -- device-side data layout and Pauli arithmetic shared by the
// libsf translation units (tableau kernels, frame kernels, host API).
//
// Representation used on the device (differs from the export convention, see
// the frame export kernel):
//   * M: the canonical RREF tableau (Invariant 1), unsigned rows, word-major
//     [W][n] planes mx, mz.
//   * D: one destabilizer row per stabilizer row (D_h anticommutes with M_h
//     only; the D rows commute with each other), signed: D_h = i^{de_h} P(dx, dz)
//     with de_h in {0, 2}.
//   * phi_0(M): the state stabilized by +M_h for every h, with <0|phi_0> =
//     2^{-r/2} real positive (0 lies in its support because M is in RREF).
//   * frame element (sigma, a) stands for a * g * D^sigma phi_0(M), where g is
//     one global phase kept on the device.  D^sigma phi_0 is stabilized by M
//     with signs sigma, i.e. it is the paper's state M^sigma (Def. 1) up to a
//     phase that the export kernel removes.
// Pauli P(x, z) = prod_q i^{x_q z_q} X^{x_q} Z^{z_q} (so x = z = 1 is Y).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define SF_MAX_W 16
#define SF_MAX_N 1024
#define SF_FULL 0xffffffffu

// status word: low byte = sf_status code, bits 8..15 = frame buffer that was
// current when the error happened (so the host can restore it).
#define SF_ST_CODE(s) ((s) & 0xffu)
#define SF_ST_CAPACITY 3u
#define SF_ST_TIMEOUT 5u
#define SF_ST_STATE 6u
#define SF_ST_INTERNAL 7u

struct sf_gate_rec { uint32_t kind, q0, q1, pad; };

struct SfDev {
    int n;          // qubits
    int W;          // words per row / phase vector (power of two >= ceil(n/64))
    int NT;         // threads of the single-CTA tableau kernels (multiple of 32, >= n)
    int nblk;       // CTAs of the per-element kernels
    uint64_t cap;   // max_elems
    // tableau, word-major [W][n]
    uint64_t *mx, *mz, *dx, *dz;
    uint32_t* de;   // [n] phase exponent of D rows (0 or 2)
    int32_t* piv;   // [n] pivot column (c < n: x_c, else z_{c-n})
    int32_t* meta;  // [0] = r (X-block size), [1] = deterministic-measure row, [2] = random flag
    double2* g;     // global phase
    // frame, double buffered; sig is word-major [W][cap]
    uint64_t* sig[2];
    double2* amp[2];
    unsigned long long* kcnt;  // [2] element counts of the two buffers
    uint32_t* status;
    // plan (written by a single-CTA prep kernel, read by the per-element kernels)
    uint64_t* plan;
    // slot table used by coalescing (children are hashed into it, amplitudes
    // accumulate there, the compaction pass empties it again)
    uint32_t* tstate;          // [tcap] 0 empty, 1 being written, 2 ready (W > 1 only)
    uint64_t* tkey;            // [W][tcap] phase vector of the slot (W = 1: all ones = empty)
    double2* tacc;             // [tcap] accumulated amplitude
    unsigned long long tcap;   // power of two >= 2 cap
    unsigned long long* tsize; // slots in use by the current merge
    double* red;               // [4 * nblk] reduction partials
    double* out;               // [8] small results (p0, p1, amplitude re, im)
};

// An empty slot key: phase vectors never set bit 63 of their last word
// (the word count W leaves at least one spare bit above qubit n-1).
#define SF_EMPTY_KEY 0xffffffffffffffffull

// ---- plan layout (in 64-bit words) ---------------------------------------
// affine map of a Clifford batch: sigma'_h = parity(A_h & sigma) ^ t_h
// A is stored by columns: column j (the image of e_j) at [j*W, j*W+W).
__host__ __device__ inline size_t plan_AT(int n, int W) { return 0; }
__host__ __device__ inline size_t plan_t(int n, int W) { return (size_t)n * W; }
// at most four Z-type Pauli terms per diagonal gate, grouped by anticommutation mask
#define SF_BR_MAXG 4
#define SF_BR_MAXT 4
// cofactor plan
__host__ __device__ inline size_t plan_cf(int n, int W) { return (size_t)n * W + W; }
// cofactor: u'[n][W], v'[n][W], eps i-powers as two bit planes [2][W], kappa[4] doubles, tau0[W], tau1[W], v[W]
__host__ __device__ inline size_t cf_u(int n, int W) { return plan_cf(n, W); }
__host__ __device__ inline size_t cf_v(int n, int W) { return cf_u(n, W) + (size_t)n * W; }
__host__ __device__ inline size_t cf_eps(int n, int W) { return cf_v(n, W) + (size_t)n * W; }
__host__ __device__ inline size_t cf_kappa(int n, int W) { return cf_eps(n, W) + 2 * W; }
__host__ __device__ inline size_t cf_tau(int n, int W) { return cf_kappa(n, W) + 4; }
__host__ __device__ inline size_t cf_vq(int n, int W) { return cf_tau(n, W) + 2 * W; }
// amplitude-query plan: y[W], zmask[W], zexp[W], flag
__host__ __device__ inline size_t plan_am(int n, int W) { return cf_vq(n, W) + W; }
__host__ __device__ inline size_t plan_words(int n, int W) { return plan_am(n, W) + 3 * W + 8; }

// ---- Pauli arithmetic -------------------------------------------------------
template <int W>
struct Pauli {
    uint64_t x[W], z[W];
    int e;  // i^e P(x, z)
};

template <int W>
__device__ __forceinline__ void pauli_id(Pauli<W>& p) {
#pragma unroll
    for (int w = 0; w < W; w++) { p.x[w] = 0; p.z[w] = 0; }
    p.e = 0;
}

// i-power of P(x1,z1) P(x2,z2) relative to P(x1^x2, z1^z2): per qubit
// (ab + cd + 2bc - (a^c)(b^d)) mod 4 for P1 = (a,b), P2 = (c,d).
template <int W>
__device__ __forceinline__ int pauli_lambda(const uint64_t* x1, const uint64_t* z1, const uint64_t* x2,
                                            const uint64_t* z2) {
    int s = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        s += __popcll(x1[w] & z1[w]) + __popcll(x2[w] & z2[w]) + 2 * __popcll(z1[w] & x2[w]) -
             __popcll((x1[w] ^ x2[w]) & (z1[w] ^ z2[w]));
    }
    return s & 3;
}

// a <- a * b
template <int W>
__device__ __forceinline__ void pauli_mul(Pauli<W>& a, const Pauli<W>& b) {
    int l = pauli_lambda<W>(a.x, a.z, b.x, b.z);
#pragma unroll
    for (int w = 0; w < W; w++) { a.x[w] ^= b.x[w]; a.z[w] ^= b.z[w]; }
    a.e = (a.e + b.e + l) & 3;
}

template <int W>
__device__ __forceinline__ int popc_and(const uint64_t* a, const uint64_t* b) {
    int s = 0;
#pragma unroll
    for (int w = 0; w < W; w++) s += __popcll(a[w] & b[w]);
    return s;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 ipow_mul(double2 a, int k) {  // a * i^k
    switch (k & 3) {
        case 0: return a;
        case 1: return make_double2(-a.y, a.x);
        case 2: return make_double2(-a.x, -a.y);
        default: return make_double2(a.y, -a.x);
    }
}

// code | buffer << 8 | site << 16 (site identifies the failing check)
__device__ __forceinline__ void set_status(uint32_t* st, uint32_t code, int buf, uint32_t site = 0) {
    atomicCAS(st, 0u, code | ((uint32_t)buf << 8) | (site << 16));
}

// ---- launch wrappers implemented in the .cu files (one kernel each) --------
void sf_launch_reset(const SfDev& d, int buf, cudaStream_t s);
void sf_launch_clifford(const SfDev& d, const void* dev_gates, int ngates, int buf, uint64_t* gws,
                        cudaStream_t s);
void sf_launch_measure_prep(const SfDev& d, uint32_t q, int buf, uint64_t* gws, cudaStream_t s);
void sf_launch_amp_prep(const SfDev& d, const uint64_t* dev_y, cudaStream_t s);
size_t sf_tableau_smem_bytes(int n, int W, int NT);

void sf_launch_affine(const SfDev& d, int buf, cudaStream_t s);
// children of a diagonal gate written out unmerged (in -> out)
void sf_launch_branch(const SfDev& d, uint32_t kind, uint32_t q0, uint32_t q1, double theta, int in_buf,
                      int out_buf, cudaStream_t s);
// children hashed into the slot table: diagonal gate (kind < 4), plain
// coalescing of a frame (kind = SF_INSERT_FRAME) or cofactor split (kind = SF_INSERT_COFACTOR)
#define SF_INSERT_FRAME 16u
#define SF_INSERT_COFACTOR 17u
void sf_launch_insert(const SfDev& d, uint32_t kind, uint32_t q0, uint32_t q1, double theta, int in_buf,
                      int out_buf, cudaStream_t s);
void sf_launch_compact(const SfDev& d, double eps, int out_buf, cudaStream_t s);
void sf_launch_filter(const SfDev& d, int x, int in_buf, int out_buf, cudaStream_t s);
void sf_launch_prob(const SfDev& d, int buf, cudaStream_t s);
void sf_launch_reduce_final(const SfDev& d, int what, cudaStream_t s);
void sf_launch_amplitude(const SfDev& d, int buf, cudaStream_t s);
void sf_launch_export(const SfDev& d, int buf, int stage_buf, cudaStream_t s);
size_t sf_affine_smem_bytes(int n, int W);
