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

#include <cmath>

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
    uint64_t* tkey;            // [tcap][W] phase vector of the slot (W = 1: all ones = empty)
    double2* tacc;             // [tcap] accumulated amplitude
    unsigned long long tcap;   // power of two >= 2 cap
    unsigned long long* tsize; // slots in use by the current merge
    double* red;               // [4 * nblk] reduction partials
    double* out;               // [8] small results (p0, p1, amplitude re, im)
    // index of each frame buffer: phase vector -> position.  Slots carry the
    // generation tag of the index that wrote them, so an index is replaced by
    // bumping the tag, never by clearing the table.
    // slot s of buffer b's index is the slot_words(W) words islot[b][s * slot_words(W) ..]:
    // word 0 = tag << 32 | position, then the phase vector (word 1 for W = 1,
    // words 2 .. W + 1 otherwise, 16-byte aligned for 128-bit accesses)
    uint64_t* islot[2];
    unsigned long long icap;   // power of two >= 2 cap
    uint32_t* itag;            // [2] tag of the valid index of each buffer (0 = none)
    unsigned long long* isize; // [2] slots used by that index (power of two)
    unsigned int* done;        // CTAs finished (last-CTA publication of tags and counts)
    unsigned long long* ipend; // index size chosen by CTA 0, published by the last CTA
    unsigned long long* ocnt;  // output counter of the merge kernels
    uint64_t* gp;              // workspace of the grid program (n <= 63 only)
    int lowrank;               // 1: low-rank forms of the affine and cofactor maps (W >= 8)
};

// What the grid program leaves known about the layout of its frame (the first
// member of its workspace d.gp): after a launch that started from one element
// and whose branches all doubled the frame in place, the element at position
// j is s_0 ^ (XOR of u[i] over the set bits i of j), n = log2(frame size).
// ok = 0: nothing known.  Valid until a kernel moves or changes the elements
// (the host tracks that and passes its verdict to the kernels that use it).
struct GpLayout {
    unsigned ok, n;
    uint64_t u[64];
};

// one program record (the layout of sf_op): kind, qubits, conditional-gate
// kind or parameter bits
struct OpRec {
    uint32_t kind, q0, q1, arg;
    double param;
};

// Whether the merging kernels (branch merge, cofactor merge, collapse,
// compaction) leave an index of their output.  Below 8 words a slot is at most
// 72 bytes and the index of the next merge is usually wanted; from 8 words on
// a slot write is a random 72..136-byte access per element, and the per-op
// path nearly always changes every phase vector (a Clifford batch) before the
// next merge, so the index is built only when a merge needs it.
__host__ __device__ constexpr bool sf_emit_index(int W) { return W < 8; }

// words per index slot and where its key starts (see SfDev::islot)
__host__ __device__ constexpr int slot_words(int W) { return W == 1 ? 2 : W + 2; }
__host__ __device__ constexpr int slot_key(int W) { return W == 1 ? 1 : 2; }

// An empty one-word slot key: with W = 1 (n <= 63) phase vectors never set
// bit 63.  Wider keys mark their slots through a separate state word.
#define SF_EMPTY_KEY 0xffffffffffffffffull

// ---- plan layout (in 64-bit words) ---------------------------------------
// affine map of a Clifford batch: sigma'_h = parity(A_h & sigma) ^ t_h
// A is stored by columns: column j (the image of e_j) at [j*W, j*W+W).
__host__ __device__ inline size_t plan_AT(int n, int W) { return 0; }
__host__ __device__ inline size_t plan_t(int n, int W) { return (size_t)n * W; }
// at most four Z-type Pauli terms per diagonal gate, grouped by anticommutation mask
#define SF_BR_MAXG 4
#define SF_BR_MAXT 4

// v[m] for m in [0, SF_BR_MAXG) by masks: a run-time subscript into a small
// per-thread array puts the array in local memory
template <typename T>
__device__ __forceinline__ T pick_grp(const T* v, int m) {
    T r = 0;
#pragma unroll
    for (int g = 0; g < SF_BR_MAXG; g++) r |= v[g] & (T)(0 - (T)(g == m));
    return r;
}
// cofactor plan
__host__ __device__ inline size_t plan_cf(int n, int W) { return (size_t)n * W + W; }
// cofactor: u'[n][W], v'[n][W], eps i-powers as two bit planes [2][W], kappa[4] doubles, tau0[W], tau1[W], v[W]
__host__ __device__ inline size_t cf_u(int n, int W) { return plan_cf(n, W); }
__host__ __device__ inline size_t cf_v(int n, int W) { return cf_u(n, W) + (size_t)n * W; }
__host__ __device__ inline size_t cf_eps(int n, int W) { return cf_v(n, W) + (size_t)n * W; }
__host__ __device__ inline size_t cf_kappa(int n, int W) { return cf_eps(n, W) + 2 * W; }
__host__ __device__ inline size_t cf_tau(int n, int W) { return cf_kappa(n, W) + 4; }
__host__ __device__ inline size_t cf_vq(int n, int W) { return cf_tau(n, W) + 2 * W; }
// rows of the old tableau anticommuting with Z_q: elements sigma and sigma ^ uq share their cofactors
__host__ __device__ inline size_t cf_uq(int n, int W) { return cf_vq(n, W) + W; }
// amplitude-query plan: y[W], zmask[W], zexp[W], flag
__host__ __device__ inline size_t plan_am(int n, int W) { return cf_uq(n, W) + W; }
// Low-rank factors of a GF(2) map given by n vectors R_h of W words (W >= 8).
// Delta_h = R_h ^ e_h for maps near the identity (the affine map of a Clifford
// gate, the cofactor's old-to-new destabilizer map U) or Delta_h = R_h (the
// cofactor's V) is written Delta_h = sum_i C[h][i] B_i over a basis
// B_0..B_{r-1}.  Block: [0] = r, or SF_LR_NONE when r > SF_LR_MAX; then
// B[SF_LR_MAX][W]; then c[SF_LR_MAX][W], c_i = (C[h][i])_h as an n-bit vector.
// (With the row sort's permutation rho split off first: see the move list.)
#define SF_LR_MAX 16
#define SF_LR_NONE 0xffffffffull
__host__ __device__ inline size_t lr_words(int W) { return 2 + 2 * (size_t)SF_LR_MAX * W; }
__host__ __device__ inline size_t lr_B(int W) { return 2; }
__host__ __device__ inline size_t lr_C(int W) { return 2 + (size_t)SF_LR_MAX * W; }
// the Clifford batch's map: factors of A ^ I (columns of A)
__host__ __device__ inline size_t plan_lr_aff(int n, int W) { return plan_am(n, W) + 3 * W + 8; }
// the cofactor's maps: factors of U ^ I and of V, then K_j[SF_LR_MAX][W] and
// omega_y[2][W] of the closed-form i-power (k_cof_lowrank)
__host__ __device__ inline size_t plan_lr_u(int n, int W) { return plan_lr_aff(n, W) + lr_words(W); }
__host__ __device__ inline size_t plan_lr_v(int n, int W) { return plan_lr_u(n, W) + lr_words(W); }
__host__ __device__ inline size_t plan_cf_k(int n, int W) { return plan_lr_v(n, W) + lr_words(W); }
__host__ __device__ inline size_t plan_cf_om(int n, int W) { return plan_cf_k(n, W) + (size_t)SF_LR_MAX * W; }
// The row sort that ends a Clifford batch or a measurement (Invariant 1)
// moves the rows whose pivot changed; the others keep their relative order.
// As a map of phase-vector bits: delete the bits at the old positions a_k
// (ascending), then insert them at the new positions e_j (ascending), e_j
// taking the bit of a_{src_j}; isrc is the inverse index.  Block: [0] = m, or
// SF_LR_NONE when more than SF_MV_MAX rows moved; a[SF_MV_MAX], e[SF_MV_MAX],
// src[SF_MV_MAX], isrc[SF_MV_MAX].  rho: the new position of every row, as
// n 32-bit words.  The low-rank factors above are taken of Delta_h = R_h ^
// e_{rho(h)}, i.e. after this permutation.
#define SF_MV_MAX 8
__host__ __device__ inline size_t mv_words() { return 1 + 4 * SF_MV_MAX; }
__host__ __device__ inline size_t plan_mv_aff(int n, int W) { return plan_cf_om(n, W) + 2 * W; }
__host__ __device__ inline size_t plan_mv_cf(int n, int W) { return plan_mv_aff(n, W) + mv_words(); }
__host__ __device__ inline size_t plan_rho_aff(int n, int W) { return plan_mv_cf(n, W) + mv_words(); }
__host__ __device__ inline size_t plan_rho_cf(int n, int W) { return plan_rho_aff(n, W) + (size_t)(n + 1) / 2; }
// plan of a diagonal gate written by the one-CTA planning kernel (W >= 8),
// 16-byte aligned
#define SF_BR_WORDS(W) (8 + 20 * (W) + 32)
__host__ __device__ inline size_t plan_br(int n, int W) {
    return (plan_rho_cf(n, W) + (size_t)(n + 1) / 2 + 1) & ~(size_t)1;
}
// the old destabilizers of a measurement, kept for the cofactor tables
// (W >= 2): x planes [W][n], z planes [W][n], phase exponents [n]
__host__ __device__ inline size_t plan_d0(int n, int W) { return plan_br(n, W) + SF_BR_WORDS(W); }
__host__ __device__ inline size_t plan_words(int n, int W) { return plan_d0(n, W) + (size_t)(2 * W + 1) * n; }

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

// product of the 32 lanes' Paulis, in every lane (for factors that commute
// with one another, where the order does not matter)
template <int W>
__device__ __forceinline__ void warp_pauli_product(Pauli<W>& p) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        Pauli<W> o;
#pragma unroll
        for (int w = 0; w < W; w++) {
            o.x[w] = __shfl_xor_sync(SF_FULL, p.x[w], off);
            o.z[w] = __shfl_xor_sync(SF_FULL, p.z[w], off);
        }
        o.e = __shfl_xor_sync(SF_FULL, p.e, off);
        pauli_mul<W>(p, o);
    }
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
// sign flip on the integer pipe: the high word goes through registers by
// explicit moves, so the flip is not turned back into an FP64 negation (an
// FP64 instruction occupies the SM's narrow FP64 pipe)
__device__ __forceinline__ double dneg_if(double x, bool neg) {
    unsigned lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
    hi ^= (unsigned)neg << 31;
    double r;
    asm("mov.b64 %0, {%1, %2};" : "=d"(r) : "r"(lo), "r"(hi));
    return r;
}
__device__ __forceinline__ double2 ipow_mul(double2 a, int k) {  // a * i^k
    switch (k & 3) {
        case 0: return a;
        case 1: return make_double2(dneg_if(a.y, true), a.x);
        case 2: return make_double2(dneg_if(a.x, true), dneg_if(a.y, true));
        default: return make_double2(a.y, dneg_if(a.x, true));
    }
}

// Terms of diagonal gate kind as sum_j c_j Z^{w_j} (Sec. IV), from
// e^{i theta} = cs + i sn (T, T-dagger: theta = +-pi/4).  Kinds 0-2:
// P(theta) = (1 + e^{i theta})/2 I + (1 - e^{i theta})/2 Z_q0, terms I, Z_q0.
// Kind 3: CR(theta) = I + (e^{i theta} - 1)(I - Z_c - Z_t + Z_c Z_t)/4, terms
// I, Z_c, Z_t, Z_c Z_t.
struct SfTerms {
    double2 c[4];
};
__host__ __device__ inline SfTerms diag_terms(uint32_t kind, double cs, double sn) {
    SfTerms T;
    if (kind <= 2) {
        T.c[0] = make_double2((1.0 + cs) * 0.5, sn * 0.5);
        T.c[1] = make_double2((1.0 - cs) * 0.5, -sn * 0.5);
        T.c[2] = T.c[3] = make_double2(0.0, 0.0);
    } else {
        const double2 dd = make_double2((cs - 1.0) * 0.25, sn * 0.25);
        T.c[0] = make_double2(1.0 + dd.x, dd.y);
        T.c[1] = T.c[2] = make_double2(-dd.x, -dd.y);
        T.c[3] = dd;
    }
    return T;
}
// computed once on the host for a launch from the host: the double-precision
// pipe of an SM is narrow, and every CTA would otherwise evaluate them
inline SfTerms diag_terms_host(uint32_t kind, double theta) {
    const double th = kind == 0 ? 0.78539816339744830962 : (kind == 1 ? -0.78539816339744830962 : theta);
    return diag_terms(kind, std::cos(th), std::sin(th));
}

// Double-precision work runs on a narrow pipe, so the per-element kernels keep
// it to the multiply-adds of the amplitudes.
// coefficient sum_t (-1)^{bit t of p} c_t of a group of nt diagonal-gate
// terms, added in the order t = 0, 1, ... (the per-element sum of the terms
// for the sign pattern p)
__device__ __forceinline__ double2 coef_pattern(const double2* c, int nt, int p) {
    double2 cf = make_double2(dneg_if(c[0].x, p & 1), dneg_if(c[0].y, p & 1));
    for (int t = 1; t < nt; t++) {
        const bool ng = (p >> t) & 1;
        cf.x += dneg_if(c[t].x, ng);
        cf.y += dneg_if(c[t].y, ng);
    }
    return cf;
}
// acc += c * a
__device__ __forceinline__ void cmul_acc(double2& acc, double2 c, double2 a) {
    acc.x = fma(c.x, a.x, acc.x);
    acc.x = fma(-c.y, a.y, acc.x);
    acc.y = fma(c.x, a.y, acc.y);
    acc.y = fma(c.y, a.x, acc.y);
}
// drop rule |a|^2 >= eps2: keep_bits is a power of two no smaller than
// sqrt(eps2) (from the exponent of eps2), so an amplitude whose larger
// component reaches it is kept on integer compares alone (rounding is monotone)
__device__ __forceinline__ unsigned long long keep_bits(double eps2) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(eps2);
    if (b == 0) return 0;
    const int e = (int)(b >> 52) - 1023;  // eps2 < 2^{e+1}
    return (unsigned long long)(((e + 2) >> 1) + 1023) << 52;
}
__device__ __forceinline__ bool amp_kept(double2 a, unsigned long long kb, double eps2) {
    const unsigned long long bx = (unsigned long long)__double_as_longlong(a.x) & 0x7fffffffffffffffull;
    const unsigned long long by = (unsigned long long)__double_as_longlong(a.y) & 0x7fffffffffffffffull;
    if ((bx > by ? bx : by) >= kb) return true;
    return a.x * a.x + a.y * a.y >= eps2;
}

// Every Clifford gate multiplies the global factor by omega^a sqrt(2)^b
// (omega = e^{i pi/4}, a mod 8, b an integer): a run of gates keeps the two
// exponents in integers and touches the double-precision factor once.
// Numerator of the phase rule of gate kind as omega^a sqrt(2)^b; cq is the
// i-power of the Hadamard numerator (2: the Y-point form, negative: zero).
__device__ __forceinline__ void cliff_num_exp(int kind, int cq, int& a, int& b) {
    a = 0;
    b = 0;
    if (kind == 0) {
        if (cq == 0 || cq == 2) b = 1;  // 2 / sqrt(2)
        else if (cq < 0) b = -1;        // 1 / sqrt(2)
        else a = cq == 1 ? 1 : 7;       // (1 + i) / sqrt(2), (1 - i) / sqrt(2)
    } else if (kind == 4) {
        a = 2;  // i
    }
}
__device__ __forceinline__ double2 cliff_factor(int a, int b) {
    double m = ldexp(1.0, b >> 1);
    if (b & 1) m *= 1.41421356237309504880;
    const double h = m * 0.70710678118654752440;
    return ipow_mul((a & 1) ? make_double2(h, h) : make_double2(m, 0.0), (a >> 1) & 3);
}

// code | buffer << 8 | site << 16 (site identifies the failing check)
__device__ __forceinline__ void set_status(uint32_t* st, uint32_t code, int buf, uint32_t site = 0) {
    atomicCAS(st, 0u, code | ((uint32_t)buf << 8) | (site << 16));
}

// ---- frame index ---------------------------------------------------------------
__device__ __forceinline__ uint32_t next_tag(uint32_t t) { return (t % 0x7ffffffeu) + 1u; }

// slots of an index for k keys: load factor at most 1/4 (1/2 for frames above
// half the capacity), which keeps the longest linear-probe chain of a pass --
// every probe a dependent L2 round trip -- short
__host__ __device__ inline unsigned long long index_slots(unsigned long long k, unsigned long long icap) {
    unsigned long long t = 64;
    while (t < 4 * k && t < icap) t <<= 1;
    return t < icap ? t : icap;
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

// Insert a key that is distinct from every other key of this generation
// (phase vectors of a frame are distinct, Def. 1): one 64-bit compare-and-swap
// claims the slot and publishes the position, the key goes beside it in the
// same sector.  Returns false only if the table is full.
template <int W>
__device__ __forceinline__ bool index_insert(const SfDev& d, int b, unsigned long long T, uint32_t tag,
                                             const uint64_t* key, uint32_t pos) {
    unsigned long long* sl = reinterpret_cast<unsigned long long*>(d.islot[b]);
    const unsigned long long mine = ((unsigned long long)tag << 32) | pos;
    unsigned long long slot = hash_sig<W>(key) & (T - 1);
    for (unsigned long long probe = 0; probe < T; probe++) {
        unsigned long long* tv = sl + slot * slot_words(W);
        unsigned long long cur = *(volatile unsigned long long*)tv;
        while ((uint32_t)(cur >> 32) != tag) {
            const unsigned long long old = atomicCAS(tv, cur, mine);
            if (old == cur) {
                if constexpr (W == 1) {
                    tv[1] = key[0];
                } else {
                    ulonglong2* kv = reinterpret_cast<ulonglong2*>(tv + slot_key(W));
#pragma unroll
                    for (int w = 0; w < W / 2; w++) kv[w] = make_ulonglong2(key[2 * w], key[2 * w + 1]);
                }
                return true;
            }
            cur = old;
        }
        slot = (slot + 1) & (T - 1);
    }
    return false;
}

// Position of key in the index of buffer b (written by an earlier kernel), or -1.
template <int W>
__device__ __forceinline__ long long index_find(const SfDev& d, int b, unsigned long long T, uint32_t tag,
                                                const uint64_t* key) {
    const uint64_t* sl = d.islot[b];
    unsigned long long slot = hash_sig<W>(key) & (T - 1);
    if constexpr (W == 1) {
        // four slots (64 bytes) per round trip, checked in probe order
        const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(sl);
        for (unsigned long long probed = 0; probed < T;) {
            const unsigned long long g0 = slot & ~3ull;
            ulonglong2 v[4];
#pragma unroll
            for (int i = 0; i < 4; i++) v[i] = __ldg(s2 + g0 + i);
            for (int i = (int)(slot & 3); i < 4; i++, probed++) {
                if ((uint32_t)(v[i].x >> 32) != tag) return -1;
                if (v[i].y == key[0]) return (long long)(uint32_t)v[i].x;
            }
            slot = (g0 + 4) & (T - 1);
        }
        return -1;
    }
    for (unsigned long long probe = 0; probe < T; probe++) {
        const uint64_t* p = sl + slot * slot_words(W);
        const uint64_t tv = __ldg(p);
        if ((uint32_t)(tv >> 32) != tag) return -1;
        const ulonglong2* kv = reinterpret_cast<const ulonglong2*>(p + slot_key(W));
        bool eq = true;
#pragma unroll
        for (int w = 0; w < W / 2; w++) {
            const ulonglong2 v = __ldg(kv + w);
            eq &= v.x == key[2 * w] && v.y == key[2 * w + 1];
        }
        if (eq) return (long long)(uint32_t)tv;
        slot = (slot + 1) & (T - 1);
    }
    return -1;
}

// index_find of the key s ^ m, formed word by word (m in shared memory, read
// at each use): no W-word copy of the key is kept in registers
template <int W>
__device__ __forceinline__ long long index_find_xor(const SfDev& d, int b, unsigned long long T, uint32_t tag,
                                                    const uint64_t* s, const uint64_t* m) {
    if constexpr (W == 1) {
        const uint64_t key = s[0] ^ m[0];
        return index_find<1>(d, b, T, tag, &key);
    } else {
        uint64_t h = 0x9E3779B97F4A7C15ull;  // hash_sig over the words of s ^ m
#pragma unroll
        for (int w = 0; w < W; w++) {
            uint64_t v = (s[w] ^ *(const volatile uint64_t*)&m[w]) + h;
            v ^= v >> 30;
            v *= 0xBF58476D1CE4E5B9ull;
            v ^= v >> 27;
            v *= 0x94D049BB133111EBull;
            v ^= v >> 31;
            h = v + 0x9E3779B97F4A7C15ull * (uint64_t)(w + 1);
        }
        const uint64_t* sl = d.islot[b];
        unsigned long long slot = h & (T - 1);
        for (unsigned long long probe = 0; probe < T; probe++) {
            const uint64_t* p = sl + slot * slot_words(W);
            const uint64_t tv = __ldg(p);
            if ((uint32_t)(tv >> 32) != tag) return -1;
            const ulonglong2* kv = reinterpret_cast<const ulonglong2*>(p + slot_key(W));
            bool eq = true;
#pragma unroll
            for (int w = 0; w < W / 2; w++) {
                const ulonglong2 v = __ldg(kv + w);
                eq &= v.x == (s[2 * w] ^ *(const volatile uint64_t*)&m[2 * w]) &&
                      v.y == (s[2 * w + 1] ^ *(const volatile uint64_t*)&m[2 * w + 1]);
            }
            if (eq) return (long long)(uint32_t)tv;
            slot = (slot + 1) & (T - 1);
        }
        return -1;
    }
}

// Reserve cnt consecutive output positions for each thread of the block with
// one atomic per block: returns the first position of this thread's range.
// Every thread of the block must call it (it synchronises the block).
__device__ __forceinline__ unsigned long long block_out_range(unsigned long long* ctr, unsigned cnt,
                                                              unsigned int* wsum, unsigned long long* bbase) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    unsigned incl = cnt;  // inclusive warp scan of the counts
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = 0;
        for (int i = 0; i < nwarp; i++) {
            const unsigned int c = wsum[i];
            wsum[i] = t;
            t += c;
        }
        *bbase = t ? atomicAdd(ctr, (unsigned long long)t) : 0ull;
    }
    __syncthreads();
    const unsigned long long o = *bbase + wsum[wid] + (incl - cnt);
    __syncthreads();
    return o;
}

// True in exactly one thread-block: the last one to finish (all of its
// threads receive the answer).  Every block of the grid must call it once.
__device__ __forceinline__ bool last_block(unsigned int* done) {
    __shared__ bool am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(done, 1u);
        am_last = (t == gridDim.x - 1);
        if (am_last) *done = 0u;
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

// ---- launch wrappers implemented in the .cu files (one kernel each) --------
void sf_launch_reset(const SfDev& d, int buf, cudaStream_t s);
void sf_launch_clifford(const SfDev& d, const void* dev_gates, int ngates, int buf, uint64_t* gws,
                        cudaStream_t s);
// single-warp version for n <= 63 (W = 1)
void sf_launch_clifford_warp(const SfDev& d, const void* dev_gates, int ngates, int buf, cudaStream_t s);
void sf_launch_measure_prep_warp(const SfDev& d, uint32_t q, int buf, cudaStream_t s);
void sf_launch_measure_prep(const SfDev& d, uint32_t q, int buf, uint64_t* gws, cudaStream_t s);
void sf_launch_amp_prep(const SfDev& d, const uint64_t* dev_y, cudaStream_t s);
// one handle's program in a single-CTA launch while the frame is small (W = 1)
void sf_launch_segment(const SfDev& d, const void* ops, unsigned long long n_ops, double eps2, unsigned seg_cap,
                       int cur, unsigned long long* consumed, unsigned long long* out_meas, cudaStream_t s);
size_t sf_segment_smem_bytes(unsigned seg_cap);
size_t sf_gprog_work_words();
cudaError_t sf_gprog_reset(const SfDev& d, cudaStream_t s);
cudaError_t sf_gprog_moved(const SfDev& d, unsigned long long* host, cudaStream_t s);
// hull_state: 0 unknown, 1 kept in the workspace by the last launch, 2 the
// frame is one element; spin_limit: polls of a grid barrier before it gives
// up; trace: record per-phase times in the workspace; trig: n_ops entries of
// scratch for e^{i theta} of the diagonal records
cudaError_t sf_launch_gprog(const SfDev& d, const void* ops, unsigned long long n_ops, double eps2, int cur,
                            int idx_ok, int hull_state, unsigned spin_limit, int trace, double2* trig,
                            unsigned long long* consumed, cudaStream_t s);
cudaError_t sf_gprog_trace(const SfDev& d, uint64_t* host, unsigned cap, unsigned* n, cudaStream_t s);
cudaError_t sf_gprog_marks(const SfDev& d, uint64_t* host, unsigned m, cudaStream_t s);
cudaError_t sf_gprog_plan_marks(const SfDev& d, uint64_t* host, unsigned m, cudaStream_t s);
size_t sf_tableau_smem_bytes(int n, int W, int NT);

void sf_launch_affine(const SfDev& d, int buf, cudaStream_t s);
// children of a diagonal gate written out unmerged (in -> out)
void sf_launch_branch(const SfDev& d, uint32_t kind, uint32_t q0, uint32_t q1, double theta, int in_buf,
                      int out_buf, cudaStream_t s);
// the elements of a frame (possibly with repeated phase vectors) hashed into the slot table
void sf_launch_insert(const SfDev& d, int in_buf, int out_buf, cudaStream_t s);
void sf_launch_compact(const SfDev& d, double eps, int out_buf, cudaStream_t s);
// diagonal gate with merging through the index of in_buf (children owned by one parent each)
void sf_launch_branch_merge(const SfDev& d, uint32_t kind, uint32_t q0, uint32_t q1, double theta, double eps,
                            int in_buf, int out_buf, cudaStream_t s);
// cofactor split with merging of the two parents of each child
void sf_launch_cof_merge(const SfDev& d, int in_buf, int out_buf, cudaStream_t s);
void sf_launch_build_index(const SfDev& d, int buf, cudaStream_t s);
void sf_launch_cof_pos(const SfDev& d, int in_buf, int out_buf, bool prob, cudaStream_t s);
void sf_launch_filter(const SfDev& d, int x, int in_buf, int out_buf, cudaStream_t s);
void sf_launch_cond(const SfDev& d, int buf, int kind, int c1, int c2, int t, double alpha, cudaStream_t s);
void sf_launch_prob(const SfDev& d, int buf, cudaStream_t s);
void sf_launch_amplitude(const SfDev& d, int buf, cudaStream_t s);
void sf_launch_export(const SfDev& d, int buf, int stage_buf, cudaStream_t s);
size_t sf_affine_smem_bytes(int n, int W);
