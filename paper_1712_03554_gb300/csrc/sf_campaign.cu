// sf_campaign.cu -- batched simulation of many independent small circuits in
// one persistent launch (up to 63 qubits, frames up to 8192 elements each).
//
// One CTA simulates one circuit at a time and pulls the next circuit from a
// work counter.  Warp 0 keeps the circuit's tableau (M, D) in registers and
// runs the tableau algebra (Table 2 conjugation, Invariant 1 repair, global
// phase, branch and cofactor plans; Sec. III-IV); all eight warps run the
// frame passes (affine phase-vector update, merged branching of diagonal
// gates, cofactor split, measurement reductions, collapse) on the circuit's
// frame, which sits in a per-CTA global workspace (L2-resident at these sizes)
// with its phase-vector index in shared memory.  Outputs are compacted with
// block scans and sums run in a fixed order, so a circuit's results do not
// depend on which CTA ran it or what ran beside it.
//
// Measurement outcomes come from the draws in the program: outcome 1 iff the
// draw u < p(1).  A conditional op applies a Clifford gate iff the parity of
// (outcome bits & mask) is 1 (classically controlled correction).
#include <algorithm>
#include <string>

#include "sf.h"
#include "sf_warp.cuh"

using namespace sfw;

namespace {

constexpr int kMaxWarps = 16;  // threads per circuit: 32..256 (campaign), 512 (program segment)
constexpr int kCampMaxCap = SF_CAMPAIGN_MAX_ELEMS;

struct CampDev {
    int n, ncirc;
    unsigned cap;
    double eps2;
    const OpRec* ops;
    const unsigned long long* off;
    uint64_t* ws_sig;  // [gridDim][2][cap]
    double2* ws_amp;   // [gridDim][2][cap]
    uint32_t* ws_idx;  // [gridDim][islots] when the index lives in global memory
    unsigned islots;
    unsigned* next;
    unsigned long long* outcomes;
    uint32_t* nmeas;
    uint32_t* kfinal;
    double* norm;
    int32_t* cstatus;
    uint64_t* ex_sig;  // [ncirc][cap] or null
    double2* ex_amp;   // [ncirc][cap]
    uint64_t* ex_tab;  // [ncirc][129]: x rows, z rows, r
    int sorted;        // coalescing strategy: 0 hash index, 1 positions sorted by phase vector
};

struct Shared {
    BrTab P;
    double2 ctab[4][16];      // group coefficient of the plan per sign pattern (half table)
    CofTab C;
    uint64_t at[64];          // columns of the composed affine map
    uint64_t tab[16 * 16];    // 4-bit lookup tables of the affine map
    uint64_t t;               // sign word of the affine map
    uint64_t rmx[64], rmz[64], rdx[64], rdz[64];
    uint32_t rde[64];
    int32_t rpiv[64];
    double red[2][kMaxWarps];
    unsigned wsum[kMaxWarps];
    Row stage[64];            // row permutation of the tableau reduction
    SfTerms ecf[32];          // terms of the diagonal records tbase .. tbase + 31
    unsigned long long tbase;
    unsigned long long obase, outcomes, oe;
    double2 g;
    double p[2];
    unsigned k, kout, nmeas;
    int cur, rx, status, circ, rnd;
};

// program records: warp 0 walks a run of Clifford gates through a window of
// 32 records per register set (lane L holds record base + L), the next window
// loading while the current one is used
__device__ __forceinline__ OpRec load_rec(const OpRec* ops, unsigned long long i, unsigned long long end) {
    OpRec o;
    if (i < end) {
        o = ops[i];
    } else {
        o.kind = 0xffffffffu;
        o.q0 = o.q1 = o.arg = 0;
        o.param = 0.0;
    }
    return o;
}

__device__ __forceinline__ OpRec shfl_rec(const OpRec& w, int src) {
    OpRec o;
    o.kind = __shfl_sync(SF_FULL, w.kind, src);
    o.q0 = __shfl_sync(SF_FULL, w.q0, src);
    o.q1 = __shfl_sync(SF_FULL, w.q1, src);
    o.arg = __shfl_sync(SF_FULL, w.arg, src);
    o.param = __shfl_sync(SF_FULL, w.param, src);
    return o;
}

__device__ __forceinline__ uint64_t hash1(uint64_t s) {
    uint64_t v = s + 0x9E3779B97F4A7C15ull;
    v ^= v >> 30;
    v *= 0xBF58476D1CE4E5B9ull;
    v ^= v >> 27;
    v *= 0x94D049BB133111EBull;
    v ^= v >> 31;
    return v;
}

__device__ __forceinline__ unsigned slots_for(unsigned k) {
    unsigned t = 64;
    while (t < 2 * k) t <<= 1;
    return t;
}

// index of the frame in buffer sig (k elements): slot = position + 1, 0 empty
__device__ void build_index(uint32_t* idx, const uint64_t* sig, unsigned k) {
    const unsigned T = slots_for(k);
    for (unsigned s = threadIdx.x; s < T; s += blockDim.x) idx[s] = 0;
    __syncthreads();
    for (unsigned j = threadIdx.x; j < k; j += blockDim.x) {
        unsigned slot = (unsigned)hash1(sig[j]) & (T - 1);
        for (unsigned probe = 0; probe < T; probe++) {
            if (atomicCAS(&idx[slot], 0u, j + 1) == 0u) break;
            slot = (slot + 1) & (T - 1);
        }
    }
    __syncthreads();
}

// The sorted alternative (the campaign's coalescing strategy "sort"): idx[0..k)
// holds the positions of the frame ordered by phase vector, found by a stable
// LSD radix sort over the n phase-vector bits, 4 bits per pass, through
// idx[k..2k) (the slot array holds at least 2k entries); lookups are binary
// searches.  Within each pass, tiles of blockDim elements keep their order: a
// warp ranks its equal digits with a match, warps before it add their counts.
__device__ void build_sorted(uint32_t* idx, const uint64_t* sig, unsigned k, int nbits) {
    __shared__ unsigned cnt[kMaxWarps][16];
    __shared__ unsigned base[16];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (int)(blockDim.x >> 5);
    uint32_t* src = idx;
    uint32_t* dst = idx + k;
    for (unsigned j = tid; j < k; j += blockDim.x) src[j] = j;
    for (int shift = 0; shift < nbits; shift += 4) {
        if (tid < 16) {
            base[tid] = 0;
            for (int w = 0; w < nw; w++) cnt[w][tid] = 0;
        }
        __syncthreads();
        for (unsigned j = tid; j < k; j += blockDim.x) atomicAdd(&base[(sig[src[j]] >> shift) & 15], 1u);
        __syncthreads();
        if (tid == 0) {
            unsigned acc = 0;
            for (int d = 0; d < 16; d++) {
                const unsigned c = base[d];
                base[d] = acc;
                acc += c;
            }
        }
        __syncthreads();
        for (unsigned tile = 0; tile < k; tile += blockDim.x) {
            const unsigned j = tile + tid;
            const bool act = j < k;
            const uint32_t pos = act ? src[j] : 0u;
            const unsigned d = act ? (unsigned)((sig[pos] >> shift) & 15) : 16u;
            const unsigned peers = __match_any_sync(SF_FULL, d);
            const unsigned rank = __popc(peers & ((1u << lane) - 1u));
            if (act && lane == __ffs(peers) - 1) cnt[warp][d] = __popc(peers);
            __syncthreads();
            if (act) {
                unsigned off = base[d] + rank;
                for (int w = 0; w < warp; w++) off += cnt[w][d];
                dst[off] = pos;
            }
            __syncthreads();
            if (tid < 16) {
                unsigned add = 0;
                for (int w = 0; w < nw; w++) {
                    add += cnt[w][tid];
                    cnt[w][tid] = 0;
                }
                base[tid] += add;
            }
            __syncthreads();
        }
        uint32_t* t = src;
        src = dst;
        dst = t;
    }
    if (src != idx)
        for (unsigned j = tid; j < k; j += blockDim.x) idx[j] = src[j];
    __syncthreads();
}

__device__ __forceinline__ int find_sorted(const uint32_t* idx, const uint64_t* sig, unsigned k, uint64_t key) {
    unsigned lo = 0, hi = k;
    while (lo < hi) {
        const unsigned mid = (lo + hi) >> 1;
        if (sig[idx[mid]] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < k && sig[idx[lo]] == key) ? (int)idx[lo] : -1;
}

__device__ __forceinline__ int find_index(const uint32_t* idx, const uint64_t* sig, unsigned k, uint64_t key) {
    const unsigned T = slots_for(k);
    unsigned slot = (unsigned)hash1(key) & (T - 1);
    for (unsigned probe = 0; probe < T; probe++) {
        const uint32_t p = idx[slot];
        if (!p) return -1;
        if (sig[p - 1] == key) return (int)(p - 1);
        slot = (slot + 1) & (T - 1);
    }
    return -1;
}

// exclusive block scan of cnt (every thread calls); returns this thread's
// offset and advances S.obase by the block total
__device__ unsigned long long block_scan_advance(Shared& S, unsigned cnt) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned v = __shfl_up_sync(SF_FULL, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) S.wsum[wid] = incl;
    __syncthreads();
    const unsigned long long base = S.obase;
    unsigned before = 0;
    for (int i = 0; i < wid; i++) before += S.wsum[i];
    const unsigned long long o = base + before + (incl - cnt);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) tot += S.wsum[i];
        S.obase = base + tot;
    }
    __syncthreads();
    return o;
}

// deterministic block sum of two doubles, result in S.p
__device__ void block_sum2(Shared& S, double a, double b) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        a += __shfl_xor_sync(SF_FULL, a, off);
        b += __shfl_xor_sync(SF_FULL, b, off);
    }
    if (lane == 0) {
        S.red[0][wid] = a;
        S.red[1][wid] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
            x += S.red[0][i];
            y += S.red[1][i];
        }
        S.p[0] = x;
        S.p[1] = y;
    }
    __syncthreads();
}

__device__ __forceinline__ double2 cof_child1(const CofTab& C, uint64_t s, double2 a, int x, uint64_t& t) {
    const int y = x ^ (__popcll(C.vq & s) & 1);
    t = y ? C.tau1 : C.tau0;
    int ip = 0;
    uint64_t bits = s;
    while (bits) {
        const int h = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        ip += (int)((C.eps0 >> h) & 1) + 2 * (int)((C.eps1 >> h) & 1) + 2 * (__popcll(C.v[h] & t) & 1);
        t ^= C.u[h];
    }
    return ipow_mul(cmul(C.kap[y], a), ip & 3);
}

// canonical-convention phase of D^sigma phi_0(M) (anchor convention), i-power
__device__ int export_phase(const Shared& S, int n, uint64_t s) {
    const int rx = S.rx;
    uint64_t b = 0;
    for (int h = rx; h < n; h++)
        if ((s >> h) & 1) b ^= 1ull << (S.rpiv[h] - n);
    for (int R = 0; R < rx; R++)
        if ((b >> S.rpiv[R]) & 1) b ^= S.rmx[R];
    uint64_t qx = 0, qz = 0;
    int qe = 0;
    uint64_t bits = s;
    while (bits) {
        const int h = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        pmul1(qx, qz, qe, S.rdx[h], S.rdz[h], (int)S.rde[h]);
    }
    const uint64_t w = b ^ qx;
    uint64_t px = 0, pz = 0;
    int pe = 0;
    for (int R = 0; R < rx; R++)
        if ((w >> S.rpiv[R]) & 1) pmul1(px, pz, pe, S.rmx[R], S.rmz[R], 0);
    if (px != w) return -1;
    return (qe + __popcll(qx & qz) + 2 * __popcll(qz & w) + pe + __popcll(px & pz)) & 3;
}

// Runs program records [o0, o1) on one circuit's state: S (frame size, buffer,
// X-block size, global phase, status, outcomes), the tableau rows in warp 0's
// registers r, the two frame buffers sigb/ampb and the index idx of the current
// buffer (valid on entry and on return).  Every thread of the block calls it.
// Exceeding cap is an error (SF_ECAPACITY in S.status); with stop_cap > 0 the
// run instead stops, at an op boundary and without error, before a diagonal
// gate or random measurement whose intermediate frame could exceed stop_cap.
// A run of up to nbm consecutive diagonal records is planned at once into
// pb/cb (warp w plans record w); after a merge that drops nothing, the
// following planned gates that keep the frame closed under its mask are
// applied in place in one pass.  Returns the index of the first record not
// applied.
__device__ __forceinline__ unsigned long long run_ops(Shared& S, Row* r, int n, uint64_t* const* sigb,
                                                      double2* const* ampb, uint32_t* idx, const OpRec* ops,
                                                      unsigned long long o0, unsigned long long o1, unsigned cap,
                                                      double eps2, unsigned stop_cap, BrTab* pb,
                                                      double2 (*cb)[4][16], int nbm, bool sorted = false) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long oi = o0;
    // the frame's index: hash slots, or positions sorted by phase vector
    const auto rebuild = [&](const uint64_t* sg, unsigned kk) {
        if (sorted) build_sorted(idx, sg, kk, n);
        else build_index(idx, sg, kk);
    };
    const auto lookup = [&](const uint64_t* sg, unsigned kk, uint64_t key) {
        return sorted ? find_sorted(idx, sg, kk, key) : find_index(idx, sg, kk, key);
    };
    unsigned long long pbase = 0, pend = 0;  // records planned in the current batch (the same in every thread)
    bool have_u = false;  // the frame is closed under the mask cu (s in F => s ^ cu in F)
    uint64_t cu = 0;
    while (oi < o1 && S.status == 0) {
        const OpRec op0 = ops[oi];
        uint32_t kind = op0.kind;
        bool cond_false = false;
        if (kind == SF_OP_COND) {
            if (op0.arg > 8) {
                if (threadIdx.x == 0) S.status = SF_EINVAL;
                __syncthreads();
                break;
            }
            const uint64_t mask = (uint64_t)__double_as_longlong(op0.param);
            cond_false = !(__popcll(S.outcomes & mask) & 1);
            kind = op0.arg;
        }
        if (cond_false) {  // conditional gate not taken
            oi++;
            continue;
        }
        if (kind <= 8) {
            // a run of consecutive Clifford gates (a conditional gate runs alone);
            // warp 0 walks it through the record window, lane 0 publishes its end
            if (warp == 0) {
                for (int hf = 0; hf < 2; hf++) {
                    const int row = lane + 32 * hf;
                    r[hf].A = row < n ? 1ull << row : 0;
                    r[hf].t0 = 0;
                }
                int rx = S.rx;
                int ga = 0, gb = 0;  // the run's phase factor omega^ga sqrt(2)^gb
                int bad = 0;
                unsigned long long gi = oi, wb = oi;
                OpRec w0 = load_rec(ops, wb + lane, o1), w1 = load_rec(ops, wb + 32 + lane, o1);
                const bool single = op0.kind == SF_OP_COND;
                for (;;) {
                    if (gi - wb >= 32) {
                        wb += 32;
                        w0 = w1;
                        w1 = load_rec(ops, wb + 32 + lane, o1);
                    }
                    const OpRec op = shfl_rec(w0, (int)(gi - wb));
                    gi++;
                    const int gk = (int)(op.kind == SF_OP_COND ? op.arg : op.kind);
                    const bool two = gk >= 6;
                    const int q0 = (int)op.q0, q1 = two ? (int)op.q1 : 0;
                    if (gk > 8 || q0 >= n || (two && (q1 >= n || q1 == q0))) {
                        bad = 1;
                        break;
                    }
                    if (!warp_clifford_gate(r, n, rx, gk, q0, q1, S.stage, ga, gb)) {
                        bad = 2;
                        break;
                    }
                    if (single || gi >= o1) break;
                    const unsigned long long d = gi - wb;  // 1..32
                    const uint32_t nk = d < 32 ? __shfl_sync(SF_FULL, w0.kind, (int)d)
                                               : __shfl_sync(SF_FULL, w1.kind, 0);
                    if (nk > 8) break;
                }
                for (int j = 0; j < n; j++) {
                    const unsigned b0 = __ballot_sync(SF_FULL, lane < n && ((r[0].A >> j) & 1));
                    const unsigned b1 = __ballot_sync(SF_FULL, lane + 32 < n && ((r[1].A >> j) & 1));
                    if (lane == 0) S.at[j] = (uint64_t)b0 | ((uint64_t)b1 << 32);
                }
                const unsigned t0 = __ballot_sync(SF_FULL, lane < n && r[0].t0);
                const unsigned t1 = __ballot_sync(SF_FULL, lane + 32 < n && r[1].t0);
                if (lane == 0) {
                    S.t = (uint64_t)t0 | ((uint64_t)t1 << 32);
                    S.rx = rx;
                    S.g = cmul(S.g, cliff_factor(ga, gb));
                    S.oe = gi;
                    if (bad) S.status = bad == 1 ? SF_EINVAL : SF_EINTERNAL;
                }
            }
            __syncthreads();
            if (S.status) break;
            // sigma' = A sigma ^ t on every element, 4-bit table lookups
            const int nc = (n + 3) >> 2;
            for (int e = threadIdx.x; e < nc * 16; e += blockDim.x) {
                const int v = e & 15, c = e >> 4;
                uint64_t acc = 0;
                for (int b = 0; b < 4; b++)
                    if (((v >> b) & 1) && 4 * c + b < n) acc ^= S.at[4 * c + b];
                S.tab[e] = acc;
            }
            __syncthreads();
            uint64_t* sg = sigb[S.cur];
            const uint64_t tw = S.t;
            for (unsigned j = threadIdx.x; j < S.k; j += blockDim.x) {
                const uint64_t s = sg[j];
                uint64_t o = tw;
                for (int c = 0; c < nc; c++) o ^= S.tab[c * 16 + ((s >> (4 * c)) & 15)];
                sg[j] = o;
            }
            __syncthreads();
            rebuild(sg, S.k);
            have_u = false;
            oi = S.oe;
            continue;
        }
        if (kind >= 16 && kind <= 19) {
            // diagonal gate, merged: owner thread computes each output (Sec. IV)
            const uint32_t gk = kind - 16;
            const int q0 = (int)op0.q0, q1 = (int)op0.q1;
            if (q0 >= n || (gk == 3 && (q1 >= n || q1 == q0))) {
                if (threadIdx.x == 0) S.status = SF_EINVAL;
                __syncthreads();
                break;
            }
            if (oi < pbase || oi >= pend) {
                // plans of the run of diagonal records from oi (at most nbm): the
                // tableau does not change within it, so warp w plans record oi + w.
                // Every warp counts the run itself, so the batch bounds agree in all
                // threads without a barrier.
                int nb = 1;
                if (nbm > 1) {
                    const unsigned long long ri = oi + lane;
                    bool dg = false;
                    if (ri < o1) {
                        const uint32_t kk = ops[ri].kind;
                        dg = kk >= SF_OP_DIAG && kk <= SF_OP_DIAG + 3;
                    }
                    const unsigned bl = __ballot_sync(SF_FULL, dg);
                    nb = bl == SF_FULL ? 32 : __ffs(~bl) - 1;
                    nb = nb < nbm ? nb : nbm;
                    nb = nb < 1 ? 1 : nb;
                }
                pbase = oi;
                pend = oi + nb;
                if (warp == 0) {
                    // the terms of the diagonal records, 32 records at a time (one per
                    // lane), so the narrow double-precision pipe runs one sincos per window
                    if (oi < S.tbase || oi + nb > S.tbase + 32) {
                        const unsigned long long ri = oi + lane;
                        uint32_t rk = 0;
                        double th = 0.0;
                        if (ri < o1) {
                            const OpRec o = ops[ri];
                            if (o.kind >= SF_OP_DIAG && o.kind <= SF_OP_DIAG + 3) {
                                rk = o.kind - SF_OP_DIAG;
                                th = rk == 0 ? 0.78539816339744830962 : (rk == 1 ? -0.78539816339744830962 : o.param);
                            }
                        }
                        double sn, cs;
                        sincos(th, &sn, &cs);
                        const SfTerms T = diag_terms(rk, cs, sn);
                        __syncwarp();
                        S.ecf[lane] = T;
                        if (lane == 0) S.tbase = oi;
                    }
                    if (nb > 1) {
                        for (int hf = 0; hf < 2; hf++) {
                            const int row = lane + 32 * hf;
                            S.rmx[row] = r[hf].mx;
                            S.rmz[row] = r[hf].mz;
                            S.rdx[row] = r[hf].dx;
                            S.rdz[row] = r[hf].dz;
                            S.rde[row] = r[hf].de;
                        }
                    }
                }
                __syncthreads();
                if (warp < nb) {
                    if (warp != 0) {
                        for (int hf = 0; hf < 2; hf++) {
                            const int row = lane + 32 * hf;
                            r[hf].mx = S.rmx[row];
                            r[hf].mz = S.rmz[row];
                            r[hf].dx = S.rdx[row];
                            r[hf].dz = S.rdz[row];
                            r[hf].de = S.rde[row];
                        }
                    }
                    const OpRec o = warp == 0 ? op0 : ops[oi + warp];
                    const uint32_t wk = o.kind - SF_OP_DIAG;
                    // a bad record is planned as a one-qubit gate on qubit 0 and
                    // rejected when the run reaches it
                    const bool okr = (int)o.q0 < n && (wk != 3 || ((int)o.q1 < n && o.q1 != o.q0));
                    warp_branch_plan_regs(r, n, okr ? wk : 2u, okr ? (int)o.q0 : 0, okr && wk == 3 ? (int)o.q1 : 0,
                                          S.ecf[oi + warp - S.tbase].c, pb[warp], cb[warp]);
                }
            }
            __syncthreads();
            // the longest run of planned records from oi that one in-place pass takes:
            // one-group gates (a phase per element) and two-group gates whose second
            // mask is the one the frame is closed under (each pair {s, s ^ u} maps
            // onto itself: phase vectors, positions and the index stay)
            const int t = (int)(oi - pbase);
            int t2 = t;
            bool pairs = false;
            while (t2 < (int)(pend - pbase) && !pb[t2].bad) {
                const BrTab& Q = pb[t2];
                if (Q.ng == 1 || (Q.ng == 2 && have_u && Q.u[1] == cu)) {
                    pairs |= Q.ng == 2;
                    t2++;
                } else {
                    break;
                }
            }
            const unsigned long long kb = keep_bits(eps2);
            if (t2 > t) {
                // the element with the smaller phase vector of each pair applies the
                // run's gates to both amplitudes: the per-gate sums, in the same order
                const unsigned k = S.k;
                const uint64_t* si = sigb[S.cur];
                double2* ai = ampb[S.cur];
                bool drop = false, miss = false;
                const auto plan = [&](int r2) { return PlanRef{&pb[r2], cb[r2]}; };
                const auto find = [&](uint64_t key) { return (long long)lookup(si, k, key); };
                for (unsigned base = 64u * warp; base < k; base += 64u * (blockDim.x >> 5))
                    inplace_run_warp<false>(si, ai, base, k, pairs, cu, t, t2, plan, find, kb, eps2, drop, miss);
                if (__syncthreads_or(miss)) {  // the frame was not closed after all
                    if (threadIdx.x == 0) S.status = SF_EINTERNAL;
                    __syncthreads();
                    break;
                }
                oi += t2 - t;
                if (!__syncthreads_or(drop)) continue;
                // amplitudes fell below the threshold: compact the frame
                const int ib = S.cur, ob = S.cur ^ 1;
                if (threadIdx.x == 0) S.obase = 0;
                __syncthreads();
                for (unsigned base = 0; base < k; base += blockDim.x) {
                    const unsigned j = base + threadIdx.x;
                    const bool act = j < k;
                    const double2 a = act ? ampb[ib][j] : make_double2(0.0, 0.0);
                    const bool keep = act && amp_kept(a, kb, eps2);
                    const unsigned long long o = block_scan_advance(S, keep ? 1u : 0u);
                    if (keep) {
                        sigb[ob][o] = sigb[ib][j];
                        ampb[ob][o] = a;
                    }
                }
                if (threadIdx.x == 0) {
                    S.k = (unsigned)S.obase;
                    S.cur = ob;
                }
                __syncthreads();
                rebuild(sigb[S.cur], S.k);
                have_u = false;
                continue;
            }
            const BrTab& P = pb[t];
            double2(*const ctab)[16] = cb[t];
            const int ng = P.ng;
            if (stop_cap && !P.bad && (unsigned long long)ng * S.k > stop_cap) break;  // stop before this op
            if (P.bad || (unsigned long long)ng * S.k > cap) {
                if (threadIdx.x == 0) S.status = P.bad ? SF_EINTERNAL : SF_ECAPACITY;
                __syncthreads();
                break;
            }
            const int ib = S.cur, ob = S.cur ^ 1;
            const uint64_t* si = sigb[ib];
            const double2* ai = ampb[ib];
            const unsigned k = S.k;
            if (threadIdx.x == 0) S.obase = 0;
            __syncthreads();
            bool drop = false;
            for (unsigned base = 0; base < k; base += blockDim.x) {
                const unsigned j = base + threadIdx.x;
                const bool act = j < k;
                uint64_t s = 0;
                double2 a = make_double2(0.0, 0.0);
                // group loops unrolled with guards and id read through pick_grp,
                // so that id and amps stay in registers
                int id[SF_BR_MAXG] = {act ? (int)j : -1, -1, -1, -1};
                if (act) {
                    s = si[j];
                    a = ai[j];
                }
#pragma unroll
                for (int g = 1; g < SF_BR_MAXG; g++)
                    if (act && g < ng) id[g] = lookup(si, k, s ^ P.u[g]);
                double2 amps[SF_BR_MAXG];
                unsigned keepm = 0;
#pragma unroll
                for (int g = 0; g < SF_BR_MAXG; g++) {
                    amps[g] = make_double2(0.0, 0.0);
                    if (g >= ng) continue;
                    bool own = act;
#pragma unroll
                    for (int g2 = 0; g2 < g; g2++) own &= pick_grp(id, P.xidx[g][g2]) < 0;
                    double2 amp = make_double2(0.0, 0.0);
                    if (own) {
#pragma unroll
                        for (int g2 = 0; g2 < SF_BR_MAXG; g2++) {
                            if (g2 >= ng) continue;
                            const int m = P.xidx[g][g2];
                            const int im = pick_grp(id, m);
                            if (im < 0) continue;
                            const double2 ap = m == 0 ? a : ai[im];
                            cmul_acc(amp, half_coef(P, ctab, g2, s ^ P.u[m]), ap);
                        }
                    }
                    amps[g] = amp;
                    if (own && amp_kept(amp, kb, eps2)) keepm |= 1u << g;
                    else if (own) drop = true;
                }
                unsigned long long o = block_scan_advance(S, __popc(keepm));
#pragma unroll
                for (int g = 0; g < SF_BR_MAXG; g++) {
                    if (!((keepm >> g) & 1u)) continue;
                    sigb[ob][o] = s ^ P.u[g];
                    ampb[ob][o] = amps[g];
                    o++;
                }
            }
            // no output dropped: every parent s gave s ^ u_g for all g, so the new
            // frame is closed under the gate's masks
            const bool dropped = __syncthreads_or(drop);
            have_u = !dropped && ng == 2;
            cu = P.u[1];
            if (threadIdx.x == 0) {
                S.k = (unsigned)S.obase;
                S.cur = ob;
            }
            __syncthreads();
            rebuild(sigb[S.cur], S.k);
            oi++;
            continue;
        }
        if (kind == SF_OP_MEASURE) {
            const int q = (int)op0.q0;
            if (q >= n || S.nmeas >= 64) {
                if (threadIdx.x == 0) S.status = SF_EINVAL;
                __syncthreads();
                break;
            }
            if (stop_cap) {  // stop before a random measurement whose cofactor could exceed stop_cap
                if (warp == 0) {
                    const bool x0 = lane < n && ((r[0].mx >> q) & 1), x1 = lane + 32 < n && ((r[1].mx >> q) & 1);
                    const bool rnd = __any_sync(SF_FULL, x0 || x1);
                    if (lane == 0) S.rnd = rnd ? 1 : 0;
                }
                __syncthreads();
                if (S.rnd && 2ull * S.k > stop_cap) break;
            }
            if (warp == 0) {
                const int rx = warp_measure_prep(r, n, S.rx, q, S.C, S.stage);
                if (lane == 0) S.rx = rx;
            }
            __syncthreads();
            if (S.C.bad || (S.C.random && 2ull * S.k > cap)) {
                if (threadIdx.x == 0) S.status = S.C.bad ? SF_EINTERNAL : SF_ECAPACITY;
                __syncthreads();
                break;
            }
            if (S.C.random) {
                // cofactor split merged: s and s ^ uq share their two children
                const int ib = S.cur, ob = S.cur ^ 1;
                const uint64_t* si = sigb[ib];
                const double2* ai = ampb[ib];
                const unsigned k = S.k;
                if (threadIdx.x == 0) S.obase = 0;
                __syncthreads();
                for (unsigned base = 0; base < k; base += blockDim.x) {
                    const unsigned j = base + threadIdx.x;
                    const bool act = j < k;
                    uint64_t s = 0, p = 0, t[2] = {0, 0};
                    double2 a = make_double2(0.0, 0.0), ap = a, cc[2] = {a, a};
                    int l = -1;
                    bool own = false;
                    if (act) {
                        s = si[j];
                        a = ai[j];
                        p = s ^ S.C.uq;
                        l = lookup(si, k, p);
                        own = l < 0 || s < p;
                        if (l >= 0) ap = ai[l];
                    }
                    unsigned keepm = 0;
                    for (int x = 0; x < 2; x++) {
                        if (!own) continue;
                        double2 c = cof_child1(S.C, s, a, x, t[x]);
                        if (l >= 0) {
                            uint64_t t2;
                            const double2 c2 = cof_child1(S.C, p, ap, x, t2);
                            c.x += c2.x;
                            c.y += c2.y;
                        }
                        cc[x] = c;
                        if (c.x * c.x + c.y * c.y >= 1e-24) keepm |= 1u << x;
                    }
                    unsigned long long o = block_scan_advance(S, __popc(keepm));
                    for (int x = 0; x < 2; x++) {
                        if (!((keepm >> x) & 1u)) continue;
                        sigb[ob][o] = t[x];
                        ampb[ob][o] = cc[x];
                        o++;
                    }
                }
                if (threadIdx.x == 0) {
                    S.k = (unsigned)S.obase;
                    S.cur = ob;
                }
                __syncthreads();
            }
            // probabilities of the two outcomes (Sec. IV), fixed summation order
            const int rq = S.C.rq;
            {
                double p0 = 0.0, p1 = 0.0;
                const uint64_t* sg = sigb[S.cur];
                const double2* am = ampb[S.cur];
                for (unsigned j = threadIdx.x; j < S.k; j += blockDim.x) {
                    const double m = am[j].x * am[j].x + am[j].y * am[j].y;
                    if ((sg[j] >> rq) & 1) p1 += m;
                    else p0 += m;
                }
                block_sum2(S, p0, p1);
            }
            const int xo = op0.param < S.p[1] ? 1 : 0;
            if (!(S.p[xo] > 0.0)) {
                if (threadIdx.x == 0) S.status = SF_ESTATE;
                __syncthreads();
                break;
            }
            const double scale = 1.0 / sqrt(S.p[xo]);
            // collapse onto the outcome
            {
                const int ib = S.cur, ob = S.cur ^ 1;
                const unsigned k = S.k;
                if (threadIdx.x == 0) S.obase = 0;
                __syncthreads();
                for (unsigned base = 0; base < k; base += blockDim.x) {
                    const unsigned j = base + threadIdx.x;
                    const bool keep = j < k && (int)((sigb[ib][j] >> rq) & 1) == xo;
                    const unsigned long long o = block_scan_advance(S, keep ? 1u : 0u);
                    if (keep) {
                        sigb[ob][o] = sigb[ib][j];
                        double2 a = ampb[ib][j];
                        a.x *= scale;
                        a.y *= scale;
                        ampb[ob][o] = a;
                    }
                }
                if (threadIdx.x == 0) {
                    S.k = (unsigned)S.obase;
                    S.cur = ob;
                    if (xo) S.outcomes |= 1ull << S.nmeas;
                    S.nmeas++;
                }
                __syncthreads();
            }
            rebuild(sigb[S.cur], S.k);
            have_u = false;
            oi++;
            continue;
        }
        if (threadIdx.x == 0) S.status = SF_EINVAL;  // unknown op
        __syncthreads();
    }
    __syncthreads();
    return oi;
}

// CT threads per circuit; GIDX: the phase-vector index in a per-CTA slice of
// global memory (L2-resident) instead of shared memory, for more CTAs per SM
template <int CT, bool GIDX>
__global__ void __launch_bounds__(CT) k_campaign(CampDev D) {
    extern __shared__ uint32_t smem_idx[];  // [slots_for(cap)] unless GIDX
    __shared__ Shared S;
    uint32_t* idx = GIDX ? D.ws_idx + (size_t)blockIdx.x * D.islots : smem_idx;
    const int n = D.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* sigb[2] = {D.ws_sig + (size_t)blockIdx.x * 2 * D.cap, D.ws_sig + ((size_t)blockIdx.x * 2 + 1) * D.cap};
    double2* ampb[2] = {D.ws_amp + (size_t)blockIdx.x * 2 * D.cap, D.ws_amp + ((size_t)blockIdx.x * 2 + 1) * D.cap};
    Row r[2];
    for (;;) {
        if (threadIdx.x == 0) S.circ = (int)atomicAdd(D.next, 1u);
        __syncthreads();
        const int ci = S.circ;
        if (ci >= D.ncirc) break;
        // |0...0>: M = Z_h, D = X_h, one element (sigma = 0, a = 1)
        if (warp == 0) {
            for (int hf = 0; hf < 2; hf++) {
                const int row = lane + 32 * hf;
                r[hf].mx = 0;
                r[hf].mz = row < n ? 1ull << row : 0;
                r[hf].dx = row < n ? 1ull << row : 0;
                r[hf].dz = 0;
                r[hf].de = 0;
                r[hf].piv = row < n ? n + row : 0x7fffffff;
                r[hf].A = row < n ? 1ull << row : 0;
                r[hf].t0 = r[hf].t1 = 0;
            }
        }
        if (threadIdx.x == 0) {
            S.k = 1;
            S.cur = 0;
            S.rx = 0;
            S.status = 0;
            S.outcomes = 0;
            S.nmeas = 0;
            S.tbase = ~0ull;
            S.g = make_double2(1.0, 0.0);
            sigb[0][0] = 0;
            ampb[0][0] = make_double2(1.0, 0.0);
        }
        __syncthreads();
        if (D.sorted) build_sorted(idx, sigb[0], 1, n);
        else build_index(idx, sigb[0], 1);
        run_ops(S, r, n, sigb, ampb, idx, D.ops, D.off[ci], D.off[ci + 1], D.cap, D.eps2, 0u, &S.P, &S.ctab, 1,
                D.sorted != 0);
        __syncthreads();
        // results
        double nr = 0.0;
        for (unsigned j = threadIdx.x; j < S.k; j += blockDim.x) {
            const double2 a = ampb[S.cur][j];
            nr += a.x * a.x + a.y * a.y;
        }
        block_sum2(S, nr, 0.0);
        if (threadIdx.x == 0) {
            D.outcomes[ci] = S.outcomes;
            D.nmeas[ci] = S.nmeas;
            D.kfinal[ci] = S.k;
            D.norm[ci] = S.p[0];
            D.cstatus[ci] = S.status;
        }
        if (D.ex_sig) {
            // canonical export: tableau rows and amplitudes in the anchor convention
            if (warp == 0) {
                for (int hf = 0; hf < 2; hf++) {
                    const int row = lane + 32 * hf;
                    if (row < 64) {
                        S.rmx[row] = r[hf].mx;
                        S.rmz[row] = r[hf].mz;
                        S.rdx[row] = r[hf].dx;
                        S.rdz[row] = r[hf].dz;
                        S.rde[row] = r[hf].de;
                        S.rpiv[row] = r[hf].piv;
                    }
                }
            }
            __syncthreads();
            uint64_t* xt = D.ex_tab + (size_t)ci * 129;
            for (int h = threadIdx.x; h < 64; h += blockDim.x) {
                xt[h] = h < n ? S.rmx[h] : 0;
                xt[64 + h] = h < n ? S.rmz[h] : 0;
            }
            if (threadIdx.x == 0) xt[128] = (uint64_t)S.rx;
            const double2 g = S.g;
            for (unsigned j = threadIdx.x; j < S.k; j += blockDim.x) {
                const uint64_t s = sigb[S.cur][j];
                const int ip = export_phase(S, n, s);
                D.ex_sig[(size_t)ci * D.cap + j] = s;
                D.ex_amp[(size_t)ci * D.cap + j] = ip < 0 ? make_double2(NAN, NAN)
                                                             : ipow_mul(cmul(g, ampb[S.cur][j]), ip);
            }
        }
        __syncthreads();
    }
}

// ---- a program on one handle's frame while it is small (sf_apply_program) ----
// The circuit engine above, run by one CTA on a frame handle's own state: the
// tableau rows are loaded into warp 0's registers, frames of up to
// kSegSmemElems elements are copied into shared memory (larger ones stay in the
// handle's buffers), the index and the plans of a diagonal run live in shared
// memory, 16 records planned at a time.  The program is
// checked before anything is touched; the run stops at an op boundary before
// a diagonal gate or random measurement whose intermediate frame could exceed
// seg_cap; the frame is left in buffer `cur` and the tableau, X-block size and
// global phase are written back.
constexpr int kSegThreads = 512;
// frames of up to this many elements stay in shared memory (96 KB for the two buffers)
constexpr unsigned kSegSmemElems = 2048;

__global__ void __launch_bounds__(kSegThreads) k_segment(SfDev d, const OpRec* ops, unsigned long long n_ops,
                                                        double eps2, unsigned seg_cap, int cur,
                                                        unsigned long long* consumed, unsigned long long* out_meas) {
    // [slots_for(seg_cap)] index slots, then (seg_cap <= kSegSmemElems) the two
    // frame buffers: 2 x seg_cap phase vectors, 2 x seg_cap amplitudes
    extern __shared__ uint32_t idx[];
    __shared__ Shared S;
    if (*(volatile uint32_t*)d.status) return;
    const int n = d.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) S.nmeas = 0;
    __syncthreads();
    bool bad = false;
    unsigned nm = 0;
    for (unsigned long long i = threadIdx.x; i < n_ops; i += blockDim.x) {
        const OpRec o = ops[i];
        const uint32_t k = o.kind == SF_OP_COND ? o.arg : o.kind;
        const bool two = (k >= 6 && k <= 8) || k == 19;
        bool ok = o.q0 < (uint32_t)n && (!two || (o.q1 < (uint32_t)n && o.q1 != o.q0));
        if (o.kind == SF_OP_COND) ok &= o.arg <= 8;
        else if (k == SF_OP_MEASURE) nm++;
        else ok &= k <= 8 || (k >= 16 && k <= 19);
        bad |= !ok;
    }
    if (nm) atomicAdd(&S.nmeas, nm);
    bad = __syncthreads_or(bad) != 0;
    if (bad || S.nmeas > 64) {
        if (threadIdx.x == 0) set_status(d.status, 1u, cur, 30u);  // SF_EINVAL: bad record
        return;
    }
    Row r[2];
    if (warp == 0) {
        for (int hf = 0; hf < 2; hf++) {
            const int row = lane + 32 * hf;
            const bool in = row < n;
            r[hf].mx = in ? d.mx[row] : 0;
            r[hf].mz = in ? d.mz[row] : 0;
            r[hf].dx = in ? d.dx[row] : 0;
            r[hf].dz = in ? d.dz[row] : 0;
            r[hf].de = in ? d.de[row] : 0;
            r[hf].piv = in ? d.piv[row] : 0x7fffffff;
            r[hf].A = in ? 1ull << row : 0;
            r[hf].t0 = r[hf].t1 = 0;
        }
    }
    // small frames live in shared memory for the whole program
    const bool in_smem = seg_cap <= kSegSmemElems;
    uint64_t* const fs = reinterpret_cast<uint64_t*>(idx + slots_for(seg_cap));
    double2* const fa = reinterpret_cast<double2*>(fs + 2 * (size_t)seg_cap);
    // then the plans of a run of diagonal records, one per warp
    BrTab* const pbs = reinterpret_cast<BrTab*>(in_smem ? reinterpret_cast<char*>(fa + 2 * (size_t)seg_cap)
                                                         : reinterpret_cast<char*>(fs));
    double2(*const cbs)[4][16] = reinterpret_cast<double2(*)[4][16]>(pbs + kSegThreads / 32);
    uint64_t* const sigb[2] = {in_smem ? fs : d.sig[cur], in_smem ? fs + seg_cap : d.sig[cur ^ 1]};
    double2* const ampb[2] = {in_smem ? fa : d.amp[cur], in_smem ? fa + seg_cap : d.amp[cur ^ 1]};
    if (threadIdx.x == 0) {
        S.k = (unsigned)d.kcnt[cur];
        S.cur = 0;
        S.rx = d.meta[0];
        S.g = *d.g;
        S.status = 0;
        S.outcomes = 0;
        S.nmeas = 0;
        S.tbase = ~0ull;
    }
    __syncthreads();
    unsigned long long done = 0;
    const bool runs = S.k <= seg_cap;
    if (runs) {
        if (in_smem) {
            for (unsigned j = threadIdx.x; j < S.k; j += blockDim.x) {
                fs[j] = d.sig[cur][j];
                fa[j] = d.amp[cur][j];
            }
            __syncthreads();
        }
        build_index(idx, sigb[0], S.k);
        done = run_ops(S, r, n, sigb, ampb, idx, ops, 0, n_ops, seg_cap, eps2, seg_cap, pbs, cbs, kSegThreads / 32);
    }
    if (runs && (in_smem || S.cur == 1)) {
        const uint64_t* fsig = sigb[S.cur];
        const double2* famp = ampb[S.cur];
        for (unsigned j = threadIdx.x; j < S.k; j += blockDim.x) {
            d.sig[cur][j] = fsig[j];
            d.amp[cur][j] = famp[j];
        }
    }
    if (warp == 0) {
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
    }
    if (threadIdx.x == 0) {
        d.meta[0] = S.rx;
        *d.g = S.g;
        d.kcnt[cur] = S.k;
        if (consumed) *consumed = done;
        if (out_meas) {
            out_meas[0] = S.outcomes;
            out_meas[1] = S.nmeas;
        }
        if (S.status) set_status(d.status, (uint32_t)S.status, cur, 31u);
        else if (!consumed && done < n_ops) set_status(d.status, SF_ST_CAPACITY, cur, 32u);
    }
}

// index for frames of up to cap elements (slots_for(cap) slots)
size_t index_slots_for(unsigned cap) {
    size_t t = 64;
    while (t < 2 * (size_t)cap) t <<= 1;
    return t;
}

using CampKernel = void (*)(CampDev);
constexpr int kShapes = 8;  // threads 32 << (i >> 1), index in global memory iff i odd
const CampKernel kKernels[kShapes] = {k_campaign<32, false>,  k_campaign<32, true>,  k_campaign<64, false>,
                                      k_campaign<64, true>,   k_campaign<128, false>, k_campaign<128, true>,
                                      k_campaign<256, false>, k_campaign<256, true>};

int shape_index(uint32_t threads, bool smem_index) {
    int i = threads == 32 ? 0 : threads == 64 ? 2 : threads == 128 ? 4 : threads == 256 ? 6 : -1;
    return i < 0 ? -1 : i + (smem_index ? 0 : 1);
}

}  // namespace

size_t sf_segment_smem_bytes(unsigned seg_cap) {
    return index_slots_for(seg_cap) * sizeof(uint32_t) +
           (seg_cap <= kSegSmemElems ? 2 * (size_t)seg_cap * (sizeof(uint64_t) + sizeof(double2)) : 0) +
           (kSegThreads / 32) * (sizeof(BrTab) + 4 * 16 * sizeof(double2));
}

void sf_launch_segment(const SfDev& d, const void* ops, unsigned long long n_ops, double eps2, unsigned seg_cap,
                       int cur, unsigned long long* consumed, unsigned long long* out_meas, cudaStream_t s) {
    // once per process, thread-safe
    static const bool attr = cudaFuncSetAttribute(k_segment, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  200 * 1024) == cudaSuccess;
    (void)attr;
    k_segment<<<1, kSegThreads, sf_segment_smem_bytes(seg_cap), s>>>(
        d, reinterpret_cast<const OpRec*>(ops), n_ops, eps2, seg_cap, cur, consumed, out_meas);
}

struct sf_campaign_s {
    int n = 0;
    unsigned cap = 0;
    cudaStream_t stream = nullptr;
    int shape = 0;
    int sorted = 0;  // coalescing strategy (CampDev::sorted)
    int nblk_of[kShapes] = {};
    size_t smem_of[kShapes] = {};
    int max_nblk = 0;
    unsigned islots = 0;
    uint64_t* ws_sig = nullptr;
    double2* ws_amp = nullptr;
    uint32_t* ws_idx = nullptr;
    unsigned* next = nullptr;
};

namespace {

sf_status launch_campaign(sf_campaign c, int shape, const sf_op* dev_ops, const uint64_t* dev_offsets,
                          uint32_t n_circuits, double drop_eps, uint64_t* dev_outcomes, uint32_t* dev_n_meas,
                          uint32_t* dev_k_final, double* dev_norm, int32_t* dev_status, uint64_t* ex_sig,
                          double* ex_amp, uint64_t* ex_tab) {
    CampDev D;
    D.n = c->n;
    D.ncirc = (int)n_circuits;
    D.cap = c->cap;
    D.eps2 = drop_eps * drop_eps;
    D.ops = reinterpret_cast<const OpRec*>(dev_ops);
    D.off = reinterpret_cast<const unsigned long long*>(dev_offsets);
    D.ws_sig = c->ws_sig;
    D.ws_amp = c->ws_amp;
    D.ws_idx = c->ws_idx;
    D.islots = c->islots;
    D.next = c->next;
    D.outcomes = reinterpret_cast<unsigned long long*>(dev_outcomes);
    D.nmeas = dev_n_meas;
    D.kfinal = dev_k_final;
    D.norm = dev_norm;
    D.cstatus = dev_status;
    D.ex_sig = ex_sig;
    D.ex_amp = reinterpret_cast<double2*>(ex_amp);
    D.ex_tab = ex_tab;
    D.sorted = c->sorted;
    if (cudaMemsetAsync(c->next, 0, sizeof(unsigned), c->stream) != cudaSuccess) return SF_ECUDA;
    const int threads = 32 << (shape >> 1);
    kKernels[shape]<<<c->nblk_of[shape], threads, c->smem_of[shape], c->stream>>>(D);
    return cudaGetLastError() == cudaSuccess ? SF_OK : SF_ECUDA;
}

}  // namespace

extern "C" {

sf_status sf_campaign_create(uint32_t n_qubits, uint32_t max_elems, void* cuda_stream, sf_campaign* out) {
    if (!out) return SF_EINVAL;
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 63 || max_elems < 1 || max_elems > kCampMaxCap) return SF_EINVAL;
    sf_campaign c = new (std::nothrow) sf_campaign_s();
    if (!c) return SF_ENOMEM;
    c->n = (int)n_qubits;
    c->cap = max_elems;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->islots = (unsigned)index_slots_for(max_elems);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete c;
        return SF_ECUDA;
    }
    // CTAs of each shape: SMs x resident CTAs per SM (registers, shared memory)
    for (int i = 0; i < kShapes; i++) {
        const bool gidx = i & 1;
        const size_t smem = gidx ? 0 : c->islots * sizeof(uint32_t);
        int per_sm = 0;
        if (cudaFuncSetAttribute(kKernels[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kKernels[i], 32 << (i >> 1), smem) !=
                cudaSuccess) {
            cudaGetLastError();
            per_sm = 0;
        }
        c->smem_of[i] = smem;
        c->nblk_of[i] = sms * per_sm;
        c->max_nblk = std::max(c->max_nblk, c->nblk_of[i]);
    }
    // default shape: 64 threads per circuit, index in shared memory while it
    // leaves room for several CTAs per SM
    c->shape = shape_index(64, c->islots * sizeof(uint32_t) <= 32768);
    if (c->nblk_of[c->shape] == 0) {
        c->shape = -1;
        for (int i = 0; i < kShapes; i++)
            if (c->nblk_of[i] > 0) { c->shape = i; break; }
    }
    const size_t ne = (size_t)c->max_nblk * 2 * max_elems;
    if (c->shape < 0 || cudaMalloc(&c->ws_sig, ne * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&c->ws_amp, ne * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->ws_idx, (size_t)c->max_nblk * c->islots * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&c->next, sizeof(unsigned)) != cudaSuccess) {
        const bool nomem = c->shape >= 0;
        sf_campaign_destroy(c);
        return nomem ? SF_ENOMEM : SF_ECUDA;
    }
    *out = c;
    return SF_OK;
}

sf_status sf_campaign_destroy(sf_campaign c) {
    if (!c) return SF_EINVAL;
    cudaStreamSynchronize(c->stream);
    if (c->ws_sig) cudaFree(c->ws_sig);
    if (c->ws_amp) cudaFree(c->ws_amp);
    if (c->ws_idx) cudaFree(c->ws_idx);
    if (c->next) cudaFree(c->next);
    delete c;
    return SF_OK;
}

sf_status sf_campaign_run(sf_campaign c, const sf_op* dev_ops, const uint64_t* dev_offsets, uint32_t n_circuits,
                          double drop_eps, uint64_t* dev_outcomes, uint32_t* dev_n_meas, uint32_t* dev_k_final,
                          double* dev_norm, int32_t* dev_status, uint64_t* dev_export_sigma,
                          double* dev_export_amp, uint64_t* dev_export_tableau) {
    if (!c || !dev_ops || !dev_offsets || !dev_outcomes || !dev_n_meas || !dev_k_final || !dev_norm ||
        !dev_status || !(drop_eps >= 0.0))
        return SF_EINVAL;
    if ((dev_export_sigma != nullptr) != (dev_export_amp != nullptr) ||
        (dev_export_sigma != nullptr) != (dev_export_tableau != nullptr))
        return SF_EINVAL;
    if (n_circuits == 0) return SF_OK;
    return launch_campaign(c, c->shape, dev_ops, dev_offsets, n_circuits, drop_eps, dev_outcomes, dev_n_meas,
                           dev_k_final, dev_norm, dev_status, dev_export_sigma, dev_export_amp, dev_export_tableau);
}

uint32_t sf_campaign_ctas(sf_campaign c) { return c ? (uint32_t)c->nblk_of[c->shape] : 0u; }

sf_status sf_campaign_set_shape(sf_campaign c, uint32_t threads_per_circuit, uint32_t smem_index) {
    if (!c) return SF_EINVAL;
    const int i = shape_index(threads_per_circuit, smem_index != 0);
    if (i < 0 || c->nblk_of[i] == 0) return SF_EINVAL;
    c->shape = i;
    return SF_OK;
}

sf_status sf_campaign_set_coalesce(sf_campaign c, uint32_t sorted_index) {
    if (!c || sorted_index > 1) return SF_EINVAL;
    c->sorted = (int)sorted_index;
    return SF_OK;
}

uint32_t sf_campaign_get_coalesce(sf_campaign c) { return c ? (uint32_t)c->sorted : 0u; }

sf_status sf_campaign_get_shape(sf_campaign c, uint32_t* threads_per_circuit, uint32_t* smem_index,
                                uint32_t* ctas) {
    if (!c) return SF_EINVAL;
    if (threads_per_circuit) *threads_per_circuit = 32u << (c->shape >> 1);
    if (smem_index) *smem_index = (c->shape & 1) ? 0u : 1u;
    if (ctas) *ctas = (uint32_t)c->nblk_of[c->shape];
    return SF_OK;
}

sf_status sf_campaign_autotune(sf_campaign c, const sf_op* dev_ops, const uint64_t* dev_offsets,
                               uint32_t n_circuits, double drop_eps, uint32_t reps, float* best_ms) {
    if (!c || !dev_ops || !dev_offsets || !(drop_eps >= 0.0) || n_circuits == 0) return SF_EINVAL;
    reps = std::max(1u, std::min(reps, 16u));
    uint64_t* outc = nullptr;
    uint32_t *nm = nullptr, *kf = nullptr;
    double* nr = nullptr;
    int32_t* st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sf_status res = SF_OK;
    if (cudaMalloc(&outc, n_circuits * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&nm, n_circuits * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&kf, n_circuits * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&nr, n_circuits * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&st, n_circuits * sizeof(int32_t)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        res = SF_ENOMEM;
    }
    int best = -1, best_sorted = 0;
    float best_t = 0.f;
    const int sorted0 = c->sorted;
    for (int cfg = 0; cfg < 2 * kShapes && res == SF_OK; cfg++) {
        const int i = cfg >> 1;
        if (c->nblk_of[i] == 0) continue;
        c->sorted = cfg & 1;
        // one untimed launch, then the mean of reps timed launches
        res = launch_campaign(c, i, dev_ops, dev_offsets, n_circuits, drop_eps, outc, nm, kf, nr, st, nullptr,
                              nullptr, nullptr);
        if (res != SF_OK) break;
        cudaEventRecord(e0, c->stream);
        for (uint32_t k = 0; k < reps && res == SF_OK; k++)
            res = launch_campaign(c, i, dev_ops, dev_offsets, n_circuits, drop_eps, outc, nm, kf, nr, st, nullptr,
                                  nullptr, nullptr);
        cudaEventRecord(e1, c->stream);
        float ms = 0.f;
        if (res != SF_OK || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            res = SF_ECUDA;
            break;
        }
        ms /= (float)reps;
        if (best < 0 || ms < best_t) {
            best = i;
            best_sorted = c->sorted;
            best_t = ms;
        }
    }
    c->sorted = sorted0;
    if (res == SF_OK && best >= 0) {
        c->shape = best;
        c->sorted = best_sorted;
        if (best_ms) *best_ms = best_t;
    }
    if (outc) cudaFree(outc);
    if (nm) cudaFree(nm);
    if (kf) cudaFree(kf);
    if (nr) cudaFree(nr);
    if (st) cudaFree(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return res;
}

}  // extern "C"
