// sf_gprog.cu -- the grid program: a run of Clifford gates and diagonal gates
// (n <= 63) applied to a frame of any size in one cooperative launch.
//
// The per-op path launches a tableau kernel, an affine pass and an index
// rebuild per Clifford run, and one merge kernel per diagonal gate; each launch
// pays its ramp, its own copy of the gate plan and a last-CTA handshake.  Here
// one persistent CTA per SM walks the records and separates the phases with a
// grid barrier instead:
//
//   Clifford run   warp 0 of CTA 0 runs ROTATE on the tableau in registers
//                  (Sec. III, Table 2) and publishes the run's affine map
//                  sigma' = A sigma ^ t; while it inverts A, the other warps of
//                  CTA 0 plan the diagonal records that follow (one each);
//                  barrier.  The map itself is applied by the next pass over
//                  the elements.
//   diagonal run   records not planned yet are planned at once, CTA c
//                  planning record c (Sec. IV: Z^w = eps D^u M^v per term,
//                  grouped by u, half table of group coefficients); barrier;
//                  then the records are applied in passes over the frame.
//
// Passes over the frame.  Every CTA keeps the frame's linear hull -- the span
// of the differences of its phase vectors -- as parity constraints (c . d = 0
// for every difference d), updated identically in every CTA: a Clifford map
// moves them, a branch along a new direction adds it.  A diagonal gate whose
// two groups differ by a mask u outside the hull has no partners in the frame
// (s ^ u is never a phase vector of it): each element writes its two children
// in place, s at its own position j and s ^ u at j + k, with no index and no
// atomics, and the records that follow and keep each pair {s, s ^ u} (a phase
// per element, or the same mask) are applied to the pair in the same pass.
// The directions of such passes and their strides are remembered while no
// element moves, so later gates along them find each partner by position.
// Gates whose masks lie in the hull go through the phase-vector index: each
// element looks up its partners, one thread owns each output and the outputs
// are reserved with one atomic per block (merge), or, when the frame is
// closed under the mask, the pair is updated in place.  The index is built
// only when a pass needs it.
//
// A measurement or conditional record ends the program (the caller continues
// per op).  Data written inside the launch by other CTAs is read through L2
// (ld.global.cg), never through the non-coherent or L1 paths.  Every barrier
// wait is bounded: on expiry the kernel sets SF_ST_TIMEOUT and returns.
#include <algorithm>

#include "sf.h"
#include "sf_warp.cuh"

using namespace sfw;

namespace {

constexpr int kGpThreads = 512;
constexpr int kGpPlans = 32;              // diagonal records planned per batch
constexpr int kGpTrace = 512;             // phases recorded by a traced launch

struct GpPlan {
    BrTab P;
    double2 ctab[4][16];
    // every term's v is orthogonal to the frame's hull where the record is
    // applied (set by the planner CTA against a hull that contains the workers'
    // hull, so it never claims too much; 0: not known)
    int orth;
    // the end of the run a fresh branch along this record's mask would take
    // (the records after it with one group or the same mask; planning CTAs)
    int rend;
    int pad_[2];
};

// The tableau of the launch.  CTA 0 writes it back at the end.
struct GpTab {
    uint64_t mx[64], mz[64], dx[64], dz[64];
    uint32_t de[64];
    int piv[64];
    int rx;       // X-block size
    double2 g;    // global phase
};

// The planning of the program runs on two CTAs ahead of the workers: the
// tableau CTA applies the Clifford runs and passes each run's tableau and map
// on (a GpTabSet), the plan CTA plans the diagonal records that follow and
// passes the whole step to the workers (a GpSet).  Each ring holds kGpRing
// steps.
constexpr int kGpRing = 4;
struct GpTabSet {
    int kind;                   // 0: Clifford run [oi, oe), 1: no Clifford run, 2: a tableau check failed, 3: end
    int np;                     // diagonal records from ds
    unsigned long long oe, ds;
    GpTab tab;
    uint64_t at[64], ainv[64];
    uint64_t t;
};
// One planned step: a Clifford run [oi, oe) with its map and the plans of the
// diagonal records [oe, oe + np) that follow it, or the plans of a diagonal
// run [oi, oi + np) alone.
struct GpSet {
    int kind;                   // 0: Clifford run and plans, 1: plans only, 2: a tableau check failed
    int np;
    unsigned long long oe;      // end of the Clifford run (kind 0)
    GpTab tab;                  // the tableau after the run
    uint64_t at[64], ainv[64];  // columns of A, rows of A^-1
    uint64_t t;
    GpPlan plans[kGpPlans];
};

// device workspace, zeroed at handle creation; err ... cleared_end is cleared
// before every launch
struct GpWork {
    GpLayout lay;                // the frame's layout after the last launch (read by the positional cofactor)
    unsigned int bar_count, bar_gen;
    unsigned int err[3];         // a failed check in phase p (between barriers p and p + 1): err[p % 3]
    unsigned int drop[3];        // an amplitude dropped in phase p: drop[p % 3]
    unsigned long long ocnt[3];  // output counters of consecutive merges, rotating
    unsigned long long fk[3][2]; // children kept by consecutive in-place branch passes (s, s ^ u), rotating
    unsigned long long moved;    // element bytes read and written by this launch's passes
    unsigned long long ring_seq[kGpRing];  // 1 + the step number published in each ring slot
    unsigned int ring_readers[kGpRing];    // worker CTAs that copied the slot's step
    unsigned long long tring_seq[kGpRing]; // the same for the tableau CTA's ring
    unsigned int tring_readers[kGpRing];   // (its one reader: the plan CTA)
    unsigned int checked;                  // the records passed the check (the planner may start)
    unsigned long long cleared_end;
    uint64_t hull[64];           // the frame's hull constraints at the end of the last launch
    uint64_t hbasis[64];         // and directions spanning the hull
    unsigned int nhb;
    unsigned int ntrace;         // phases recorded by the last traced launch
    // per phase of a traced launch: what ran (code | elements << 8), CTA 0's
    // start and arrival time, the last arrival's time and CTA (ns, %globaltimer)
    uint64_t trace[kGpTrace][5];
    uint64_t marks[kGpTrace][8];  // checkpoints inside each traced phase (CTA 0)
    // per planning step of a traced launch (%globaltimer, thread 0 of the planning
    // CTAs): the tableau CTA's start and publication of the step, then the plan
    // CTA's take of the tableau, copy done, plans done, runs' ends and hull map
    // done, hull walk and verdicts done, publication
    uint64_t pmarks[kGpTrace][8];
    GpSet ring[kGpRing];
    GpTabSet tring[kGpRing];
};

// With three CTAs or more, the last two plan (the tableau CTA, then the plan
// CTA) and the others work on the frame; otherwise every CTA plans for itself
__device__ __forceinline__ bool gp_piped() { return gridDim.x >= 3; }
__device__ __forceinline__ unsigned gp_nwork() { return gp_piped() ? gridDim.x - 2 : gridDim.x; }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" : : "l"(p), "l"(v) : "memory");
}

__shared__ unsigned s_phase;   // phase of the grid program this CTA is in
__shared__ int s_drop;         // an amplitude was dropped in the phase that ended at the last barrier
__shared__ unsigned s_spin;    // barrier polls before giving up
__shared__ int s_trace;        // record per-phase times
__shared__ unsigned s_gen0;    // barrier generation at launch start
__shared__ uint64_t s_tstart;  // CTA 0: when the current phase started
__shared__ uint64_t s_code;    // CTA 0: what the current phase runs

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// checkpoint i of the current phase (traced launches, CTA 0, one thread)
__device__ __forceinline__ void gp_mark(GpWork* w, int i) {
    if (s_trace && blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned ti = s_phase - s_gen0;
        if (ti < (unsigned)kGpTrace) w->marks[ti][i] = gtimer();
    }
}

// checkpoint i of planning step st (traced launches, thread 0 of a planning CTA)
__device__ __forceinline__ void gp_pmark(GpWork* w, unsigned st, int i) {
    if (s_trace && threadIdx.x == 0 && st < (unsigned)kGpTrace) w->pmarks[st][i] = gtimer();
}

// the phase about to end ran `code` over k elements (traced launches, CTA 0)
__device__ __forceinline__ void gp_phase(int code, unsigned long long k) {
    if (blockIdx.x == 0 && threadIdx.x == 0) s_code = (uint64_t)code | ((uint64_t)k << 8);
}

// a failed check of this CTA: every CTA stops at the next barrier
__device__ __forceinline__ void gp_fail(GpWork* w) { atomicExch(&w->err[s_phase % 3], 1u); }
// an amplitude of this CTA fell below the drop threshold in this phase
__device__ __forceinline__ void gp_dropped(GpWork* w) { atomicExch(&w->drop[s_phase % 3], 1u); }

// Grid barrier: every CTA passes the same sequence of barriers.  Thread 0
// arrives with one atomic; the last arrival resets the count and bumps the
// generation, the others poll it, at most s_spin times.  Returns false in
// every thread of every CTA if a check failed in the phase that ends here, and
// in the CTA whose wait ran out (which also fails the phase, so that a CTA
// still passing this barrier stops at its next one).  The error word of a
// phase is cleared two phases ahead, once every CTA has read it.
__device__ bool gp_barrier(GpWork* w, unsigned& gen, uint32_t* status, int buf) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned g = gen;
        int ok = 1;
        const uint64_t t_arr = s_trace ? gtimer() : 0;
        const unsigned ti = g - s_gen0;
        if (s_trace && blockIdx.x == 0 && ti < (unsigned)kGpTrace) {
            w->trace[ti][0] = s_code;
            w->trace[ti][1] = s_tstart;
            w->trace[ti][2] = t_arr;
        }
        if (atomicAdd(&w->bar_count, 1u) == gp_nwork() - 1) {
            if (s_trace && ti < (unsigned)kGpTrace) {
                w->trace[ti][3] = t_arr;
                w->trace[ti][4] = blockIdx.x;
            }
            w->bar_count = 0;
            __threadfence();
            atomicExch(&w->bar_gen, g + 1);
        } else {
            unsigned spins = 0;
            while (ld_acquire(&w->bar_gen) == g) {
                if (++spins > s_spin) {
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        if (s_trace && blockIdx.x == 0) {
            s_tstart = gtimer();
            s_code = 0;
        }
        __threadfence();
        if (!ok) {
            set_status(status, SF_ST_TIMEOUT, buf, 40u);
            atomicExch(&w->err[g % 3], 1u);
        }
        if (__ldcg(&w->err[g % 3])) ok = 0;
        s_drop = __ldcg(&w->drop[g % 3]) != 0;
        if (blockIdx.x == 0) w->err[(g + 2) % 3] = w->drop[(g + 2) % 3] = 0;
        gen = g + 1;
        s_phase = g + 1;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---- the frame's hull (span of the differences of its phase vectors) ------------
// kept as up to 64 parity constraints c (c . d = 0 for every difference d);
// zero constraints say nothing.  All of a CTA's threads read the same values.

// u lies outside the hull: some constraint has odd parity with it (per warp, no sync)
__device__ __forceinline__ bool hull_fresh(const uint64_t* hc, uint64_t u) {
    const int lane = threadIdx.x & 31;
    const bool odd = (__popcll(hc[lane] & u) & 1) | (__popcll(hc[lane + 32] & u) & 1);
    return __any_sync(SF_FULL, odd);
}

// the hull grows by u (warp 0; the caller synchronises the block afterwards):
// one constraint with odd parity is added to the other odd ones and dropped
__device__ __forceinline__ void hull_add(uint64_t* hc, uint64_t u) {
    const int lane = threadIdx.x & 31;
    uint64_t c0 = hc[lane], c1 = hc[lane + 32];
    const bool o0 = __popcll(c0 & u) & 1, o1 = __popcll(c1 & u) & 1;
    const unsigned b0 = __ballot_sync(SF_FULL, o0), b1 = __ballot_sync(SF_FULL, o1);
    if (!(b0 | b1)) return;
    const int p = b0 ? __ffs(b0) - 1 : 32 + __ffs(b1) - 1;
    const uint64_t cp = __shfl_sync(SF_FULL, p < 32 ? c0 : c1, p & 31);
    if (o0) c0 ^= cp;
    if (o1) c1 ^= cp;
    hc[lane] = c0;
    hc[lane + 32] = c1;
}

// The same on constraints held in registers by warp 0 (lane i: constraints i
// and i + 32), for a walk that tests and grows the hull many times in a row.
__device__ __forceinline__ bool hull_fresh_r(uint64_t c0, uint64_t c1, uint64_t u) {
    const bool odd = (__popcll(c0 & u) & 1) | (__popcll(c1 & u) & 1);
    return __any_sync(SF_FULL, odd);
}
__device__ __forceinline__ void hull_add_r(uint64_t& c0, uint64_t& c1, uint64_t u) {
    const bool o0 = __popcll(c0 & u) & 1, o1 = __popcll(c1 & u) & 1;
    const unsigned b0 = __ballot_sync(SF_FULL, o0), b1 = __ballot_sync(SF_FULL, o1);
    if (!(b0 | b1)) return;
    const int p = b0 ? __ffs(b0) - 1 : 32 + __ffs(b1) - 1;
    const uint64_t cp = __shfl_sync(SF_FULL, p < 32 ? c0 : c1, p & 31);
    if (o0) c0 ^= cp;
    if (o1) c1 ^= cp;
}

// position of key in the index of buffer b (written in this launch), or -1.
// Linear probing, read four slots (64 bytes) per round trip: the slots of an
// aligned group are loaded together and checked in probe order.
__device__ __forceinline__ long long gp_find(const SfDev& d, int b, unsigned long long T, uint32_t tag, uint64_t key) {
    const ulonglong2* sl = reinterpret_cast<const ulonglong2*>(d.islot[b]);
    unsigned long long slot = hash_sig<1>(&key) & (T - 1);
    for (unsigned long long probed = 0; probed < T;) {
        const unsigned long long g0 = slot & ~3ull;
        ulonglong2 v[4];
#pragma unroll
        for (int i = 0; i < 4; i++) v[i] = __ldcg(sl + g0 + i);
        for (int i = (int)(slot & 3); i < 4; i++, probed++) {
            if ((uint32_t)(v[i].x >> 32) != tag) return -1;
            if (v[i].y == key) return (long long)(uint32_t)v[i].x;
        }
        slot = (g0 + 4) & (T - 1);
    }
    return -1;
}

// ROTATE over the run of Clifford records from oi (warp 0 of a CTA) on the
// CTA's tableau: the rows in registers, written back with the X-block size and
// global phase.  The composed affine map sigma' = A sigma ^ t goes to at
// (column j = image of e_j) and *t, the rows of A^-1 to ainv (A^-T tracked
// through the reduction, so no inversion follows); returns the run's end, or
// ~0 if a tableau check failed.  cstage: 64 words of shared memory.
__device__ unsigned long long gp_clifford_run(GpTab& T, const OpRec* ops, unsigned long long oi,
                                              unsigned long long o1, int n, Row* stage, uint64_t* cstage, uint64_t* at,
                                              uint64_t* ainv, uint64_t* t_out) {
    const int lane = threadIdx.x & 31;
    Row r[2];
    uint64_t C[2];  // rows of A^-T, riding with the rows
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        const bool in = row < n;
        r[hf].mx = in ? T.mx[row] : 0;
        r[hf].mz = in ? T.mz[row] : 0;
        r[hf].dx = in ? T.dx[row] : 0;
        r[hf].dz = in ? T.dz[row] : 0;
        r[hf].de = in ? T.de[row] : 0;
        r[hf].piv = in ? T.piv[row] : 0x7fffffff;
        r[hf].A = in ? (1ull << row) : 0;
        C[hf] = r[hf].A;
        r[hf].t0 = 0;
        r[hf].t1 = 0;
    }
    int rx = T.rx;
    int ga = 0, gb = 0;  // the run's phase factor omega^ga sqrt(2)^gb
    unsigned long long gi = oi;
    bool good = true;
    // records are read 32 at a time, lane L holding record wb + L
    unsigned long long wb = gi;
    OpRec wr;
    wr.kind = 0xffffffffu;
    if (wb + lane < o1) wr = ops[wb + lane];
    for (;;) {
        if (gi - wb >= 32) {
            wb = gi;
            wr.kind = 0xffffffffu;
            if (wb + lane < o1) wr = ops[wb + lane];
        }
        const int src = (int)(gi - wb);
        const uint32_t kind = __shfl_sync(SF_FULL, wr.kind, src);
        if (gi >= o1 || kind > 8) break;
        if (kind >= 3 && kind <= 5) {
            // consecutive Pauli gates multiplied into P = i^e X^a Z^b (each gate
            // applied after the product so far: X_q flips a_q; Z_q X^a = (-1)^{a_q}
            // X^a Z_q; Y_q = i X_q Z_q), then applied once
            uint64_t pa = 0, pb = 0;
            int pe = 0;
            for (;;) {
                if (gi - wb >= 32) {
                    wb = gi;
                    wr.kind = 0xffffffffu;
                    if (wb + lane < o1) wr = ops[wb + lane];
                }
                const int sp = (int)(gi - wb);
                const uint32_t kp = __shfl_sync(SF_FULL, wr.kind, sp);
                if (gi >= o1 || kp < 3 || kp > 5) break;
                const int q = (int)__shfl_sync(SF_FULL, wr.q0, sp);
                const uint64_t m = 1ull << q;
                const int aq = (int)((pa >> q) & 1);
                if (kp == 3) {
                    pa ^= m;
                } else if (kp == 5) {
                    pe += 2 * aq;
                    pb ^= m;
                } else {
                    pe += 1 + 2 * aq;
                    pa ^= m;
                    pb ^= m;
                }
                gi++;
            }
            if (!warp_pauli_run(r, n, rx, pa, pb, pe & 3, ga)) {
                good = false;
                break;
            }
            continue;
        }
        const int q0 = (int)__shfl_sync(SF_FULL, wr.q0, src);
        const int q1 = kind >= 6 ? (int)__shfl_sync(SF_FULL, wr.q1, src) : 0;
        if (!warp_clifford_gate(r, n, rx, (int)kind, q0, q1, stage, ga, gb, C, cstage)) {
            good = false;
            break;
        }
        gi++;
    }
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        if (row < n) {
            T.mx[row] = r[hf].mx;
            T.mz[row] = r[hf].mz;
            T.dx[row] = r[hf].dx;
            T.dz[row] = r[hf].dz;
            T.de[row] = r[hf].de;
            T.piv[row] = r[hf].piv;
        }
    }
    for (int j = 0; j < n; j++) {
        const unsigned b0 = __ballot_sync(SF_FULL, lane < n && ((r[0].A >> j) & 1));
        const unsigned b1 = __ballot_sync(SF_FULL, lane + 32 < n && ((r[1].A >> j) & 1));
        const unsigned c0 = __ballot_sync(SF_FULL, lane < n && ((C[0] >> j) & 1));
        const unsigned c1 = __ballot_sync(SF_FULL, lane + 32 < n && ((C[1] >> j) & 1));
        if (lane == 0) {
            at[j] = (uint64_t)b0 | ((uint64_t)b1 << 32);
            ainv[j] = (uint64_t)c0 | ((uint64_t)c1 << 32);  // row j of A^-1 = column j of A^-T
        }
    }
    const unsigned t0 = __ballot_sync(SF_FULL, lane < n && r[0].t0);
    const unsigned t1 = __ballot_sync(SF_FULL, lane + 32 < n && r[1].t0);
    if (lane == 0) {
        *t_out = (uint64_t)t0 | ((uint64_t)t1 << 32);
        T.rx = rx;
        T.g = cmul(T.g, cliff_factor(ga, gb));
    }
    __syncwarp();
    return good ? gi : ~0ull;
}

// Plan of diagonal record o (one warp) from the CTA's tableau, with its four
// term coefficients from the launch's table
__device__ void gp_plan(const GpTab& T, int n, const OpRec& o, const double2* cf, GpPlan& out) {
    const int lane = threadIdx.x & 31;
    Row r[2];
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        const bool in = row < n;
        r[hf].mx = in ? T.mx[row] : 0;
        r[hf].mz = in ? T.mz[row] : 0;
        r[hf].dx = in ? T.dx[row] : 0;
        r[hf].dz = in ? T.dz[row] : 0;
        r[hf].de = in ? T.de[row] : 0;
    }
    const uint32_t kind = o.kind - SF_OP_DIAG;
    double2 c[4];
#pragma unroll
    for (int j = 0; j < 4; j++) c[j] = __ldcg(&cf[j]);
    warp_branch_plan_regs(r, n, kind, (int)o.q0, kind == 3 ? (int)o.q1 : 0, c, out.P, out.ctab);
    __syncwarp();
}

// number of consecutive diagonal records from ri, at most kGpPlans (every lane)
__device__ __forceinline__ int diag_count(const OpRec* ops, unsigned long long ri, unsigned long long n_ops) {
    const int lane = threadIdx.x & 31;
    bool dg = false;
    if (ri + lane < n_ops) {
        const uint32_t kk = ops[ri + lane].kind;
        dg = kk >= SF_OP_DIAG && kk <= SF_OP_DIAG + 3;
    }
    const unsigned bl = __ballot_sync(SF_FULL, dg);
    const int nb = bl == SF_FULL ? 32 : __ffs(~bl) - 1;
    return nb < kGpPlans ? nb : kGpPlans;
}

// elements [lo, hi) of CTA b: contiguous chunks, whole warps, all CTAs busy
__device__ __forceinline__ void gp_chunk(unsigned long long k, unsigned long long& lo, unsigned long long& hi) {
    const unsigned nw = gp_nwork();
    const unsigned long long per = ((k + nw - 1) / nw + 31) / 32 * 32;
    lo = min(k, (unsigned long long)blockIdx.x * per);
    hi = min(k, lo + per);
}

// One record r of an in-place run applied to the pair (s0, a0), (s1, a1) with
// s1 = s0 ^ u (u the mask of its second group, if it has one): each output
// sums its own group-0 term and its partner's group-1 term, in that order (the
// order of the per-gate merge).  A missing partner enters with a1 = 0.
// Without kPairs only (s0, a0) is updated (every record has one group).
template <bool kPairs>
__device__ __forceinline__ void pair_step(const GpPlan& pl, uint64_t s0, uint64_t s1, double2& a0, double2& a1) {
    const BrTab& Q = pl.P;
    double2 n0 = make_double2(0.0, 0.0);
    cmul_acc(n0, half_coef(Q, pl.ctab, 0, s0), a0);
    if (kPairs) {
        double2 n1 = make_double2(0.0, 0.0);
        if (Q.ng == 2) cmul_acc(n0, half_coef(Q, pl.ctab, 1, s1), a1);
        cmul_acc(n1, half_coef(Q, pl.ctab, 0, s1), a1);
        if (Q.ng == 2) cmul_acc(n1, half_coef(Q, pl.ctab, 1, s0), a0);
        a1 = n1;
    }
    a0 = n0;
}

// ---- runs whose coefficients do not depend on the element ------------------------
// A term's sign pattern bit parity(v . s) is the same for every phase vector s
// of the frame when v is orthogonal to every direction of the hull (the
// differences of the frame's phase vectors).  When that holds for every term
// of every record of a run, each record acts on the pair (s, s ^ u) through one
// 2x2 matrix for the whole frame, and the run is their product, formed once by
// a warp as a tree (5 levels instead of one dependent step per record); each
// element then takes a single 2x2 product.

struct Cm2 {  // 2x2 complex matrix (a0', a1') = M (a0, a1)
    double2 m00, m01, m10, m11;
};

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a * b + c
    double2 r;
    r.x = fma(a.x, b.x, c.x);
    r.x = fma(-a.y, b.y, r.x);
    r.y = fma(a.x, b.y, c.y);
    r.y = fma(a.y, b.x, r.y);
    return r;
}
__device__ __forceinline__ double2 cprod(double2 a, double2 b) { return cfma(a, b, make_double2(0.0, 0.0)); }

// Warp 0: if every term of records [r0, r1) (at most 32) is orthogonal to the
// hull directions hb[0 .. nhb), the product of their pair matrices at
// (s0, s0 ^ u) into *out and true (every lane); otherwise false.
__device__ bool uniform_run(const GpPlan* spl, int r0, int r1, const uint64_t* hb, int nhb, uint64_t s0, uint64_t u,
                            bool flags, double (*cm)[8], Cm2* out) {
    const int lane = threadIdx.x & 31;
    const int r = r0 + lane;
    if (flags) {  // the planner's per-record verdicts
        if (!__all_sync(SF_FULL, r >= r1 || spl[r].orth)) return false;
    } else {
    // every term against every hull direction: the directions in registers
    // (lane L holds hb[L] and hb[L + 32]), each record's terms read by all lanes
    // at once, all of its words in one batch of independent loads
    const uint64_t h0 = lane < nhb ? hb[lane] : 0ull, h1 = lane + 32 < nhb ? hb[lane + 32] : 0ull;
    bool odd = false;
    for (int rr = r0; rr < r1; rr++) {
        const BrTab& Q = spl[rr].P;
        const int ng = Q.ng;
        int nt[4];
        uint64_t v[4][4];
#pragma unroll
        for (int g = 0; g < 4; g++) {
            nt[g] = Q.nt[g];
#pragma unroll
            for (int t = 0; t < 4; t++) v[g][t] = Q.v[g][t];
        }
#pragma unroll
        for (int g = 0; g < 4; g++)
#pragma unroll
            for (int t = 0; t < 4; t++)
                if (g < ng && t < nt[g]) odd |= ((__popcll(v[g][t] & h0) | __popcll(v[g][t] & h1)) & 1) != 0;
    }
    if (__any_sync(SF_FULL, odd)) return false;
    }
    Cm2 M;
    M.m00 = M.m11 = make_double2(1.0, 0.0);
    M.m01 = M.m10 = make_double2(0.0, 0.0);
    if (r < r1) {
        const BrTab& Q = spl[r].P;
        const uint64_t s1 = s0 ^ u;
        M.m00 = half_coef(Q, spl[r].ctab, 0, s0);
        M.m11 = half_coef(Q, spl[r].ctab, 0, s1);
        if (Q.ng == 2) {
            M.m01 = half_coef(Q, spl[r].ctab, 1, s1);
            M.m10 = half_coef(Q, spl[r].ctab, 1, s0);
        }
    }
    // The product, later records on the left, as a tree of ceil(log2(records))
    // levels through shared memory: each 2x2 complex product is spread over 8
    // lanes, one real output each (4 fused multiply-adds), so that 4 products
    // fill one warp instruction -- a double-precision instruction occupies the
    // pipe as long for one active lane as for 32.
    if (r < r1) {
        cm[lane][0] = M.m00.x; cm[lane][1] = M.m00.y;
        cm[lane][2] = M.m01.x; cm[lane][3] = M.m01.y;
        cm[lane][4] = M.m10.x; cm[lane][5] = M.m10.y;
        cm[lane][6] = M.m11.x; cm[lane][7] = M.m11.y;
    }
    __syncwarp();
    const int o = lane & 7, e = o >> 1, im = o & 1, ri = e >> 1, cj = e & 1;
    for (int cnt = r1 - r0; cnt > 1;) {
        const int np = cnt >> 1;  // products (2q + 1) x (2q); an odd last matrix carries over
        double res[4];
#pragma unroll
        for (int rd = 0; rd < 4; rd++) {
            const int q = 4 * rd + (lane >> 3);
            double v = 0.0;
            if (q < np) {
                const double* X = cm[2 * q + 1];
                const double* Y = cm[2 * q];
                // entry (ri, cj) = X[ri][0] Y[0][cj] + X[ri][1] Y[1][cj]
                const double a0r = X[(2 * ri) * 2], a0i = X[(2 * ri) * 2 + 1];
                const double a1r = X[(2 * ri + 1) * 2], a1i = X[(2 * ri + 1) * 2 + 1];
                const double b0r = Y[cj * 2], b0i = Y[cj * 2 + 1];
                const double b1r = Y[(2 + cj) * 2], b1i = Y[(2 + cj) * 2 + 1];
                // re: a0r b0r - a0i b0i + a1r b1r - a1i b1i
                // im: a0r b0i + a0i b0r + a1r b1i + a1i b1r
                // (operands selected and signs flipped by integer operations, so
                // every lane issues the same four double-precision instructions)
                const double y1 = im ? b0i : b0r, y2 = im ? b0r : b0i;
                const double y3 = im ? b1i : b1r, y4 = im ? b1r : b1i;
                const double x2 = dneg_if(a0i, !im), x4 = dneg_if(a1i, !im);
                v = fma(a0r, y1, fma(x2, y2, fma(a1r, y3, x4 * y4)));
            }
            res[rd] = v;
        }
        const double carry = (cnt & 1) && lane < 8 ? cm[cnt - 1][lane] : 0.0;
        __syncwarp();
#pragma unroll
        for (int rd = 0; rd < 4; rd++) {
            const int q = 4 * rd + (lane >> 3);
            if (q < np) cm[q][o] = res[rd];
        }
        if ((cnt & 1) && lane < 8) cm[np][lane] = carry;
        __syncwarp();
        cnt = np + (cnt & 1);
    }
    if (lane == 0) {
        M.m00 = make_double2(cm[0][0], cm[0][1]);
        M.m01 = make_double2(cm[0][2], cm[0][3]);
        M.m10 = make_double2(cm[0][4], cm[0][5]);
        M.m11 = make_double2(cm[0][6], cm[0][7]);
        *out = M;
    }
    __syncwarp();
    return true;
}

// kept-children counts of a warp added to the pass's counters
__device__ __forceinline__ void add_counts(unsigned long long* ctr, unsigned c0, unsigned c1) {
    c0 = __reduce_add_sync(SF_FULL, c0);
    c1 = __reduce_add_sync(SF_FULL, c1);
    if ((threadIdx.x & 31) == 0) {
        if (c0) atomicAdd(&ctr[0], (unsigned long long)c0);
        if (c1) atomicAdd(&ctr[1], (unsigned long long)c1);
    }
}

// hull_state: 0 nothing known about the frame's hull, 1 the constraints in
// w->hull hold, 2 the frame is one element (the hull is {0}).  idx_ok0: the
// index of buffer cur0 is valid.
__global__ void __launch_bounds__(kGpThreads) k_gprog(SfDev d, GpWork* w, const OpRec* ops, unsigned long long n_ops,
                                                      double eps2, int cur0, int idx_ok0, int hull_state,
                                                      unsigned spin_limit, int trace, double2* trig,
                                                      unsigned long long* consumed) {
    extern __shared__ GpPlan spl[];  // [kGpPlans]: the plans of the current diagonal run
    __shared__ BrTab pm;             // a plan moved to the coordinates before a pending affine map
    __shared__ GpTab s_tab;          // this CTA's copy of the tableau
    // the last Clifford run's map: columns of A, rows of A^-1 (first the rows of A), t
    __shared__ uint64_t s_ainv[64], s_at[64];
    __shared__ uint64_t s_t;
    __shared__ unsigned long long s_oe;
    __shared__ uint64_t tab[16 * 16];
    __shared__ Row stage[64];
    __shared__ uint64_t s_cst[64];
    __shared__ unsigned int wsum[kGpThreads / 32];
    __shared__ unsigned long long bbase;
    __shared__ uint64_t s_hc[64];            // hull constraints
    __shared__ uint64_t s_hb[64];            // directions spanning the hull
    __shared__ int s_nhb;
    __shared__ Cm2 s_comp;                   // product of a run's pair matrices
    __shared__ double s_cm[32][8];           // ... and the levels of its tree
    __shared__ int s_uni;                    // ... valid for the current pass
    __shared__ uint64_t s_ref;               // a phase vector of the frame (new coordinates)
    __shared__ int s_take, s_np, s_kind;     // a planned step taken from the ring: ok, records, kind
    __shared__ int s_png[kGpPlans], s_pm[kGpPlans];  // plan CTA: groups (-1 bad) and hull size per record
    __shared__ uint64_t s_pu1[kGpPlans];             // ... and the mask of group 1
    __shared__ uint64_t s_pu[64];            // directions whose partners are found by position ...
    __shared__ unsigned long long s_pk[64];  // ... and their strides
    if (*(volatile uint32_t*)d.status) return;
    const int n = d.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned gen = 0;
    if (threadIdx.x == 0) {
        gen = ld_acquire(&w->bar_gen);
        s_phase = gen;
        s_spin = spin_limit;
        s_trace = trace;
        s_gen0 = gen;
        s_tstart = trace ? gtimer() : 0;
        s_code = 0;
    }
    if (threadIdx.x < 64) {
        const int i = threadIdx.x;
        s_hc[i] = hull_state == 2 ? (i < n ? 1ull << i : 0ull) : (hull_state == 1 ? __ldcg(&w->hull[i]) : 0ull);
        // nothing known: every unit vector may be a direction of the hull
        s_hb[i] = hull_state == 1 ? __ldcg(&w->hbasis[i]) : (hull_state == 0 && i < n ? 1ull << i : 0ull);
        if (i == 0) s_nhb = hull_state == 1 ? (int)__ldcg(&w->nhb) : (hull_state == 0 ? n : 0);
    }
    for (int row = threadIdx.x; row < n; row += blockDim.x) {
        s_tab.mx[row] = __ldcg(&d.mx[row]);
        s_tab.mz[row] = __ldcg(&d.mz[row]);
        s_tab.dx[row] = __ldcg(&d.dx[row]);
        s_tab.dz[row] = __ldcg(&d.dz[row]);
        s_tab.de[row] = __ldcg(&d.de[row]);
        s_tab.piv[row] = __ldcg(&d.piv[row]);
    }
    if (threadIdx.x == 0) {
        s_tab.rx = __ldcg(&d.meta[0]);
        s_tab.g = __ldcg(d.g);
    }
    __syncthreads();
    if (gp_piped() && blockIdx.x >= gridDim.x - 2) {
        // ---- the planning CTAs.  The Clifford runs, their maps and the plans of
        // the diagonal records depend on the tableau alone, never on the frame,
        // so they run ahead of the workers while those run the passes of earlier
        // steps: the tableau CTA applies the Clifford runs (the only chain from
        // step to step), the plan CTA plans each step's records from the
        // tableau it is handed.  Every wait is bounded and ends early when a
        // worker has failed.
        const unsigned nw = gp_nwork();
        const unsigned long long lim = 64ull * spin_limit;
        const int nwarps = (int)(blockDim.x >> 5);
        // thread 0 polls *p until it reads v (eq) or anything but v (!eq)
        auto wait_u32 = [&](const unsigned* p, unsigned v) -> bool {
            if (threadIdx.x == 0) {
                unsigned long long spins = 0;
                int okw = 1;
                while (ld_acquire(p) != v) {
                    if (*(volatile uint32_t*)d.status || ++spins > lim) {
                        okw = 0;
                        break;
                    }
                    __nanosleep(100);
                }
                s_uni = okw;
            }
            __syncthreads();
            return s_uni != 0;
        };
        if (blockIdx.x == gridDim.x - 2) {
            // ---- tableau CTA
            if (!wait_u32(&w->checked, 1u)) return;  // the records passed the check
            unsigned long long poi = 0;
            unsigned tset = 0;
            int tk = 0;
            for (;;) {
                bool cliff = false, stop = poi >= n_ops;
                if (!stop) {
                    const uint32_t kind = ops[poi].kind;
                    cliff = kind <= 8;
                    stop = !cliff && !(kind >= SF_OP_DIAG && kind <= SF_OP_DIAG + 3);
                }
                const unsigned e = tset % kGpRing;
                if (tset >= kGpRing && !wait_u32(&w->tring_readers[e], 1u)) return;
                gp_pmark(w, tset, 0);
                GpTabSet* T = &w->tring[e];
                int np = 0;
                unsigned long long oe = poi, ds = poi;
                if (stop) {
                    tk = 3;
                } else if (cliff) {
                    if (warp == 0) {
                        const unsigned long long o =
                            gp_clifford_run(s_tab, ops, poi, n_ops, n, stage, s_cst, s_at, s_ainv, &s_t);
                        if (lane == 0) s_oe = o;
                    }
                    __syncthreads();
                    oe = s_oe;
                    if (oe == ~0ull) {
                        tk = 2;
                    } else {
                        tk = 0;
                        ds = oe;
                        np = diag_count(ops, oe, n_ops);
                    }
                } else {
                    tk = 1;
                    np = diag_count(ops, poi, n_ops);
                }
                {
                    const uint64_t* src = reinterpret_cast<const uint64_t*>(&s_tab);
                    uint64_t* dst = reinterpret_cast<uint64_t*>(&T->tab);
                    for (int i = threadIdx.x; i < (int)(sizeof(GpTab) / 8); i += blockDim.x) dst[i] = src[i];
                    if (threadIdx.x < 64) {
                        T->at[threadIdx.x] = s_at[threadIdx.x];
                        T->ainv[threadIdx.x] = s_ainv[threadIdx.x];
                    }
                    if (threadIdx.x == 0) {
                        T->t = s_t;
                        T->kind = tk;
                        T->np = np;
                        T->oe = oe;
                        T->ds = ds;
                    }
                }
                __threadfence();
                __syncthreads();
                if (threadIdx.x == 0) {
                    w->tring_readers[e] = 0;
                    __threadfence();
                    st_release64(&w->tring_seq[e], (unsigned long long)tset + 1ull);
                }
                gp_pmark(w, tset, 1);
                tset++;
                if (tk >= 2) break;
                poi = ds + np;
            }
            return;
        }
        // ---- plan CTA
        unsigned pset = 0;
        for (;;) {
            const unsigned te = pset % kGpRing;
            if (threadIdx.x == 0) {  // the tableau CTA's step pset
                unsigned long long spins = 0;
                int okw = 1;
                while (ld_acquire64(&w->tring_seq[te]) != (unsigned long long)pset + 1ull) {
                    if (*(volatile uint32_t*)d.status || ++spins > lim) {
                        okw = 0;
                        break;
                    }
                    __nanosleep(64);
                }
                s_uni = okw;
            }
            __syncthreads();
            if (!s_uni) return;
            gp_pmark(w, pset, 2);
            const GpTabSet* T = &w->tring[te];
            {
                const uint64_t* src = reinterpret_cast<const uint64_t*>(&T->tab);
                uint64_t* dst = reinterpret_cast<uint64_t*>(&s_tab);
                for (int i = threadIdx.x; i < (int)(sizeof(GpTab) / 8); i += blockDim.x) dst[i] = __ldcg(&src[i]);
                if (threadIdx.x < 64) {
                    s_at[threadIdx.x] = __ldcg(&T->at[threadIdx.x]);
                    s_ainv[threadIdx.x] = __ldcg(&T->ainv[threadIdx.x]);
                }
            }
            const int tk = __ldcg(&T->kind), np = __ldcg(&T->np);
            const unsigned long long oe = __ldcg(&T->oe), ds = __ldcg(&T->ds);
            if (threadIdx.x == 0) s_t = __ldcg(&T->t);
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(&w->tring_readers[te], 1u);
            gp_pmark(w, pset, 3);
            if (tk == 3) return;  // the workers stop at the same record
            const unsigned e = pset % kGpRing;
            if (pset >= kGpRing && !wait_u32(&w->ring_readers[e], nw)) return;
            GpSet* S = &w->ring[e];
            if (tk < 2) {
                for (int r = warp; r < np; r += nwarps) gp_plan(s_tab, n, ops[ds + r], &trig[4 * (ds + r)], spl[r]);
                __syncthreads();
            }
            gp_pmark(w, pset, 4);
            if (tk == 0) {
                // the hull moves with the run's map, as in the workers
                const int i = threadIdx.x;
                uint64_t hc = 0, hb = 0;
                if (i < 64) {
                    const uint64_t c = s_hc[i];
                    for (int h = 0; h < n; h++)
                        if ((c >> h) & 1) hc ^= s_ainv[h];
                    if (i < s_nhb) {
                        const uint64_t u = s_hb[i];
                        for (int j = 0; j < n; j++)
                            if ((u >> j) & 1) hb ^= s_at[j];
                    }
                }
                __syncthreads();
                if (i < 64) {
                    s_hc[i] = hc;
                    if (i < s_nhb) s_hb[i] = hb;
                }
                __syncthreads();
            }
            if (tk < 2) {
                // what the scans below read of each plan, one thread per record
                for (int r = threadIdx.x; r < np; r += blockDim.x) {
                    s_png[r] = spl[r].P.bad ? -1 : spl[r].P.ng;
                    s_pu1[r] = spl[r].P.u[1];
                }
                __syncthreads();
                // the run a fresh branch at record r would take: the records after
                // it with one group or the same mask
                for (int r = threadIdx.x; r < np; r += blockDim.x) {
                    const uint64_t u = s_pu1[r];
                    int t2 = r + 1;
                    while (t2 < np && (s_png[t2] == 1 || (s_png[t2] == 2 && s_pu1[t2] == u))) t2++;
                    spl[r].rend = t2;
                }
            }
            gp_pmark(w, pset, 5);
            if (tk < 2 && warp == 0) {
                // Per record: are its terms orthogonal to the hull where the workers
                // apply it?  The hull is followed record by record as the workers
                // change theirs -- a fresh direction joins after its whole run (the
                // records that follow with one group or the same mask are checked
                // against the hull before it), a merge's masks join after it -- except
                // that it always grows where the workers skip a direction whose
                // children all vanished, so it contains theirs and a yes is safe.
                // Directions are only appended within a batch, so the walk records
                // for each record how many of them it is checked against (lane 0
                // keeps the count), and the checks then run on every warp.
                // the constraints stay in registers for the walk (lane i: i, i + 32)
                // and the direction count in lane 0's register
                uint64_t c0 = s_hc[lane], c1 = s_hc[lane + 32];
                int nhb = s_nhb;
                uint64_t pend = 0;
                bool have_pend = false;
                for (int r = 0; r < np; r++) {
                    const int ng = s_png[r];
                    const uint64_t u1 = s_pu1[r];
                    const bool cont = have_pend && (ng == 1 || (ng == 2 && u1 == pend));
                    if (!cont && have_pend) {
                        if (hull_fresh_r(c0, c1, pend)) {
                            hull_add_r(c0, c1, pend);
                            if (lane == 0 && nhb < 64) s_hb[nhb] = pend;
                            nhb += nhb < 64;
                        }
                        have_pend = false;
                    }
                    if (lane == 0) s_pm[r] = nhb;  // directions the record is checked against
                    if (cont) continue;
                    if (ng == 2 && hull_fresh_r(c0, c1, u1)) {
                        pend = u1;
                        have_pend = true;
                    } else {
                        for (int g = 1; g < ng; g++) {
                            const uint64_t ug = spl[r].P.u[g];
                            if (hull_fresh_r(c0, c1, ug)) {
                                hull_add_r(c0, c1, ug);
                                if (lane == 0 && nhb < 64) s_hb[nhb] = ug;
                                nhb += nhb < 64;
                            }
                        }
                    }
                }
                if (have_pend && hull_fresh_r(c0, c1, pend)) {
                    hull_add_r(c0, c1, pend);
                    if (lane == 0 && nhb < 64) s_hb[nhb] = pend;
                    nhb += nhb < 64;
                }
                s_hc[lane] = c0;
                s_hc[lane + 32] = c1;
                if (lane == 0) s_nhb = nhb;
                __syncwarp();
            }
            __syncthreads();
            if (tk < 2) {
                // the verdicts, one record per warp and one hull direction per
                // lane (the walk above fixed how many directions each record is
                // checked against): a term fails when its parity with some
                // direction is odd
                for (int r = warp; r < np; r += nwarps) {
                    const BrTab& Q = spl[r].P;
                    const int ng = Q.ng, m = s_pm[r];
                    unsigned acc = 0;  // bit 4 g + t: term t of group g has odd parity with a direction
                    for (int i = lane; i < m; i += 32) {
                        const uint64_t h = s_hb[i];
#pragma unroll
                        for (int g = 0; g < 4; g++) {
                            const int nt = g < ng ? Q.nt[g] : 0;
#pragma unroll
                            for (int t = 0; t < 4; t++)
                                if (t < nt) acc |= (unsigned)(__popcll(Q.v[g][t] & h) & 1) << (4 * g + t);
                        }
                    }
                    acc = __reduce_or_sync(SF_FULL, acc);
                    if (lane == 0) spl[r].orth = acc == 0;
                }
            }
            __syncthreads();
            gp_pmark(w, pset, 6);
            {
                const uint64_t* src = reinterpret_cast<const uint64_t*>(&spl[0]);
                uint64_t* dst = reinterpret_cast<uint64_t*>(&S->plans[0]);
                const int words = (tk < 2 ? np : 0) * (int)(sizeof(GpPlan) / 8);
                for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
                const uint64_t* tsrc = reinterpret_cast<const uint64_t*>(&s_tab);
                uint64_t* tdst = reinterpret_cast<uint64_t*>(&S->tab);
                for (int i = threadIdx.x; i < (int)(sizeof(GpTab) / 8); i += blockDim.x) tdst[i] = tsrc[i];
                if (threadIdx.x < 64) {
                    S->at[threadIdx.x] = s_at[threadIdx.x];
                    S->ainv[threadIdx.x] = s_ainv[threadIdx.x];
                }
                if (threadIdx.x == 0) {
                    S->t = s_t;
                    S->kind = tk;
                    S->np = np;
                    S->oe = oe;
                }
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                w->ring_readers[e] = 0;
                __threadfence();
                st_release64(&w->ring_seq[e], (unsigned long long)pset + 1ull);
            }
            gp_pmark(w, pset, 7);
            pset++;
            if (tk == 2) return;
        }
    }
    // every record is checked before anything is touched
    {
        bool bad = false;
        for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_ops;
             i += (unsigned long long)gp_nwork() * blockDim.x) {
            const OpRec o = ops[i];
            const uint32_t k = o.kind == SF_OP_COND ? o.arg : o.kind;
            const bool two = (k >= 6 && k <= 8) || k == SF_OP_DIAG + 3;
            bool ok = o.q0 < (uint32_t)n && (!two || (o.q1 < (uint32_t)n && o.q1 != o.q0));
            if (o.kind == SF_OP_COND) ok &= o.arg <= 8;
            else ok &= k <= 8 || (k >= SF_OP_DIAG && k <= SF_OP_DIAG + 3) || k == SF_OP_MEASURE;
            bad |= !ok;
            // the term coefficients of every diagonal record (from e^{i theta}),
            // computed once here, spread over the grid (the double-precision
            // pipe of one SM is narrow, and the plans are the planner's pace)
            if (ok && o.kind >= SF_OP_DIAG && o.kind <= SF_OP_DIAG + 3) {
                const uint32_t kd = o.kind - SF_OP_DIAG;
                const double th = kd == 0 ? 0.78539816339744830962 : (kd == 1 ? -0.78539816339744830962 : o.param);
                double sn, cs;
                sincos(th, &sn, &cs);
                const SfTerms Tm = diag_terms(kd, cs, sn);
#pragma unroll
                for (int j = 0; j < 4; j++) trig[4 * i + j] = Tm.c[j];
            }
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) {
            set_status(d.status, 1u, cur0, 42u);  // SF_EINVAL: bad record
            gp_fail(w);
        }
        gp_phase(10, n_ops);
        if (!gp_barrier(w, gen, d.status, cur0)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) st_release32(&w->checked, 1u);
    }
    int cur = cur0;
    const bool piped = gp_piped();  // the planning CTAs plan ahead (the workers take their steps)
    unsigned long long k = d.kcnt[cur0];
    const unsigned long long k_init = k;
    if (blockIdx.x == 0 && threadIdx.x == 0) w->lay.ok = 0;  // written again at a normal end
    uint32_t tag[2] = {d.itag[0], d.itag[1]};
    unsigned long long isz[2] = {d.isize[0], d.isize[1]};
    bool ivalid[2] = {false, false};  // the index of buffer b describes its current contents
    ivalid[cur0] = idx_ok0 != 0;
    unsigned long long oi = 0;
    unsigned nmerge = 0, nfresh = 0;
    int npos = 0;         // entries of s_pu / s_pk
    bool ok = true;
    bool have_u = false;  // the frame is closed under the mask cu (s in F => s ^ cu in F)
    uint64_t cu = 0;
    unsigned npre = 0;    // records at oi planned by the last Clifford phase
    // The last Clifford run's map sigma' = A sigma ^ t is not yet applied to the
    // phase vectors (the tableau is already new); the next pass over the
    // elements applies it.  The hull and the positional directions are kept in
    // the new coordinates from the Clifford phase on.
    bool aff = false;
    const int nc = (n + 3) >> 2;
    uint64_t tw = 0;
    // element bytes of a pass (phase vector 8 B, amplitude 16 B), counted once
    auto account = [&](unsigned long long bytes) {
        if (blockIdx.x == 0 && threadIdx.x == 0) w->moved += bytes;
    };
    // 4-bit lookup tables of the pending map (columns of A from the workspace)
    auto affine_tables = [&]() {
        for (int e = threadIdx.x; e < nc * 16; e += blockDim.x) {
            const int v = e & 15, c = e >> 4;
            uint64_t acc = 0;
#pragma unroll
            for (int b = 0; b < 4; b++)
                if (((v >> b) & 1) && 4 * c + b < n) acc ^= s_at[4 * c + b];
            tab[e] = acc;
        }
        tw = s_t;
        __syncthreads();
    };
    auto affine_of = [&](uint64_t x) {
        uint64_t o = tw;
        for (int c = 0; c < nc; c++) o ^= tab[c * 16 + ((x >> (4 * c)) & 15)];
        return o;
    };
    // the map applied to every phase vector in place (positions unchanged)
    auto affine_pass = [&]() {
        affine_tables();
        uint64_t* S = d.sig[cur];
        unsigned long long lo, hi;
        gp_chunk(k, lo, hi);
        for (unsigned long long j = lo + threadIdx.x; j < hi; j += blockDim.x) S[j] = affine_of(__ldcg(&S[j]));
        ivalid[cur] = false;
        aff = false;
        account(16 * k);
    };
    // the Clifford run's map moves the hull constraints (c -> A^-T c: the XOR of
    // the rows of A^-1 that c selects) and the positional directions (u -> A u)
    auto move_hull = [&]() {
        uint64_t hc = 0, pu = 0;
        const int i = threadIdx.x;
        if (i < 64) {
            const uint64_t c = s_hc[i];
            for (int h = 0; h < n; h++)
                if ((c >> h) & 1) hc ^= s_ainv[h];
            if (i < npos) {
                const uint64_t u = s_pu[i];
                for (int j = 0; j < n; j++)
                    if ((u >> j) & 1) pu ^= s_at[j];
            }
        }
        uint64_t hb = 0;
        if (i < s_nhb) {
            const uint64_t u = s_hb[i];
            for (int j = 0; j < n; j++)
                if ((u >> j) & 1) hb ^= s_at[j];
        }
        __syncthreads();
        if (i < 64) {
            s_hc[i] = hc;
            if (i < npos) s_pu[i] = pu;
            if (i < s_nhb) s_hb[i] = hb;
        }
        __syncthreads();
    };
    // the hull grows by u (warp 0; the caller synchronises the block): a new
    // direction joins the basis and removes one constraint
    auto hull_grow = [&](uint64_t u) {
        if (warp != 0) return;
        if (!hull_fresh(s_hc, u)) return;
        hull_add(s_hc, u);
        if (lane == 0 && s_nhb < 64) s_hb[s_nhb++] = u;
        __syncwarp();
    };
    // records [r0, r1) with frame-independent coefficients multiplied into
    // s_comp (runs of three records or more, frames of one element or more);
    // the pending map is applied to the reference phase vector when aff is set
    // (its tables built).  Every thread learns whether it worked.
    auto compose = [&](int r0, int r1, uint64_t u) {
        if (threadIdx.x == 0) {
            const uint64_t s = k ? __ldcg(&d.sig[cur][0]) : 0;
            s_ref = aff ? affine_of(s) : s;
        }
        __syncthreads();
        if (warp == 0) {
            const bool uni = k && r1 - r0 >= 3 && uniform_run(spl, r0, r1, s_hb, s_nhb, s_ref, u, piped, s_cm, &s_comp);
            if (lane == 0) s_uni = uni;
        }
        __syncthreads();
        return s_uni != 0;
    };
    // stride of a direction with positional partners, or 0
    auto pos_stride = [&](uint64_t u) {
        unsigned long long st = 0;
        for (int i = 0; i < npos; i++)
            if (s_pu[i] == u) st = s_pk[i];
        return st;
    };
    // the index of buffer b, built from its phase vectors as they are stored
    auto build_index = [&](int b) {
        const uint32_t tg = next_tag(tag[b]);
        const unsigned long long T = index_slots(k, d.icap);
        unsigned long long lo, hi;
        gp_chunk(k, lo, hi);
        for (unsigned long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
            const uint64_t s = __ldcg(&d.sig[b][j]);
            ok &= index_insert<1>(d, b, T, tg, &s, (uint32_t)j);
        }
        tag[b] = tg;
        isz[b] = T;
        ivalid[b] = true;
        account(8 * k);
        gp_phase(7, k);
        if (!ok) {
            set_status(d.status, SF_ST_TIMEOUT, b, 43u);  // index full
            gp_fail(w);
        }
        return gp_barrier(w, gen, d.status, b);
    };
    // the elements of positions [0, m) of buffer cur with |a| >= eps, compacted
    // into the other buffer (order of the reservations)
    auto compact = [&](unsigned long long m, bool& moved) {
        const int in = cur, out = cur ^ 1;
        unsigned long long* ctr = &w->ocnt[nmerge % 3];
        if (blockIdx.x == 0 && threadIdx.x == 0) w->ocnt[(nmerge + 1) % 3] = 0;
        const unsigned long long kb = keep_bits(eps2);
        unsigned long long lo, hi;
        gp_chunk(m, lo, hi);
        for (unsigned long long base = lo; base < hi; base += blockDim.x) {
            const unsigned long long j = base + threadIdx.x;
            const bool act = j < hi;
            uint64_t s0 = 0;
            double2 a = make_double2(0.0, 0.0);
            if (act) {
                s0 = __ldcg(&d.sig[in][j]);
                a = __ldcg(&d.amp[in][j]);
            }
            const bool keep = act && amp_kept(a, kb, eps2);
            const unsigned long long o = block_out_range(ctr, keep ? 1u : 0u, wsum, &bbase);
            if (keep) {
                d.sig[out][o] = s0;
                d.amp[out][o] = a;
            }
        }
        gp_phase(6, m);
        moved = gp_barrier(w, gen, d.status, in);
        k = __ldcg(ctr);
        account(24 * (m + k));
        cur = out;
        ivalid[out] = false;
        nmerge++;
        have_u = false;
        npos = 0;
    };
    // on a failed check: the frame stays in buffer cur (its count and the
    // index tags go back for the host's error path), and the launch ends
    // the tableau of the launch back to the handle (CTA 0)
    auto store_tableau = [&]() {
        if (blockIdx.x != 0) return;
        for (int row = threadIdx.x; row < n; row += blockDim.x) {
            d.mx[row] = s_tab.mx[row];
            d.mz[row] = s_tab.mz[row];
            d.dx[row] = s_tab.dx[row];
            d.dz[row] = s_tab.dz[row];
            d.de[row] = s_tab.de[row];
            d.piv[row] = s_tab.piv[row];
        }
        if (threadIdx.x == 0) {
            d.meta[0] = s_tab.rx;
            *d.g = s_tab.g;
        }
    };
    auto bail = [&]() {
        store_tableau();
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            d.kcnt[cur] = k;
            for (int b = 0; b < 2; b++) {
                d.itag[b] = ivalid[b] ? tag[b] : next_tag(tag[b]);
                d.isize[b] = isz[b];
            }
        }
    };
    // the next planned step from the ring (workers, when the grid has a planner
    // CTA): the tableau after its Clifford run, the run's map and the plans of
    // its diagonal records, copied into this CTA's shared memory through L2
    unsigned nset = 0;
    auto take_set = [&]() -> bool {
        const unsigned e = nset % kGpRing;
        if (threadIdx.x == 0) {
            unsigned long long spins = 0;
            int okw = 1;
            while (ld_acquire64(&w->ring_seq[e]) != (unsigned long long)nset + 1ull) {
                if (*(volatile uint32_t*)d.status || ++spins > s_spin) {
                    okw = 0;
                    break;
                }
                __nanosleep(64);
            }
            s_take = okw;
        }
        __syncthreads();
        if (!s_take) return false;
        const GpSet* S = &w->ring[e];
        {
            const uint64_t* src = reinterpret_cast<const uint64_t*>(&S->tab);
            uint64_t* dst = reinterpret_cast<uint64_t*>(&s_tab);
            for (int i = threadIdx.x; i < (int)(sizeof(GpTab) / 8); i += blockDim.x) dst[i] = __ldcg(&src[i]);
        }
        if (threadIdx.x < 64) {
            s_at[threadIdx.x] = __ldcg(&S->at[threadIdx.x]);
            s_ainv[threadIdx.x] = __ldcg(&S->ainv[threadIdx.x]);
        }
        const int np = __ldcg(&S->np);
        if (threadIdx.x == 0) {
            s_t = __ldcg(&S->t);
            s_kind = __ldcg(&S->kind);
            s_np = np;
            s_oe = __ldcg(&S->oe);
        }
        {
            const uint64_t* src = reinterpret_cast<const uint64_t*>(&S->plans[0]);
            uint64_t* dst = reinterpret_cast<uint64_t*>(&spl[0]);
            const int words = np * (int)(sizeof(GpPlan) / 8);
            for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldcg(&src[i]);
        }
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&w->ring_readers[e], 1u);
        nset++;
        return true;
    };
    // a wait for the planner that ran out: every worker stops at the next barrier
    auto set_timeout = [&]() {
        if (threadIdx.x == 0) {
            set_status(d.status, SF_ST_TIMEOUT, cur, 51u);
            gp_fail(w);
        }
        gp_barrier(w, gen, d.status, cur);
        if (aff) affine_pass();
        bail();
    };
    while (oi < n_ops) {
        const uint32_t kind = ops[oi].kind;
        if (kind <= 8) {
            // ---- Clifford run: every CTA applies it to its own tableau (one warp),
            // then inverts the map (that warp) while its other warps plan the
            // diagonal records that follow; no grid barrier, no global traffic
            gp_mark(w, 0);
            if (piped) {
                // the planner CTA ran the Clifford run and planned what follows
                if (!take_set()) return set_timeout();
                gp_mark(w, 1);
                if (s_kind >= 2) {  // a tableau check failed
                    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, cur, 41u);
                    if (aff) affine_pass();
                    return bail();
                }
                npre = (unsigned)s_np;
                have_u = false;
                oi = s_oe;
                aff = true;
                move_hull();
                gp_mark(w, 3);
                continue;
            }
            if (warp == 0) {
                const unsigned long long oe = gp_clifford_run(s_tab, ops, oi, n_ops, n, stage, s_cst, s_at, s_ainv, &s_t);
                if (lane == 0) s_oe = oe;
            }
            __syncthreads();
            gp_mark(w, 1);
            const unsigned long long oe = s_oe;
            if (oe == ~0ull) {  // a tableau check failed (in every CTA alike)
                if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, cur, 41u);
                return bail();
            }
            const int np = diag_count(ops, oe, n_ops);
            for (int r = warp; r < np; r += (int)(blockDim.x >> 5))
                gp_plan(s_tab, n, ops[oe + r], &trig[4 * (oe + r)], spl[r]);
            __syncthreads();
            gp_mark(w, 2);
            npre = (unsigned)np;
            have_u = false;
            oi = oe;
            aff = true;
            move_hull();
            gp_mark(w, 3);
            continue;
        }
        if (kind < SF_OP_DIAG || kind > SF_OP_DIAG + 3) break;  // measurement or conditional gate
        // ---- diagonal run: all plans first (unless the Clifford phase made them),
        // then the records in passes over the frame
        int nb = (int)npre;
        npre = 0;
        if (nb == 0) {  // plans of a diagonal run without a Clifford run before it
            if (piped) {
                if (!take_set()) return set_timeout();
                nb = s_np;
            } else {  // the one CTA plans it, one warp per record
                nb = diag_count(ops, oi, n_ops);
                for (int r = warp; r < nb; r += (int)(blockDim.x >> 5))
                    gp_plan(s_tab, n, ops[oi + r], &trig[4 * (oi + r)], spl[r]);
                __syncthreads();
            }
        }
        int t = 0;
        while (t < nb) {
            const BrTab& P0 = spl[t].P;  // the plan in the tableau's coordinates
            const int ng = P0.ng;
            if (P0.bad) {
                if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, cur, 44u);
                if (aff) affine_pass();  // the frame must match the tableau when the launch ends
                return bail();
            }
            const unsigned long long kb = keep_bits(eps2);
            // ---- a branch along a direction outside the hull: no element has a
            // partner, so each writes its two children in place (s at j, s ^ u at
            // j + k); the following records that keep every pair are applied to it
            // in the same pass
            if (ng == 2 && hull_fresh(s_hc, P0.u[1])) {
                const uint64_t u = P0.u[1];
                int t2 = t + 1;
                if (piped) {
                    t2 = spl[t].rend;  // the plan CTA found it
                } else {
                    while (t2 < nb && !spl[t2].P.bad &&
                           (spl[t2].P.ng == 1 || (spl[t2].P.ng == 2 && spl[t2].P.u[1] == u)))
                        t2++;
                }
                if (2 * k > d.cap) {
                    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_CAPACITY, cur, 0u);
                    if (aff) affine_pass();
                    return bail();
                }
                gp_mark(w, 4);
                if (aff) affine_tables();
                const bool uni = compose(t, t2, u);
                const Cm2 cm = s_comp;
                gp_mark(w, 5);
                unsigned long long* fk = w->fk[nfresh % 3];
                if (blockIdx.x == 0 && threadIdx.x == 0) w->fk[(nfresh + 1) % 3][0] = w->fk[(nfresh + 1) % 3][1] = 0;
                uint64_t* S = d.sig[cur];
                double2* A = d.amp[cur];
                unsigned long long lo, hi;
                gp_chunk(k, lo, hi);
                unsigned c0 = 0, c1 = 0;
                for (unsigned long long base = lo; base < hi; base += blockDim.x) {
                    const unsigned long long j = base + threadIdx.x;
                    if (j < hi) {
                        const uint64_t s = __ldcg(&S[j]);
                        double2 a0 = __ldcg(&A[j]), a1 = make_double2(0.0, 0.0);
                        const uint64_t s0 = aff ? affine_of(s) : s, s1 = s0 ^ u;
                        if (uni) {
                            a1 = cprod(cm.m10, a0);
                            a0 = cprod(cm.m00, a0);
                        } else {
                            for (int r = t; r < t2; r++) pair_step<true>(spl[r], s0, s1, a0, a1);
                        }
                        S[j] = s0;
                        A[j] = a0;
                        S[j + k] = s1;
                        A[j + k] = a1;
                        c0 += amp_kept(a0, kb, eps2);
                        c1 += amp_kept(a1, kb, eps2);
                    }
                }
                gp_mark(w, 6);
                add_counts(fk, c0, c1);
                gp_phase(3 | ((t2 - t) << 4), k);
                if (!gp_barrier(w, gen, d.status, cur)) return bail();
                const unsigned long long K0 = __ldcg(&fk[0]), K1 = __ldcg(&fk[1]);
                gp_mark(w, 7);
                account(72 * k);
                aff = false;
                nfresh++;
                ivalid[cur] = false;
                t = t2;
                if (K0 == k && K1 == k) {  // every child kept: the frame doubles
                    hull_grow(u);
                    if (threadIdx.x == 0 && npos < 64) {
                        s_pu[npos] = u;
                        s_pk[npos] = k;
                    }
                    npos = npos < 64 ? npos + 1 : npos;
                    __syncthreads();
                    k *= 2;
                    have_u = true;
                    cu = u;
                } else if (K0 == k && K1 == 0) {  // the mask's children all vanished: same positions
                    have_u = false;
                } else {
                    hull_grow(u);
                    __syncthreads();
                    bool moved = true;
                    compact(2 * k, moved);
                    if (!moved) return bail();
                }
                continue;
            }
            // ---- in-place run: one-group records (a phase per element) and two-group
            // records whose mask the frame is closed under (each pair {s, s ^ u} maps
            // onto itself); phase vectors and positions stay
            int t2 = t;
            bool pairs = false;
            uint64_t pu = 0;
            while (t2 < nb && !spl[t2].P.bad) {
                const BrTab& Q = spl[t2].P;
                if (Q.ng == 1) {
                    t2++;
                } else if (Q.ng == 2 && (pairs ? Q.u[1] == pu
                                               : ((have_u && Q.u[1] == cu) || pos_stride(Q.u[1]) != 0))) {
                    pairs = true;
                    pu = Q.u[1];
                    t2++;
                } else {
                    break;
                }
            }
            if (t2 > t) {
                const unsigned long long st = pairs ? pos_stride(pu) : 0;
                bool drop = false, miss = false;
                if (st && k % (2 * st)) {  // positions no longer pair up: a bookkeeping fault
                    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_INTERNAL, cur, 50u);
                    if (aff) affine_pass();
                    return bail();
                }
                const bool wrote_sig = aff && (!pairs || st);
                if (!pairs || st) {
                    // partners by position (or none): the pending map is applied on the way
                    if (aff) affine_tables();
                    const bool uni = compose(t, t2, pairs ? pu : 0);
                    const Cm2 cm = s_comp;
                    uint64_t* S = d.sig[cur];
                    double2* A = d.amp[cur];
                    const unsigned long long items = pairs ? k / 2 : k;
                    unsigned long long lo, hi;
                    gp_chunk(items, lo, hi);
                    for (unsigned long long m = lo + threadIdx.x; m < hi; m += blockDim.x) {
                        unsigned long long p0 = m, p1 = 0;
                        if (pairs) {
                            const unsigned long long b = m / st;
                            p0 = m + b * st;  // 2 b st + (m - b st)
                            p1 = p0 + st;
                        }
                        uint64_t s0 = __ldcg(&S[p0]);
                        uint64_t s1 = pairs ? __ldcg(&S[p1]) : 0;
                        if (aff) {
                            s0 = affine_of(s0);
                            if (pairs) s1 = affine_of(s1);
                        }
                        if (pairs && s1 != (s0 ^ pu)) {
                            miss = true;
                            continue;
                        }
                        double2 a0 = __ldcg(&A[p0]);
                        double2 a1 = pairs ? __ldcg(&A[p1]) : make_double2(0.0, 0.0);
                        if (uni) {
                            const double2 b0 = cfma(cm.m01, a1, cprod(cm.m00, a0));
                            a1 = cfma(cm.m11, a1, cprod(cm.m10, a0));
                            a0 = b0;
                        } else if (pairs) {
                            for (int r = t; r < t2; r++) pair_step<true>(spl[r], s0, s1, a0, a1);
                        } else {
                            for (int r = t; r < t2; r++) pair_step<false>(spl[r], s0, s1, a0, a1);
                        }
                        if (aff) S[p0] = s0;
                        A[p0] = a0;
                        drop |= !amp_kept(a0, kb, eps2);
                        if (pairs) {
                            if (aff) S[p1] = s1;
                            A[p1] = a1;
                            drop |= !amp_kept(a1, kb, eps2);
                        }
                    }
                    if (aff) {
                        ivalid[cur] = false;
                        aff = false;
                    }
                } else {
                    // partners through the index (the frame was closed under pu by a merge,
                    // which left its index; no map is pending then)
                    if (aff) {
                        affine_pass();
                        gp_phase(8, k);
                        if (!gp_barrier(w, gen, d.status, cur)) return bail();
                    }
                    if (!ivalid[cur] && !build_index(cur)) return bail();
                    const uint64_t* S = d.sig[cur];
                    double2* A = d.amp[cur];
                    unsigned long long lo, hi;
                    gp_chunk(k, lo, hi);
                    const auto plan = [&](int r) { return PlanRef{&spl[r].P, spl[r].ctab}; };
                    const int c_ = cur;
                    const auto find = [&](uint64_t key) { return gp_find(d, c_, isz[c_], tag[c_], key); };
                    for (unsigned long long base = lo + 64ull * warp; base < hi; base += 64ull * (blockDim.x >> 5))
                        inplace_run_warp<true>(S, A, base, hi, true, pu, t, t2, plan, find, kb, eps2, drop, miss);
                }
                if (miss) {  // the frame is not closed after all
                    set_status(d.status, SF_ST_INTERNAL, cur, 47u);
                    gp_fail(w);
                }
                if (__syncthreads_or(drop) && threadIdx.x == 0) gp_dropped(w);
                gp_phase(4 | ((t2 - t) << 4), k);
                if (!gp_barrier(w, gen, d.status, cur)) return bail();
                account(40 * k + (wrote_sig ? 8 * k : 0));
                t = t2;
                if (!s_drop) continue;
                // ---- amplitudes fell below the threshold: compact the frame
                bool moved = true;
                compact(k, moved);
                if (!moved) return bail();
                continue;
            }
            // ---- merge of record t into the other buffer through the input's index
            if ((unsigned long long)ng * k > d.cap) {
                if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.status, SF_ST_CAPACITY, cur, 0u);
                if (aff) affine_pass();
                return bail();
            }
            if (!ivalid[cur] && !build_index(cur)) return bail();
            if (aff) {
                // the phase vectors are still those before the map sigma' = A sigma ^ t:
                // partners at A^-1 u, sign patterns from A^T v flipped by parity(v & t);
                // outputs are written in the new coordinates
                affine_tables();
                {
                    const uint64_t* src = reinterpret_cast<const uint64_t*>(&P0);
                    uint64_t* dst = reinterpret_cast<uint64_t*>(&pm);
                    for (int i = threadIdx.x; i < (int)(sizeof(BrTab) / 8); i += blockDim.x) dst[i] = src[i];
                }
                __syncthreads();
                const int tid = threadIdx.x;
                if (tid < ng) {  // u'_g = A^-1 u_g
                    uint64_t x = 0;
                    for (int i = 0; i < n; i++) x |= (uint64_t)(__popcll(s_ainv[i] & P0.u[tid]) & 1) << i;
                    pm.u[tid] = x;
                } else if (tid >= 32 && tid < 48) {  // v' = A^T v
                    const int g = (tid - 32) >> 2, tt = (tid - 32) & 3;
                    if (g < ng && tt < P0.nt[g]) {
                        uint64_t x = 0;
                        for (int j = 0; j < n; j++) x |= (uint64_t)(__popcll(s_at[j] & P0.v[g][tt]) & 1) << j;
                        pm.v[g][tt] = x;
                    }
                } else if (tid >= 64 && tid < 64 + ng) {  // the pattern bits flipped by t
                    const int g = tid - 64;
                    int f = 0;
                    for (int tt = 0; tt < P0.nt[g]; tt++) f |= (__popcll(P0.v[g][tt] & tw) & 1) << tt;
                    pm.fl[g] = f;
                }
                __syncthreads();
            }
            const BrTab& P = aff ? pm : P0;  // the plan in the frame's coordinates
            const double2(*const ctab)[16] = spl[t].ctab;
            const int in = cur, out = cur ^ 1;
            const unsigned long long Tin = isz[in], Tout = index_slots((unsigned long long)ng * k, d.icap);
            const uint32_t tag_in = tag[in], tag_out = next_tag(tag[out]);
            unsigned long long* ctr = &w->ocnt[nmerge % 3];
            // the counter of the next merge was last read before the previous barrier
            if (blockIdx.x == 0 && threadIdx.x == 0) w->ocnt[(nmerge + 1) % 3] = 0;
            const uint64_t* Si = d.sig[in];
            const double2* Ai = d.amp[in];
            uint64_t* So = d.sig[out];
            double2* Ao = d.amp[out];
            unsigned long long lo, hi;
            gp_chunk(k, lo, hi);
            bool drop = false;
            for (unsigned long long base = lo; base < hi; base += blockDim.x) {
                const unsigned long long j = base + threadIdx.x;
                const bool act = j < hi;
                uint64_t s = 0;
                double2 a = make_double2(0.0, 0.0);
                // group loops unrolled with guards and id read through pick_grp,
                // so that id and amps stay in registers
                long long id[SF_BR_MAXG] = {act ? (long long)j : -1, -1, -1, -1};
                if (act) {
                    s = __ldcg(&Si[j]);
                    a = __ldcg(&Ai[j]);
                }
#pragma unroll
                for (int g = 1; g < SF_BR_MAXG; g++)
                    if (act && g < ng) id[g] = gp_find(d, in, Tin, tag_in, s ^ P.u[g]);
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
                            const long long im = pick_grp(id, m);
                            if (im < 0) continue;
                            const double2 ap = m == 0 ? a : __ldcg(&Ai[im]);
                            cmul_acc(amp, half_coef(P, ctab, g2, s ^ P.u[m]), ap);
                        }
                    }
                    amps[g] = amp;
                    if (own && amp_kept(amp, kb, eps2)) keepm |= 1u << g;
                    else if (own) drop = true;
                }
                unsigned long long o = block_out_range(ctr, __popc(keepm), wsum, &bbase);
                const uint64_t sn = aff && act ? affine_of(s) : s;  // the parent in the new coordinates
#pragma unroll
                for (int g = 0; g < SF_BR_MAXG; g++) {
                    if (!((keepm >> g) & 1u)) continue;
                    const uint64_t tau = sn ^ P0.u[g];
                    So[o] = tau;
                    Ao[o] = amps[g];
                    ok &= index_insert<1>(d, out, Tout, tag_out, &tau, (uint32_t)o);
                    o++;
                }
            }
            if (!ok) {
                set_status(d.status, SF_ST_TIMEOUT, in, 45u);  // index full
                gp_fail(w);
            }
            if (__syncthreads_or(drop) && threadIdx.x == 0) gp_dropped(w);
            for (int g = 1; g < ng; g++) hull_grow(P0.u[g]);  // directions new to the hull
            gp_phase(5, k);
            if (!gp_barrier(w, gen, d.status, in)) return bail();
            account(24 * k);
            k = __ldcg(ctr);
            account(24 * k);
            cur = out;
            tag[out] = tag_out;
            isz[out] = Tout;
            ivalid[out] = true;
            nmerge++;
            npos = 0;  // outputs sit where their reservations put them
            // no output dropped: every parent s gave s ^ u_g for all g, so the new
            // frame is closed under the gate's masks
            have_u = !s_drop && ng == 2;
            cu = P0.u[1];
            aff = false;
            t++;
        }
        oi += nb;
    }
    if (aff) {  // a Clifford run at the end of the program
        affine_pass();
        gp_phase(8, k);
        if (!gp_barrier(w, gen, d.status, cur)) return bail();
    }
    // the frame goes back to buffer cur0 (without an index)
    if (cur != cur0) {
        unsigned long long lo, hi;
        gp_chunk(k, lo, hi);
        for (unsigned long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
            d.sig[cur0][j] = __ldcg(&d.sig[cur][j]);
            d.amp[cur0][j] = __ldcg(&d.amp[cur][j]);
        }
        ivalid[cur0] = false;
        account(48 * k);
    }
    store_tableau();
    if (blockIdx.x == 0) {
        if (threadIdx.x < 64) w->lay.u[threadIdx.x] = threadIdx.x < npos ? s_pu[threadIdx.x] : 0ull;
        if (threadIdx.x < 64 && hull_state != 0) {
            w->hull[threadIdx.x] = s_hc[threadIdx.x];
            w->hbasis[threadIdx.x] = s_hb[threadIdx.x];
            if (threadIdx.x == 0) w->nhb = (unsigned)s_nhb;
        }
        if (threadIdx.x == 0) {
            d.kcnt[cur0] = k;
            for (int b = 0; b < 2; b++) {  // an index that went stale gets a tag it never had
                d.itag[b] = ivalid[b] ? tag[b] : next_tag(tag[b]);
                d.isize[b] = isz[b];
            }
            if (consumed) *consumed = oi;
            if (trace) w->ntrace = gen - s_gen0;
            // positions still enumerate the span of the doubling directions
            bool lay = k_init == 1 && npos < 64 && k == (1ull << npos);
            for (int i = 0; i < npos && lay; i++) lay = s_pk[i] == (1ull << i);
            w->lay.n = (unsigned)npos;
            w->lay.ok = lay ? 1u : 0u;
        }
    }
}

}  // namespace

size_t sf_gprog_work_words() { return (sizeof(GpWork) + 7) / 8; }

// clears the per-launch words of the workspace (stream-ordered)
cudaError_t sf_gprog_clear(const SfDev& d, cudaStream_t s) {
    GpWork* w = reinterpret_cast<GpWork*>(d.gp);
    return cudaMemsetAsync(&w->err[0], 0, offsetof(GpWork, cleared_end) - offsetof(GpWork, err), s);
}

// element bytes moved by the last launch (stream-ordered copy into *host)
cudaError_t sf_gprog_moved(const SfDev& d, unsigned long long* host, cudaStream_t s) {
    GpWork* w = reinterpret_cast<GpWork*>(d.gp);
    return cudaMemcpyAsync(host, &w->moved, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
}

// checkpoints inside the phases of the last traced launch (8 per phase)
cudaError_t sf_gprog_marks(const SfDev& d, uint64_t* host, unsigned m, cudaStream_t s) {
    GpWork* w = reinterpret_cast<GpWork*>(d.gp);
    m = std::min(m, (unsigned)kGpTrace);
    return m ? cudaMemcpyAsync(host, &w->marks[0][0], m * 8 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s)
             : cudaSuccess;
}

// the planning CTAs' checkpoints of the last traced launch (8 per step)
cudaError_t sf_gprog_plan_marks(const SfDev& d, uint64_t* host, unsigned m, cudaStream_t s) {
    GpWork* w = reinterpret_cast<GpWork*>(d.gp);
    m = std::min(m, (unsigned)kGpTrace);
    return m ? cudaMemcpyAsync(host, &w->pmarks[0][0], m * 8 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s)
             : cudaSuccess;
}

// the phase records of the last traced launch (stream-ordered copies)
cudaError_t sf_gprog_trace(const SfDev& d, uint64_t* host, unsigned cap, unsigned* n, cudaStream_t s) {
    GpWork* w = reinterpret_cast<GpWork*>(d.gp);
    cudaError_t e = cudaMemcpyAsync(n, &w->ntrace, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const unsigned m = std::min(std::min(*n, cap), (unsigned)kGpTrace);
    *n = m;
    return m ? cudaMemcpyAsync(host, &w->trace[0][0], m * 5 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s)
             : cudaSuccess;
}

// resets the barrier after a launch that gave up waiting
cudaError_t sf_gprog_reset(const SfDev& d, cudaStream_t s) {
    return cudaMemsetAsync(d.gp, 0, sizeof(GpWork), s);
}

cudaError_t sf_launch_gprog(const SfDev& d, const void* ops, unsigned long long n_ops, double eps2, int cur,
                            int idx_ok, int hull_state, unsigned spin_limit, int trace, double2* trig,
                            unsigned long long* consumed, cudaStream_t s) {
    static int grid = 0;  // one CTA per SM, all resident (checked once per process)
    if (grid == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_gprog, cudaFuncAttributeMaxDynamicSharedMemorySize, kGpPlans * sizeof(GpPlan));
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gprog, kGpThreads, kGpPlans * sizeof(GpPlan));
        if (e != cudaSuccess) return e;
        if (per < 1) return cudaErrorCooperativeLaunchTooLarge;
        grid = sms;
    }
    cudaError_t e = sf_gprog_clear(d, s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kGpThreads);
    cfg.dynamicSmemBytes = kGpPlans * sizeof(GpPlan);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_gprog, d, reinterpret_cast<GpWork*>(d.gp), reinterpret_cast<const OpRec*>(ops),
                              n_ops, eps2, cur, idx_ok, hull_state, spin_limit, trace, trig, consumed);
}
