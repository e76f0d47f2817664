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
//                  barrier.  The map itself is applied by the next merge
//                  (partners at A^-1 u, sign patterns from A^T v); any other
//                  follower gets a pass that rewrites and re-indexes the
//                  phase vectors first.
//   diagonal run   records not planned yet are planned at once, CTA c
//                  planning record c (Sec. IV: Z^w = eps D^u M^v per term,
//                  grouped by u, half table of group coefficients); barrier;
//                  then per record every CTA merges its share of the elements
//                  into the other buffer (owner rule, outputs reserved with one
//                  atomic per block, inserted into the output index); barrier.
//                  Once a merge drops nothing the frame is closed under its
//                  mask, and the following gates that keep it closed are
//                  applied in place to each pair's amplitudes in one pass.
//
// A measurement or conditional record ends the program (the caller continues
// per op).  Data written inside the launch by other CTAs is read through L2
// (ld.global.cg), never through the non-coherent or L1 paths.  Every barrier
// wait is bounded: on expiry the kernel sets SF_ST_TIMEOUT and returns.
#include "sf.h"
#include "sf_warp.cuh"

using namespace sfw;

namespace {

constexpr int kGpThreads = 512;
constexpr int kGpPlans = 32;              // diagonal records planned per batch
constexpr unsigned kGpSpinLimit = 1u << 20;  // barrier polls (100 ns apart) before giving up

struct GpPlan {
    BrTab P;
    double2 ctab[4][16];
};

// device workspace, zeroed at handle creation; err, drop and ocnt are
// cleared before every launch
struct GpWork {
    unsigned int bar_count, bar_gen;
    unsigned int err[3];         // a failed check in phase p (between barriers p and p + 1): err[p % 3]
    unsigned int drop[3];        // an amplitude dropped in phase p: drop[p % 3]
    unsigned long long ocnt[3];  // output counters of consecutive merges, rotating
    unsigned long long oe;       // end of the current Clifford run
    unsigned int npre;           // diagonal records after it already planned into plans[0 .. npre)
    uint64_t AT[64];             // affine map of the current Clifford run: column j = image of e_j
    uint64_t t;
    uint64_t Ainv[64];           // rows of the inverse of its linear part
    GpPlan plans[kGpPlans];
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__shared__ unsigned s_phase;  // phase of the grid program this CTA is in
__shared__ int s_drop;        // an amplitude was dropped in the phase that ended at the last barrier

// a failed check of this CTA: every CTA stops at the next barrier
__device__ __forceinline__ void gp_fail(GpWork* w) { atomicExch(&w->err[s_phase % 3], 1u); }
// an amplitude of this CTA fell below the drop threshold in this phase
__device__ __forceinline__ void gp_dropped(GpWork* w) { atomicExch(&w->drop[s_phase % 3], 1u); }

// Grid barrier: every CTA passes the same sequence of barriers.  Thread 0
// arrives with one atomic; the last arrival resets the count and bumps the
// generation, the others poll it with a bound.  Returns false in every
// thread of every CTA if a check failed in the phase that ends here, and in
// the CTA whose wait ran out.  The error word of a phase is cleared two
// phases ahead, once every CTA has read it.
__device__ bool gp_barrier(GpWork* w, unsigned& gen, uint32_t* status, int buf) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned g = gen;
        int ok = 1;
        if (atomicAdd(&w->bar_count, 1u) == gridDim.x - 1) {
            w->bar_count = 0;
            __threadfence();
            atomicExch(&w->bar_gen, g + 1);
        } else {
            unsigned spins = 0;
            while (ld_acquire(&w->bar_gen) == g) {
                if (++spins > kGpSpinLimit) {
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        if (!ok) set_status(status, SF_ST_TIMEOUT, buf, 40u);
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

// ROTATE over the run of Clifford records from oi (warp 0 of CTA 0): the
// tableau in registers, written back with the X-block size and global phase;
// the composed affine map goes to the workspace, the run's end to w->oe.
__device__ void gp_clifford_run(const SfDev& d, GpWork* w, const OpRec* ops, unsigned long long oi,
                                unsigned long long o1, Row* stage, uint64_t* arows, int buf) {
    const int n = d.n, lane = threadIdx.x & 31;
    Row r[2];
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        const bool in = row < n;
        r[hf].mx = in ? __ldcg(&d.mx[row]) : 0;
        r[hf].mz = in ? __ldcg(&d.mz[row]) : 0;
        r[hf].dx = in ? __ldcg(&d.dx[row]) : 0;
        r[hf].dz = in ? __ldcg(&d.dz[row]) : 0;
        r[hf].de = in ? __ldcg(&d.de[row]) : 0;
        r[hf].piv = in ? __ldcg(&d.piv[row]) : 0x7fffffff;
        r[hf].A = in ? (1ull << row) : 0;
        r[hf].t0 = 0;
        r[hf].t1 = 0;
    }
    int rx = __ldcg(&d.meta[0]);
    int ga = 0, gb = 0;  // the run's phase factor omega^ga sqrt(2)^gb
    unsigned long long gi = oi;
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
        const int q0 = (int)__shfl_sync(SF_FULL, wr.q0, src);
        const int q1 = kind >= 6 ? (int)__shfl_sync(SF_FULL, wr.q1, src) : 0;
        if (!warp_clifford_gate(r, n, rx, (int)kind, q0, q1, stage, ga, gb)) {
            if (lane == 0) {
                set_status(d.status, SF_ST_INTERNAL, buf, 41u);
                gp_fail(w);
            }
            break;
        }
        gi++;
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
    for (int j = 0; j < n; j++) {
        const unsigned b0 = __ballot_sync(SF_FULL, lane < n && ((r[0].A >> j) & 1));
        const unsigned b1 = __ballot_sync(SF_FULL, lane + 32 < n && ((r[1].A >> j) & 1));
        if (lane == 0) w->AT[j] = (uint64_t)b0 | ((uint64_t)b1 << 32);
    }
    // rows of A, inverted next while other warps plan
    for (int hf = 0; hf < 2; hf++)
        if (lane + 32 * hf < n) arows[lane + 32 * hf] = r[hf].A;
    const unsigned t0 = __ballot_sync(SF_FULL, lane < n && r[0].t0);
    const unsigned t1 = __ballot_sync(SF_FULL, lane + 32 < n && r[1].t0);
    if (lane == 0) {
        w->t = (uint64_t)t0 | ((uint64_t)t1 << 32);
        d.meta[0] = rx;
        *d.g = cmul(*d.g, cliff_factor(ga, gb));
        w->oe = gi;
    }
}

// Plan of diagonal record o (warp 0 of one CTA) into the workspace.
__device__ void gp_plan(const SfDev& d, const OpRec& o, GpPlan& sp, GpPlan* out) {
    const int n = d.n, lane = threadIdx.x & 31;
    Row r[2];
    for (int hf = 0; hf < 2; hf++) {
        const int row = lane + 32 * hf;
        const bool in = row < n;
        r[hf].mx = in ? __ldcg(&d.mx[row]) : 0;
        r[hf].mz = in ? __ldcg(&d.mz[row]) : 0;
        r[hf].dx = in ? __ldcg(&d.dx[row]) : 0;
        r[hf].dz = in ? __ldcg(&d.dz[row]) : 0;
        r[hf].de = in ? __ldcg(&d.de[row]) : 0;
    }
    const uint32_t kind = o.kind - SF_OP_DIAG;
    const double th = kind == 0 ? 0.78539816339744830962 : (kind == 1 ? -0.78539816339744830962 : o.param);
    double sn, cs;
    sincos(th, &sn, &cs);
    const SfTerms T = diag_terms(kind, cs, sn);
    warp_branch_plan_regs(r, n, kind, (int)o.q0, kind == 3 ? (int)o.q1 : 0, T.c, sp.P, sp.ctab);
    __syncwarp();
    const uint64_t* src = reinterpret_cast<const uint64_t*>(&sp);
    uint64_t* dst = reinterpret_cast<uint64_t*>(out);
    for (int i = lane; i < (int)(sizeof(GpPlan) / 8); i += 32) dst[i] = src[i];
}

// elements [lo, hi) of CTA b: contiguous chunks, whole warps, all CTAs busy
__device__ __forceinline__ void gp_chunk(unsigned long long k, unsigned long long& lo, unsigned long long& hi) {
    const unsigned long long per = ((k + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
    lo = min(k, (unsigned long long)blockIdx.x * per);
    hi = min(k, lo + per);
}

__global__ void __launch_bounds__(kGpThreads) k_gprog(SfDev d, GpWork* w, const OpRec* ops, unsigned long long n_ops,
                                                      double eps2, int cur0, unsigned long long* consumed) {
    extern __shared__ GpPlan spl[];  // [kGpPlans]: the plans of the current diagonal run
    __shared__ GpPlan sp;            // scratch of the planning warp
    __shared__ BrTab pm;             // a plan moved to the coordinates before a pending affine map
    __shared__ uint64_t s_ainv[64], s_at[64];
    __shared__ uint64_t tab[16 * 16];
    __shared__ Row stage[64];
    __shared__ unsigned int wsum[kGpThreads / 32];
    __shared__ unsigned long long bbase;
    __shared__ int s_nb;
    if (*(volatile uint32_t*)d.status) return;
    const int n = d.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned gen = 0;
    if (threadIdx.x == 0) {
        gen = ld_acquire(&w->bar_gen);
        s_phase = gen;
    }
    __syncthreads();
    // every record is checked before anything is touched
    {
        bool bad = false;
        for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_ops;
             i += (unsigned long long)gridDim.x * blockDim.x) {
            const OpRec o = ops[i];
            const uint32_t k = o.kind == SF_OP_COND ? o.arg : o.kind;
            const bool two = (k >= 6 && k <= 8) || k == SF_OP_DIAG + 3;
            bool ok = o.q0 < (uint32_t)n && (!two || (o.q1 < (uint32_t)n && o.q1 != o.q0));
            if (o.kind == SF_OP_COND) ok &= o.arg <= 8;
            else ok &= k <= 8 || (k >= SF_OP_DIAG && k <= SF_OP_DIAG + 3) || k == SF_OP_MEASURE;
            bad |= !ok;
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) {
            set_status(d.status, 1u, cur0, 42u);  // SF_EINVAL: bad record
            gp_fail(w);
        }
        if (!gp_barrier(w, gen, d.status, cur0)) return;
    }
    int cur = cur0;
    unsigned long long k = d.kcnt[cur0];
    uint32_t tag[2] = {d.itag[0], d.itag[1]};
    unsigned long long isz[2] = {d.isize[0], d.isize[1]};
    unsigned long long oi = 0;
    unsigned nmerge = 0;
    bool ok = true;
    bool have_u = false;  // the frame is closed under the mask cu (s in F => s ^ cu in F)
    uint64_t cu = 0;
    unsigned npre = 0;    // records at oi planned by the last Clifford phase
    // The last Clifford run's map sigma' = A sigma ^ t is not yet applied to the
    // phase vectors (the tableau is already new); the next merge applies it.
    bool aff = false;
    const int nc = (n + 3) >> 2;
    uint64_t tw = 0;
    // 4-bit lookup tables of the pending map (columns of A from the workspace)
    auto affine_tables = [&]() {
        for (int e = threadIdx.x; e < nc * 16; e += blockDim.x) {
            const int v = e & 15, c = e >> 4;
            uint64_t acc = 0;
#pragma unroll
            for (int b = 0; b < 4; b++)
                if (((v >> b) & 1) && 4 * c + b < n) acc ^= __ldcg(&w->AT[4 * c + b]);
            tab[e] = acc;
        }
        tw = __ldcg(&w->t);
        __syncthreads();
    };
    auto affine_of = [&](uint64_t x) {
        uint64_t o = tw;
        for (int c = 0; c < nc; c++) o ^= tab[c * 16 + ((x >> (4 * c)) & 15)];
        return o;
    };
    // the map applied to every phase vector, which go into a fresh index
    auto affine_pass = [&]() {
        affine_tables();
        const uint32_t tg = next_tag(tag[cur]);
        const unsigned long long T = index_slots(k, d.icap);
        uint64_t* S = d.sig[cur];
        unsigned long long lo, hi;
        gp_chunk(k, lo, hi);
        for (unsigned long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
            const uint64_t o = affine_of(__ldcg(&S[j]));
            S[j] = o;
            ok &= index_insert<1>(d, cur, T, tg, &o, (uint32_t)j);
        }
        tag[cur] = tg;
        isz[cur] = T;
        if (!ok) {
            set_status(d.status, SF_ST_TIMEOUT, cur, 43u);  // index full
            gp_fail(w);
        }
        aff = false;
    };
    // on a failed check: the frame stays in buffer cur (its count and the
    // index tags go back for the host's error path), and the launch ends
    auto bail = [&]() {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            d.kcnt[cur] = k;
            for (int b = 0; b < 2; b++) {
                d.itag[b] = tag[b];
                d.isize[b] = isz[b];
            }
        }
    };
    while (oi < n_ops) {
        const uint32_t kind = ops[oi].kind;
        if (kind <= 8) {
            // ---- Clifford run: tableau in one warp of CTA 0, whose other warps then plan
            // the diagonal records that follow (one record each) in the same phase;
            // then the affine pass with a fresh index
            if (blockIdx.x == 0) {
                if (warp == 0) gp_clifford_run(d, w, ops, oi, n_ops, stage, s_ainv, cur);
                __syncthreads();
                if (warp == 0) {
                    // rows of A^-1, for a merge that reads the phase vectors before the map
                    const uint64_t av[2] = {lane < n ? s_ainv[lane] : 0, lane + 32 < n ? s_ainv[lane + 32] : 0};
                    uint64_t iv[2];
                    if (!warp_gf2_inverse(av, n, iv) && lane == 0) {
                        set_status(d.status, SF_ST_INTERNAL, cur, 49u);
                        gp_fail(w);
                    }
                    for (int hf = 0; hf < 2; hf++)
                        if (lane + 32 * hf < n) w->Ainv[lane + 32 * hf] = iv[hf];
                }
                const unsigned long long oe = __ldcg(&w->oe);
                const unsigned long long ri = oe + lane;
                bool dg = false;
                if (ri < n_ops) {
                    const uint32_t kk = ops[ri].kind;
                    dg = kk >= SF_OP_DIAG && kk <= SF_OP_DIAG + 3;
                }
                const unsigned bl = __ballot_sync(SF_FULL, dg);
                int np = bl == SF_FULL ? 32 : __ffs(~bl) - 1;
                np = np < (int)(blockDim.x >> 5) - 1 ? np : (int)(blockDim.x >> 5) - 1;
                if (*(volatile uint32_t*)d.status) np = 0;
                if (warp >= 1 && warp - 1 < np) gp_plan(d, ops[oe + warp - 1], spl[warp - 1], &w->plans[warp - 1]);
                if (threadIdx.x == 0) w->npre = (unsigned)np;
            }
            if (!gp_barrier(w, gen, d.status, cur)) return bail();
            npre = __ldcg(&w->npre);
            have_u = false;
            oi = __ldcg(&w->oe);
            // a following merge of two or more groups reads the phase vectors before
            // the map (partners at A^-1 u, sign patterns from A^T v); otherwise the
            // map is applied now
            if (npre > 0 && !__ldcg(&w->plans[0].P.bad) && __ldcg(&w->plans[0].P.ng) >= 2) {
                aff = true;
                continue;
            }
            affine_pass();
            if (!gp_barrier(w, gen, d.status, cur)) return bail();
            continue;
        }
        if (kind < SF_OP_DIAG || kind > SF_OP_DIAG + 3) break;  // measurement or conditional gate
        // ---- diagonal run: all plans first (unless the Clifford phase made them),
        // then one merge per record
        int nb = (int)npre;
        npre = 0;
        if (nb == 0) {
        if (warp == 0) {
            const unsigned long long ri = oi + lane;
            bool dg = false;
            if (ri < n_ops) {
                const uint32_t kk = ops[ri].kind;
                dg = kk >= SF_OP_DIAG && kk <= SF_OP_DIAG + 3;
            }
            const unsigned bl = __ballot_sync(SF_FULL, dg);
            int nb = bl == SF_FULL ? 32 : __ffs(~bl) - 1;
            nb = nb < kGpPlans ? nb : kGpPlans;
            if (lane == 0) s_nb = nb < (int)gridDim.x ? nb : (int)gridDim.x;
        }
        __syncthreads();
        nb = s_nb;
        if ((int)blockIdx.x < nb && warp == 0) gp_plan(d, ops[oi + blockIdx.x], sp, &w->plans[blockIdx.x]);
        if (!gp_barrier(w, gen, d.status, cur)) return bail();
        }
        {
            const uint64_t* src = reinterpret_cast<const uint64_t*>(w->plans);
            uint64_t* dst = reinterpret_cast<uint64_t*>(spl);
            for (int i = threadIdx.x; i < nb * (int)(sizeof(GpPlan) / 8); i += blockDim.x) dst[i] = __ldcg(&src[i]);
        }
        __syncthreads();
        int t = 0;
        while (t < nb) {
            // the longest run from t that one in-place pass takes: one-group gates
            // (a phase per element) and two-group gates whose second mask is the one
            // the frame is closed under (each pair {s, s ^ u} maps onto itself)
            int t2 = t;
            bool pairs = false;
            while (t2 < nb && !spl[t2].P.bad) {
                const BrTab& Q = spl[t2].P;
                if (Q.ng == 1 || (Q.ng == 2 && have_u && Q.u[1] == cu)) {
                    pairs |= Q.ng == 2;
                    t2++;
                } else {
                    break;
                }
            }
            if (t2 > t) {
                // ---- in-place run: the element with the smaller phase vector of each pair
                // applies the run's gates to both amplitudes (same sums, same order, as
                // the per-gate merge); phase vectors, positions and the index stay
                const unsigned long long kb = keep_bits(eps2);
                const uint64_t* S = d.sig[cur];
                double2* A = d.amp[cur];
                unsigned long long lo, hi;
                gp_chunk(k, lo, hi);
                bool drop = false, miss = false;
                const auto plan = [&](int r) { return PlanRef{&spl[r].P, spl[r].ctab}; };
                const int c_ = cur;
                const auto find = [&](uint64_t key) { return gp_find(d, c_, isz[c_], tag[c_], key); };
                for (unsigned long long base = lo + 64ull * warp; base < hi; base += 64ull * (blockDim.x >> 5))
                    inplace_run_warp<true>(S, A, base, hi, pairs, cu, t, t2, plan, find, kb, eps2, drop, miss);
                if (miss) {  // the frame is not closed after all
                    set_status(d.status, SF_ST_INTERNAL, cur, 47u);
                    gp_fail(w);
                }
                if (__syncthreads_or(drop) && threadIdx.x == 0) gp_dropped(w);
                if (!gp_barrier(w, gen, d.status, cur)) return bail();
                t = t2;
                if (!s_drop) continue;
                // ---- amplitudes fell below the threshold: compact the frame
                const int in = cur, out = cur ^ 1;
                const unsigned long long Tout = index_slots(k, d.icap);
                const uint32_t tag_out = next_tag(tag[out]);
                unsigned long long* ctr = &w->ocnt[nmerge % 3];
                if (blockIdx.x == 0 && threadIdx.x == 0) w->ocnt[(nmerge + 1) % 3] = 0;
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
                        ok &= index_insert<1>(d, out, Tout, tag_out, &s0, (uint32_t)o);
                    }
                }
                if (!ok) {
                    set_status(d.status, SF_ST_TIMEOUT, in, 48u);  // index full
                    gp_fail(w);
                }
                if (!gp_barrier(w, gen, d.status, in)) return bail();
                k = __ldcg(ctr);
                cur = out;
                tag[out] = tag_out;
                isz[out] = Tout;
                nmerge++;
                have_u = false;
                continue;
            }
            // ---- merge of record t into the other buffer
            const BrTab& P0 = spl[t].P;  // the plan in the tableau's coordinates
            const int ng = P0.ng;
            if (P0.bad || (unsigned long long)ng * k > d.cap) {
                if (blockIdx.x == 0 && threadIdx.x == 0)
                    set_status(d.status, P0.bad ? SF_ST_INTERNAL : SF_ST_CAPACITY, cur, P0.bad ? 44u : 0u);
                if (aff) affine_pass();  // the frame must match the tableau when the launch ends
                return bail();
            }
            if (aff) {
                // the phase vectors are still those before the map sigma' = A sigma ^ t:
                // partners at A^-1 u, sign patterns from A^T v flipped by parity(v & t);
                // outputs are written in the new coordinates
                affine_tables();
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    s_ainv[i] = __ldcg(&w->Ainv[i]);
                    s_at[i] = __ldcg(&w->AT[i]);
                }
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
            const unsigned long long kb = keep_bits(eps2);
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
                long long id[4] = {act ? (long long)j : -1, -1, -1, -1};
                if (act) {
                    s = __ldcg(&Si[j]);
                    a = __ldcg(&Ai[j]);
                    for (int g = 1; g < ng; g++) id[g] = gp_find(d, in, Tin, tag_in, s ^ P.u[g]);
                }
                double2 amps[4];
                unsigned keepm = 0;
                for (int g = 0; g < ng; g++) {
                    bool own = act;
                    for (int g2 = 0; g2 < g; g2++) own &= id[P.xidx[g][g2]] < 0;
                    double2 amp = make_double2(0.0, 0.0);
                    if (own) {
                        for (int g2 = 0; g2 < ng; g2++) {
                            const int m = P.xidx[g][g2];
                            if (id[m] < 0) continue;
                            const double2 ap = m == 0 ? a : __ldcg(&Ai[id[m]]);
                            cmul_acc(amp, half_coef(P, ctab, g2, s ^ P.u[m]), ap);
                        }
                    }
                    amps[g] = amp;
                    if (own && amp_kept(amp, kb, eps2)) keepm |= 1u << g;
                    else if (own) drop = true;
                }
                unsigned long long o = block_out_range(ctr, __popc(keepm), wsum, &bbase);
                const uint64_t sn = aff && act ? affine_of(s) : s;  // the parent in the new coordinates
                for (int g = 0; g < ng; g++) {
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
            if (!gp_barrier(w, gen, d.status, in)) return bail();
            k = __ldcg(ctr);
            cur = out;
            tag[out] = tag_out;
            isz[out] = Tout;
            nmerge++;
            // no output dropped: every parent s gave s ^ u_g for all g, so the new
            // frame is closed under the gate's masks
            have_u = !s_drop && ng == 2;
            cu = P0.u[1];
            aff = false;
            t++;
        }
        oi += nb;
    }
    if (aff) {  // not reached in practice: a pending map always has a merge after it
        affine_pass();
        if (!gp_barrier(w, gen, d.status, cur)) return bail();
    }
    // the frame goes back to buffer cur0, indexed
    if (cur != cur0) {
        const uint32_t tg = next_tag(tag[cur0]);
        const unsigned long long T = index_slots(k, d.icap);
        unsigned long long lo, hi;
        gp_chunk(k, lo, hi);
        for (unsigned long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
            const uint64_t s = __ldcg(&d.sig[cur][j]);
            d.sig[cur0][j] = s;
            d.amp[cur0][j] = __ldcg(&d.amp[cur][j]);
            ok &= index_insert<1>(d, cur0, T, tg, &s, (uint32_t)j);
        }
        if (!ok) set_status(d.status, SF_ST_TIMEOUT, cur0, 46u);
        tag[cur0] = tg;
        isz[cur0] = T;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d.kcnt[cur0] = k;
        d.itag[cur0] = tag[cur0];
        d.isize[cur0] = isz[cur0];
        d.itag[cur0 ^ 1] = tag[cur0 ^ 1];  // stale, but its tag must not repeat
        d.isize[cur0 ^ 1] = isz[cur0 ^ 1];
        if (consumed) *consumed = oi;
    }
}

}  // namespace

size_t sf_gprog_work_words() { return (sizeof(GpWork) + 7) / 8; }

// clears the per-launch words of the workspace (stream-ordered)
cudaError_t sf_gprog_clear(const SfDev& d, cudaStream_t s) {
    GpWork* w = reinterpret_cast<GpWork*>(d.gp);
    return cudaMemsetAsync(&w->err[0], 0, offsetof(GpWork, oe) - offsetof(GpWork, err), s);
}

// resets the barrier after a launch that gave up waiting
cudaError_t sf_gprog_reset(const SfDev& d, cudaStream_t s) {
    return cudaMemsetAsync(d.gp, 0, sizeof(GpWork), s);
}

cudaError_t sf_launch_gprog(const SfDev& d, const void* ops, unsigned long long n_ops, double eps2, int cur,
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
                              n_ops, eps2, cur, consumed);
}
