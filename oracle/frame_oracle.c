/*
 * frame_oracle.c -- plain, slow, single-threaded CPU stabilizer-frame simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  It shares no code with the CUDA library and is loaded only
 * by the tests, by __graft_entry__.smoke() and by bench.py's CPU-baseline leg.
 *
 * It follows the paper (Garcia & Markov, "Simulation of Quantum Circuits via
 * Stabilizer Frames") step by step, in the paper's order and notation:
 *   - Pauli literals in two bits, 00=I 01=Z 10=X 11=Y (Sec. II-B, tableau
 *     encoding); products of literals by Table 1 (looked up, not derived).
 *   - Conjugation of a row by H, P(=S), CNOT by Table 2 (looked up); the other
 *     Clifford kinds are compositions of those three (Corollary 1 style:
 *     P^3 = P^dagger, Z = P^2, X = H Z H, CZ = H_t CNOT H_t, SWAP = 3 CNOT).
 *   - The stabilizer matrix M is kept in row-reduced echelon form after every
 *     operation (Invariant 1) by full Gauss-Jordan elimination over the columns
 *     x_0..x_{n-1}, z_0..z_{n-1}; the row operations are recorded once per gate
 *     and replayed on every phase vector ("memoise the updates to M", Sec. III).
 *   - Global phases of the frame states follow the five-step algorithm of
 *     Sec. III ("Global phases of states in F"), with the basis state |b> of
 *     step 2 read as the anchor b*(sigma): the support element whose bits at
 *     every X-block pivot qubit are 0, where psi_can(M, sigma) has amplitude
 *     2^{-r/2} (real, positive).  Step 3-4 evaluate U^dagger on the new anchor,
 *     summing over the (at most four) basis states the gate mixes.
 *   - Amplitudes of a frame state at a basis point use Observation 1 solved in
 *     closed form on the RREF: multiply the X-block rows selected by the pivot
 *     bits of (y xor b*) and read the i-power of the product.
 *   - Diagonal non-Clifford gates branch each element by the anticommutation
 *     mask (Sec. IV, T gate as a two-term sum): P(theta) = alpha I + beta Z_t.
 *     The controlled phase of Eq. 3 is applied as
 *     P(theta/2)_c P(theta/2)_t CNOT P(-theta/2)_t CNOT.
 *   - COFACTOR (Sec. III) for random-outcome measurements: the measurement
 *     update of Sec. II-B forced to each outcome, children weighted by the
 *     five-step phase rule with U = the projector.
 *   - Toffoli and controlled-R(alpha) by cofactors (Eq. 2 and Eq. 3): COFACTOR
 *     on the two qubits, then X_t (or the phase e^{i alpha}) applied to the
 *     states of the 11 cofactor only.
 *   - Coalescing = the set semantics of Def. 1: sort, merge equal phase
 *     vectors, drop |a| < eps.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { OF_OK = 0, OF_EINVAL = 1, OF_ENOMEM = 2, OF_ECAPACITY = 3, OF_ESTATE = 6 };

/* ---- element ranges (Sec. V) -----------------------------------------------
 * The per-element loops of ROTATE, branching, COFACTOR and the amplitude sum
 * touch each phase vector independently.  Sec. V runs them by splitting the
 * phase vectors into equal consecutive ranges, one thread per range, joined
 * before the operation returns; of_set_threads chooses the number of ranges
 * (default 1: plain sequential loops).  Every element is computed by the same
 * code either way, so frames are identical; sums over the frame are added per
 * range and then range by range.                                              */
#define OF_MAX_THREADS 256
static int g_threads = 1;

int of_set_threads(int t) {
    g_threads = t < 1 ? 1 : (t > OF_MAX_THREADS ? OF_MAX_THREADS : t);
    return g_threads;
}

typedef void (*range_fn)(void* ctx, size_t lo, size_t hi, int part);
typedef struct { range_fn fn; void* ctx; size_t lo, hi; int part; } range_job;

static void* range_run(void* p) {
    range_job* j = (range_job*)p;
    j->fn(j->ctx, j->lo, j->hi, j->part);
    return NULL;
}

/* fn over [0, k) in at most g_threads consecutive ranges; returns the number
 * of ranges used (range i is part i) */
static int for_ranges(size_t k, range_fn fn, void* ctx) {
    int T = g_threads;
    if ((size_t)T > k) T = k ? (int)k : 1;
    if (T <= 1) {
        fn(ctx, 0, k, 0);
        return 1;
    }
    range_job jobs[OF_MAX_THREADS];
    pthread_t th[OF_MAX_THREADS];
    int started[OF_MAX_THREADS];
    size_t per = (k + T - 1) / T;
    for (int t = 0; t < T; t++) {
        size_t lo = (size_t)t * per, hi = lo + per;
        jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].part = t;
        jobs[t].lo = lo < k ? lo : k;
        jobs[t].hi = hi < k ? hi : k;
        started[t] = t > 0 && pthread_create(&th[t], NULL, range_run, &jobs[t]) == 0;
    }
    for (int t = 0; t < T; t++)
        if (!started[t]) range_run(&jobs[t]);
    for (int t = 1; t < T; t++)
        if (started[t]) pthread_join(th[t], NULL);
    return T;
}

/* literals: (x<<1)|z  ->  I=0, Z=1, X=2, Y=3 */
enum { LI = 0, LZ = 1, LX = 2, LY = 3 };

/* ---- Table 1: multiplication of Pauli literals (row * column) -------------
 * entry = (phase exponent k of i^k, result literal).                         */
static const int T1_PHASE[4][4] = {
    /*        I  Z  X  Y   (column operand) */
    /* I */ {0, 0, 0, 0},
    /* Z */ {0, 0, 1, 3}, /* Z*X = iY, Z*Y = -iX */
    /* X */ {0, 3, 0, 1}, /* X*Z = -iY, X*Y = iZ */
    /* Y */ {0, 1, 3, 0}, /* Y*Z = iX, Y*X = -iZ */
};
static const int T1_RES[4][4] = {
    {LI, LZ, LX, LY},
    {LZ, LI, LY, LX},
    {LX, LY, LI, LZ},
    {LY, LX, LZ, LI},
};

/* ---- Table 2: conjugation by H, P and CNOT -------------------------------
 * one-qubit: out literal and sign bit for input literal                       */
static const int T2_H_OUT[4] = {LI, LX, LZ, LY};  /* Z->X, X->Z, Y->-Y */
static const int T2_H_SGN[4] = {0, 0, 0, 1};
static const int T2_P_OUT[4] = {LI, LZ, LY, LX};  /* Z->Z, X->Y, Y->-X */
static const int T2_P_SGN[4] = {0, 0, 0, 1};
/* CNOT (control = qubit 1, target = qubit 2) on the six generators of the
 * table; other two-qubit literals are products of these (Table 1).            */
static void t2_cnot_single(int which, int lit, int* o1, int* o2) {
    /* which = 1: literal on control, identity on target; which = 2: reverse */
    if (which == 1) {
        switch (lit) {
            case LI: *o1 = LI; *o2 = LI; break;
            case LX: *o1 = LX; *o2 = LX; break; /* X1 I2 -> X1 X2 */
            case LY: *o1 = LY; *o2 = LX; break; /* Y1 I2 -> Y1 X2 */
            default: *o1 = LZ; *o2 = LI; break; /* Z1 I2 -> Z1 I2 */
        }
    } else {
        switch (lit) {
            case LI: *o1 = LI; *o2 = LI; break;
            case LX: *o1 = LI; *o2 = LX; break; /* I1 X2 -> I1 X2 */
            case LY: *o1 = LZ; *o2 = LY; break; /* I1 Y2 -> Z1 Y2 */
            default: *o1 = LZ; *o2 = LZ; break; /* I1 Z2 -> Z1 Z2 */
        }
    }
}

int ot_pauli_mult(int a, int b, int* phase) {
    *phase = T1_PHASE[a][b];
    return T1_RES[a][b];
}

/* one-qubit conjugation by H (g=0) or P (g=1) */
static int conj1(int g, int lit, int* sgn) {
    if (g == 0) { *sgn ^= T2_H_SGN[lit]; return T2_H_OUT[lit]; }
    *sgn ^= T2_P_SGN[lit];
    return T2_P_OUT[lit];
}

/* CNOT conjugation of the literal pair (l1 on control, l2 on target).
 * (l1 x l2) = (l1 x I)(I x l2): conjugate both factors, multiply by Table 1.
 * Returns the i-power of the product (0 or 2 for Hermitian inputs).        */
static int conj_cnot(int* l1, int* l2) {
    int a1, a2, b1, b2, p1, p2;
    t2_cnot_single(1, *l1, &a1, &a2);
    t2_cnot_single(2, *l2, &b1, &b2);
    *l1 = ot_pauli_mult(a1, b1, &p1);
    *l2 = ot_pauli_mult(a2, b2, &p2);
    return (p1 + p2) & 3;
}

/* Conjugate a literal pair by the named Clifford; kinds as include/sf.h:
 * H=0 S=1 SDG=2 X=3 Y=4 Z=5 CNOT=6 CZ=7 SWAP=8.  Two-qubit gates act on
 * (l0 on q0, l1 on q1).  Returns the sign bit of the conjugated operator.   */
int ot_conjugate(int kind, int* l0, int* l1) {
    int sgn = 0, t;
    switch (kind) {
        case 0: *l0 = conj1(0, *l0, &sgn); break;
        case 1: *l0 = conj1(1, *l0, &sgn); break;
        case 2: /* P^dagger = P^3 */
            for (t = 0; t < 3; t++) *l0 = conj1(1, *l0, &sgn);
            break;
        case 5: /* Z = P^2 */
            for (t = 0; t < 2; t++) *l0 = conj1(1, *l0, &sgn);
            break;
        case 3: /* X = H Z H */
            *l0 = conj1(0, *l0, &sgn);
            for (t = 0; t < 2; t++) *l0 = conj1(1, *l0, &sgn);
            *l0 = conj1(0, *l0, &sgn);
            break;
        case 4: /* Y = i X Z: conjugation by Z then by X */
            for (t = 0; t < 2; t++) *l0 = conj1(1, *l0, &sgn);
            *l0 = conj1(0, *l0, &sgn);
            for (t = 0; t < 2; t++) *l0 = conj1(1, *l0, &sgn);
            *l0 = conj1(0, *l0, &sgn);
            break;
        case 6: sgn ^= conj_cnot(l0, l1) >> 1; break;
        case 7: /* CZ = H_t CNOT H_t */
            *l1 = conj1(0, *l1, &sgn);
            sgn ^= conj_cnot(l0, l1) >> 1;
            *l1 = conj1(0, *l1, &sgn);
            break;
        case 8: /* SWAP = CNOT(0,1) CNOT(1,0) CNOT(0,1) */
            sgn ^= conj_cnot(l0, l1) >> 1;
            sgn ^= conj_cnot(l1, l0) >> 1;
            sgn ^= conj_cnot(l0, l1) >> 1;
            break;
        default: return -1;
    }
    return sgn;
}

/* ---- frame ------------------------------------------------------------------ */
typedef struct {
    int n, W;
    uint64_t *x, *z; /* n*W, row-major, unsigned rows of M */
    int* piv;        /* pivot column of each row, column c<n is x_c, else z_{c-n} */
    int r;           /* X-block size */
    size_t k, cap;
    uint64_t* sig;   /* k*W */
    cplx* a;
} ofr;

typedef struct { int type, h, i, c; } gop; /* type 0: M_h <- M_h M_i (sign bit c); 1: swap */
typedef struct { gop* v; size_t n, cap; } gprog;

static void prog_push(gprog* p, int type, int h, int i, int c) {
    if (p->n == p->cap) {
        p->cap = p->cap ? 2 * p->cap : 64;
        p->v = (gop*)realloc(p->v, p->cap * sizeof(gop));
    }
    p->v[p->n].type = type; p->v[p->n].h = h; p->v[p->n].i = i; p->v[p->n].c = c;
    p->n++;
}

static inline int getb(const uint64_t* v, int q) { return (int)((v[q >> 6] >> (q & 63)) & 1u); }
static inline void flipb(uint64_t* v, int q) { v[q >> 6] ^= (uint64_t)1 << (q & 63); }
static inline void setb(uint64_t* v, int q, int b) {
    if (getb(v, q) != b) flipb(v, q);
}
static inline int lit_of(const uint64_t* x, const uint64_t* z, int q) { return (getb(x, q) << 1) | getb(z, q); }
static inline void put_lit(uint64_t* x, uint64_t* z, int q, int l) {
    setb(x, q, (l >> 1) & 1);
    setb(z, q, l & 1);
}

/* Ordered product (x1,z1) * (x2,z2) by Table 1, qubit by qubit; result into
 * (xo,zo), returns the i-power.                                              */
static int row_product(int n, const uint64_t* x1, const uint64_t* z1, const uint64_t* x2,
                       const uint64_t* z2, uint64_t* xo, uint64_t* zo) {
    int ph = 0;
    for (int q = 0; q < n; q++) {
        int p, l = ot_pauli_mult(lit_of(x1, z1, q), lit_of(x2, z2, q), &p);
        ph += p;
        put_lit(xo, zo, q, l);
    }
    return ph & 3;
}

static int col_bit(const ofr* f, int h, int c) {
    return c < f->n ? getb(f->x + (size_t)h * f->W, c) : getb(f->z + (size_t)h * f->W, c - f->n);
}

static void swap_rows(ofr* f, int a, int b) {
    for (int w = 0; w < f->W; w++) {
        uint64_t t = f->x[(size_t)a * f->W + w];
        f->x[(size_t)a * f->W + w] = f->x[(size_t)b * f->W + w];
        f->x[(size_t)b * f->W + w] = t;
        t = f->z[(size_t)a * f->W + w];
        f->z[(size_t)a * f->W + w] = f->z[(size_t)b * f->W + w];
        f->z[(size_t)b * f->W + w] = t;
    }
}

/* M_h <- M_h * M_i; returns the sign bit of the product (rows commute, so the
 * i-power is 0 or 2).                                                          */
static int rowsum(ofr* f, int h, int i) {
    int W = f->W;
    uint64_t* xo = (uint64_t*)calloc(W, 8);
    uint64_t* zo = (uint64_t*)calloc(W, 8);
    int ph = row_product(f->n, f->x + (size_t)h * W, f->z + (size_t)h * W, f->x + (size_t)i * W,
                         f->z + (size_t)i * W, xo, zo);
    memcpy(f->x + (size_t)h * W, xo, 8 * W);
    memcpy(f->z + (size_t)h * W, zo, 8 * W);
    free(xo);
    free(zo);
    return (ph >> 1) & 1;
}

/* Gauss-Jordan elimination to the canonical RREF (Invariant 1), recording the
 * row operations into prog.  Returns 0, or -1 if the rows are dependent.     */
static int gauss_jordan(ofr* f, gprog* prog) {
    int n = f->n, next = 0;
    for (int c = 0; c < 2 * n && next < n; c++) {
        int p = -1;
        for (int h = next; h < n; h++)
            if (col_bit(f, h, c)) { p = h; break; }
        if (p < 0) continue;
        if (p != next) {
            swap_rows(f, p, next);
            prog_push(prog, 1, p, next, 0);
        }
        for (int h = 0; h < n; h++) {
            if (h != next && col_bit(f, h, c)) {
                int cb = rowsum(f, h, next);
                prog_push(prog, 0, h, next, cb);
            }
        }
        f->piv[next] = c;
        next++;
    }
    if (next != n) return -1;
    f->r = 0;
    for (int h = 0; h < n; h++)
        if (f->piv[h] < n) f->r++;
    return 0;
}

static void replay(const gprog* prog, uint64_t* s) {
    for (size_t t = 0; t < prog->n; t++) {
        const gop* o = &prog->v[t];
        if (o->type == 0) {
            if (getb(s, o->i) ^ o->c) flipb(s, o->h);
        } else {
            int a = getb(s, o->h), b = getb(s, o->i);
            setb(s, o->h, b);
            setb(s, o->i, a);
        }
    }
}

/* anchor b*(sigma): bits at every X-pivot are 0, Z-rows hold with signs sigma. */
static void anchor(const ofr* f, const uint64_t* s, uint64_t* b) {
    int n = f->n, W = f->W;
    memset(b, 0, 8 * W);
    for (int h = f->r; h < n; h++)
        if (getb(s, h)) flipb(b, f->piv[h] - n);
    for (int h = 0; h < f->r; h++)
        if (getb(b, f->piv[h]))
            for (int w = 0; w < W; w++) b[w] ^= f->x[(size_t)h * W + w];
}

static int popc_and(int W, const uint64_t* a, const uint64_t* b) {
    int c = 0;
    for (int w = 0; w < W; w++) c += __builtin_popcountll(a[w] & b[w]);
    return c;
}

/* <y | psi_can(M, sigma)> (Observation 1 in closed form on the RREF). */
static cplx amp_at(const ofr* f, const uint64_t* s, const uint64_t* y) {
    int n = f->n, W = f->W;
    for (int h = f->r; h < n; h++)
        if ((popc_and(W, f->z + (size_t)h * W, y) & 1) != getb(s, h)) return 0.0;
    uint64_t* b = (uint64_t*)calloc(W, 8);
    uint64_t* d = (uint64_t*)calloc(W, 8);
    uint64_t* px = (uint64_t*)calloc(W, 8);
    uint64_t* pz = (uint64_t*)calloc(W, 8);
    anchor(f, s, b);
    for (int w = 0; w < W; w++) d[w] = y[w] ^ b[w];
    int nu = 0, sg = 0;
    for (int h = 0; h < f->r; h++) {
        if (!getb(d, f->piv[h])) continue;
        nu += row_product(n, px, pz, f->x + (size_t)h * W, f->z + (size_t)h * W, px, pz);
        sg += getb(s, h);
    }
    cplx v = 0.0;
    if (memcmp(px, d, 8 * W) == 0) {
        sg += popc_and(W, pz, b);
        int ip = (nu + popc_and(W, px, pz)) & 3;
        static const cplx IP[4] = {1.0, I, -1.0, -I};
        v = IP[ip] * ((sg & 1) ? -1.0 : 1.0) * pow(2.0, -0.5 * f->r);
    }
    free(b); free(d); free(px); free(pz);
    return v;
}

/* ---- small unitaries of the Clifford kinds (step 3 of the phase algorithm) ---
 * 1-qubit: U[out][in]; 2-qubit local index = bit(q0) + 2*bit(q1).            */
static void gate_matrix(int kind, cplx U[4][4], int* nq) {
    memset(U, 0, sizeof(cplx) * 16);
    const double r = 1.0 / sqrt(2.0);
    *nq = 1;
    switch (kind) {
        case 0: U[0][0] = r; U[0][1] = r; U[1][0] = r; U[1][1] = -r; break;
        case 1: U[0][0] = 1; U[1][1] = I; break;
        case 2: U[0][0] = 1; U[1][1] = -I; break;
        case 3: U[0][1] = 1; U[1][0] = 1; break;
        case 4: U[0][1] = -I; U[1][0] = I; break;
        case 5: U[0][0] = 1; U[1][1] = -1; break;
        case 6: /* CNOT control q0 target q1: |c t> -> |c, t^c> */
            *nq = 2; U[0][0] = 1; U[3][1] = 1; U[2][2] = 1; U[1][3] = 1; break;
        case 7: *nq = 2; U[0][0] = 1; U[1][1] = 1; U[2][2] = 1; U[3][3] = -1; break;
        case 8: *nq = 2; U[0][0] = 1; U[2][1] = 1; U[1][2] = 1; U[3][3] = 1; break;
    }
}

/* ---- API -------------------------------------------------------------------- */
static void frame_reset(ofr* f) {
    int n = f->n, W = f->W;
    memset(f->x, 0, 8 * (size_t)n * W);
    memset(f->z, 0, 8 * (size_t)n * W);
    for (int h = 0; h < n; h++) {
        flipb(f->z + (size_t)h * W, h);
        f->piv[h] = n + h;
    }
    f->r = 0;
    f->k = 1;
    memset(f->sig, 0, 8 * (size_t)W);
    f->a[0] = 1.0;
}

static int reserve(ofr* f, size_t k) {
    if (k <= f->cap) return 0;
    size_t c = f->cap ? f->cap : 16;
    while (c < k) c *= 2;
    uint64_t* s = (uint64_t*)realloc(f->sig, c * 8 * f->W);
    cplx* a = (cplx*)realloc(f->a, c * sizeof(cplx));
    if (!s || !a) return -1;
    f->sig = s; f->a = a; f->cap = c;
    return 0;
}

void* of_create(int n) {
    if (n <= 0) return NULL;
    ofr* f = (ofr*)calloc(1, sizeof(ofr));
    f->n = n;
    f->W = (n + 63) / 64;
    f->x = (uint64_t*)calloc((size_t)n * f->W, 8);
    f->z = (uint64_t*)calloc((size_t)n * f->W, 8);
    f->piv = (int*)calloc(n, sizeof(int));
    reserve(f, 16);
    frame_reset(f);
    return f;
}

void of_reset(void* h) { frame_reset((ofr*)h); }

void of_destroy(void* h) {
    ofr* f = (ofr*)h;
    if (!f) return;
    free(f->x); free(f->z); free(f->piv); free(f->sig); free(f->a); free(f);
}

static ofr* clone_tableau(const ofr* f) {
    ofr* g = (ofr*)calloc(1, sizeof(ofr));
    g->n = f->n; g->W = f->W; g->r = f->r;
    g->x = (uint64_t*)malloc(8 * (size_t)f->n * f->W);
    g->z = (uint64_t*)malloc(8 * (size_t)f->n * f->W);
    g->piv = (int*)malloc(sizeof(int) * f->n);
    memcpy(g->x, f->x, 8 * (size_t)f->n * f->W);
    memcpy(g->z, f->z, 8 * (size_t)f->n * f->W);
    memcpy(g->piv, f->piv, sizeof(int) * f->n);
    return g;
}
static void free_tableau(ofr* g) { free(g->x); free(g->z); free(g->piv); free(g); }

/* Steps of the five-step phase rule (Sec. III) for elements [lo, hi) of a
 * ROTATE: sign flips and the recorded row operations give sigma', the new
 * anchor b'*(sigma') is mapped back through U^dagger and read on the old M. */
typedef struct {
    ofr* f;
    const ofr* old;
    const gprog* prog;
    const uint64_t* flip;
    int q0, q1, two, nq;
    cplx U[4][4];
    double scale;
} rot_ctx;

static void rotate_range(void* vctx, size_t lo_j, size_t hi_j, int part) {
    (void)part;
    rot_ctx* cx = (rot_ctx*)vctx;
    ofr* f = cx->f;
    int W = f->W, q0 = cx->q0, q1 = cx->q1, two = cx->two;
    uint64_t* s = (uint64_t*)malloc(8 * W);
    uint64_t* b = (uint64_t*)malloc(8 * W);
    uint64_t* y = (uint64_t*)malloc(8 * W);
    for (size_t j = lo_j; j < hi_j; j++) {
        uint64_t* sj = f->sig + j * W;
        for (int w = 0; w < W; w++) s[w] = sj[w] ^ cx->flip[w];
        replay(cx->prog, s);
        anchor(f, s, b); /* new anchor b'*(sigma') on the new M */
        int lo = getb(b, q0) | (two ? getb(b, q1) << 1 : 0);
        cplx om = 0.0;
        for (int li = 0; li < (1 << cx->nq); li++) {
            if (cx->U[lo][li] == 0.0) continue;
            memcpy(y, b, 8 * W);
            setb(y, q0, li & 1);
            if (two) setb(y, q1, (li >> 1) & 1);
            om += cx->U[lo][li] * amp_at(cx->old, sj, y);
        }
        om *= cx->scale;
        memcpy(sj, s, 8 * W);
        f->a[j] *= om;
    }
    free(s); free(b); free(y);
}

/* ROTATE(F, U) for one Clifford gate (Sec. III). */
static int clifford_one(ofr* f, int kind, int q0, int q1) {
    int n = f->n, W = f->W, two = (kind >= 6);
    if (q0 < 0 || q0 >= n || (two && (q1 < 0 || q1 >= n || q1 == q0)) || kind < 0 || kind > 8)
        return OF_EINVAL;
    ofr* old = clone_tableau(f);
    /* conjugate every row; flip bits go to the phase vectors */
    uint64_t* flip = (uint64_t*)calloc(W, 8);
    for (int h = 0; h < n; h++) {
        uint64_t *xr = f->x + (size_t)h * W, *zr = f->z + (size_t)h * W;
        int l0 = lit_of(xr, zr, q0), l1 = two ? lit_of(xr, zr, q1) : 0;
        int s = ot_conjugate(kind, &l0, &l1);
        put_lit(xr, zr, q0, l0);
        if (two) put_lit(xr, zr, q1, l1);
        if (s) flipb(flip, h);
    }
    gprog prog = {0};
    if (gauss_jordan(f, &prog) != 0) { free(flip); free_tableau(old); return OF_ESTATE; }
    rot_ctx cx;
    cx.f = f; cx.old = old; cx.prog = &prog; cx.flip = flip;
    cx.q0 = q0; cx.q1 = q1; cx.two = two;
    gate_matrix(kind, cx.U, &cx.nq);
    cx.scale = pow(2.0, 0.5 * f->r);
    for_ranges(f->k, rotate_range, &cx);
    free(flip); free(prog.v);
    free_tableau(old);
    return OF_OK;
}

int of_clifford(void* h, const uint32_t* gates, size_t ng) {
    ofr* f = (ofr*)h;
    for (size_t g = 0; g < ng; g++) {
        int st = clifford_one(f, (int)gates[4 * g], (int)gates[4 * g + 1], (int)gates[4 * g + 2]);
        if (st) return st;
    }
    return OF_OK;
}

/* merge equal phase vectors (sort), dropping |a| < eps */
static int cmp_W;
static int cmp_sig(const void* A, const void* B) {
    const uint64_t* a = (const uint64_t*)A;
    const uint64_t* b = (const uint64_t*)B;
    for (int w = cmp_W - 1; w >= 0; w--) {
        if (a[w] < b[w]) return -1;
        if (a[w] > b[w]) return 1;
    }
    return 0;
}

static void merge_frame(ofr* f, double eps) {
    int W = f->W;
    size_t k = f->k, rec = 8 * W + sizeof(cplx);
    unsigned char* buf = (unsigned char*)malloc(k * rec + 1);
    for (size_t j = 0; j < k; j++) {
        memcpy(buf + j * rec, f->sig + j * W, 8 * W);
        memcpy(buf + j * rec + 8 * W, &f->a[j], sizeof(cplx));
    }
    cmp_W = W;
    qsort(buf, k, rec, cmp_sig);
    size_t out = 0, j = 0;
    while (j < k) {
        cplx acc;
        memcpy(&acc, buf + j * rec + 8 * W, sizeof(cplx));
        size_t e = j + 1;
        while (e < k && cmp_sig(buf + e * rec, buf + j * rec) == 0) {
            cplx t;
            memcpy(&t, buf + e * rec + 8 * W, sizeof(cplx));
            acc += t;
            e++;
        }
        if (cabs(acc) >= eps) {
            memcpy(f->sig + out * W, buf + j * rec, 8 * W);
            f->a[out] = acc;
            out++;
        }
        j = e;
    }
    f->k = out;
    free(buf);
}

/* one term c * Z^w applied to every element, children appended to dst */
typedef struct {
    const ofr* f;
    const uint64_t *w, *m;
    cplx c;
    uint64_t* dsig;
    cplx* da;
} term_ctx;

static void term_range(void* vctx, size_t lo, size_t hi, int part) {
    (void)part;
    term_ctx* cx = (term_ctx*)vctx;
    const ofr* f = cx->f;
    int W = f->W;
    uint64_t* b = (uint64_t*)malloc(8 * W);
    for (size_t j = lo; j < hi; j++) {
        const uint64_t* s = f->sig + j * W;
        anchor(f, s, b);
        int p = popc_and(W, b, cx->w) & 1;
        for (int t = 0; t < W; t++) cx->dsig[j * W + t] = s[t] ^ cx->m[t];
        cx->da[j] = cx->c * (p ? -1.0 : 1.0) * f->a[j];
    }
    free(b);
}

static void branch_term(const ofr* f, const uint64_t* w, cplx c, uint64_t* dsig, cplx* da) {
    int W = f->W, n = f->n;
    uint64_t* m = (uint64_t*)calloc(W, 8);
    for (int h = 0; h < n; h++)
        if (popc_and(W, f->x + (size_t)h * W, w) & 1) flipb(m, h);
    term_ctx cx = {f, w, m, c, dsig, da};
    for_ranges(f->k, term_range, &cx);
    free(m);
}

/* P(theta)_t = alpha I + beta Z_t (Sec. IV, T gate as a cofactor sum) */
static int phase_gate(ofr* f, int t, double theta, int merge) {
    int W = f->W;
    size_t k = f->k;
    if (reserve(f, 2 * k)) return OF_ENOMEM;
    cplx e = cexp(I * theta);
    cplx alpha = (1.0 + e) / 2.0, beta = (1.0 - e) / 2.0;
    uint64_t* w = (uint64_t*)calloc(W, 8);
    flipb(w, t);
    branch_term(f, w, beta, f->sig + k * W, f->a + k);
    for (size_t j = 0; j < k; j++) f->a[j] *= alpha;
    f->k = 2 * k;
    free(w);
    if (merge) merge_frame(f, 0.0);
    return OF_OK;
}

int of_nonclifford(void* h, uint32_t kind, uint32_t q0, uint32_t q1, double theta) {
    ofr* f = (ofr*)h;
    int n = f->n;
    if ((int)q0 >= n) return OF_EINVAL;
    switch (kind) {
        case 0: return phase_gate(f, (int)q0, M_PI / 4.0, 0);
        case 1: return phase_gate(f, (int)q0, -M_PI / 4.0, 0);
        case 2: return phase_gate(f, (int)q0, theta, 0);
        case 3: {
            if ((int)q1 >= n || q1 == q0) return OF_EINVAL;
            uint32_t cn[4] = {6, q0, q1, 0};
            int st;
            if ((st = phase_gate(f, (int)q0, theta / 2.0, 1))) return st;
            if ((st = phase_gate(f, (int)q1, theta / 2.0, 1))) return st;
            if ((st = of_clifford(f, cn, 1))) return st;
            if ((st = phase_gate(f, (int)q1, -theta / 2.0, 1))) return st;
            return of_clifford(f, cn, 1);
        }
    }
    return OF_EINVAL;
}

int of_coalesce(void* h, double eps, size_t* k) {
    ofr* f = (ofr*)h;
    merge_frame(f, eps);
    if (k) *k = f->k;
    return OF_OK;
}

#define OF_MEASURE_EPS 1e-12

static int find_zq_row(const ofr* f, int q) {
    int n = f->n, W = f->W;
    for (int h = f->r; h < n; h++) {
        if (f->piv[h] != n + q) continue;
        const uint64_t* zr = f->z + (size_t)h * W;
        int only = 1;
        for (int w = 0; w < W; w++) {
            uint64_t want = (q >> 6) == w ? ((uint64_t)1 << (q & 63)) : 0;
            if (zr[w] != want) only = 0;
        }
        return only ? h : -1;
    }
    return -1;
}

/* the two cofactors of elements [lo, hi): child x of element j goes to slot
 * 2j + x (valid[2j + x] = 1 when its weight is nonzero) */
typedef struct {
    ofr* f;
    const ofr* old;
    const gprog* prog;
    const uint64_t* anti;
    const int* cb;
    int piv_row, q;
    double scale;
    uint64_t* nsig;
    cplx* na;
    unsigned char* valid;
} cof_ctx;

static void cof_range(void* vctx, size_t lo, size_t hi, int part) {
    (void)part;
    cof_ctx* cx = (cof_ctx*)vctx;
    ofr* f = cx->f;
    int n = f->n, W = f->W;
    uint64_t* s = (uint64_t*)malloc(8 * W);
    uint64_t* b = (uint64_t*)malloc(8 * W);
    for (size_t j = lo; j < hi; j++) {
        const uint64_t* sj = f->sig + j * W;
        for (int x = 0; x < 2; x++) {
            memcpy(s, sj, 8 * W);
            for (int h = 0; h < n; h++)
                if (getb(cx->anti, h) && (getb(sj, cx->piv_row) ^ cx->cb[h])) flipb(s, h);
            setb(s, cx->piv_row, x);
            replay(cx->prog, s);
            anchor(f, s, b);
            cplx om = (getb(b, cx->q) == x) ? amp_at(cx->old, sj, b) * cx->scale : 0.0;
            if (om == 0.0) continue;
            memcpy(cx->nsig + (2 * j + x) * W, s, 8 * W);
            cx->na[2 * j + x] = f->a[j] * om;
            cx->valid[2 * j + x] = 1;
        }
    }
    free(s); free(b);
}

/* COFACTOR(F, q) (Sec. III): if q is random in M, the measurement update of
 * Sec. II-B forced to each outcome, every element split into its two
 * cofactors weighted by the five-step phase rule, then merged.  Afterwards
 * Z_q is a canonical row of M.                                               */
static int cofactor(ofr* f, uint32_t q) {
    int n = f->n, W = f->W;
    int piv_row = -1;
    for (int h = 0; h < n; h++)
        if (getb(f->x + (size_t)h * W, (int)q)) { piv_row = h; break; }
    if (piv_row >= 0) {
        ofr* old = clone_tableau(f);
        /* rows anticommuting with Z_q are multiplied by R_j, R_j becomes Z_q */
        uint64_t* anti = (uint64_t*)calloc(W, 8);
        int* cb = (int*)calloc(n, sizeof(int));
        for (int h = 0; h < n; h++) {
            if (h == piv_row || !getb(f->x + (size_t)h * W, (int)q)) continue;
            flipb(anti, h);
            cb[h] = rowsum(f, h, piv_row);
        }
        memset(f->x + (size_t)piv_row * W, 0, 8 * W);
        memset(f->z + (size_t)piv_row * W, 0, 8 * W);
        flipb(f->z + (size_t)piv_row * W, (int)q);
        gprog prog = {0};
        if (gauss_jordan(f, &prog)) return OF_ESTATE;
        size_t k = f->k;
        uint64_t* nsig = (uint64_t*)malloc(2 * k * 8 * W + 8);
        cplx* na = (cplx*)malloc(2 * k * sizeof(cplx) + 16);
        cof_ctx cx;
        cx.f = f; cx.old = old; cx.prog = &prog; cx.anti = anti; cx.cb = cb;
        cx.piv_row = piv_row; cx.q = (int)q; cx.scale = pow(2.0, 0.5 * f->r);
        cx.nsig = nsig; cx.na = na;
        cx.valid = (unsigned char*)calloc(2 * k + 1, 1);
        for_ranges(k, cof_range, &cx);
        /* children in element order, as one sequential pass would append them */
        size_t out = 0;
        for (size_t c = 0; c < 2 * k; c++) {
            if (!cx.valid[c]) continue;
            if (out != c) {
                memmove(nsig + out * W, nsig + c * W, 8 * W);
                na[out] = na[c];
            }
            out++;
        }
        free(cx.valid);
        if (reserve(f, out)) return OF_ENOMEM;
        memcpy(f->sig, nsig, out * 8 * W);
        memcpy(f->a, na, out * sizeof(cplx));
        f->k = out;
        free(nsig); free(na); free(anti); free(cb); free(prog.v);
        free_tableau(old);
        merge_frame(f, OF_MEASURE_EPS);
    }
    return OF_OK;
}

/* COFACTOR(F, q), then the measurement sum of Sec. IV; collapse keeps the
 * consistent states and renormalises.                                       */
int of_measure(void* hh, uint32_t q, int collapse, double* p0, double* p1) {
    ofr* f = (ofr*)hh;
    int W = f->W;
    if ((int)q >= f->n || collapse < -1 || collapse > 1) return OF_EINVAL;
    int st = cofactor(f, q);
    if (st) return st;
    int R = find_zq_row(f, (int)q);
    if (R < 0) return OF_ESTATE;
    double pr[2] = {0.0, 0.0};
    for (size_t j = 0; j < f->k; j++) {
        double m = creal(f->a[j]) * creal(f->a[j]) + cimag(f->a[j]) * cimag(f->a[j]);
        pr[getb(f->sig + j * W, R)] += m;
    }
    if (p0) *p0 = pr[0];
    if (p1) *p1 = pr[1];
    if (collapse >= 0) {
        if (pr[collapse] <= 0.0) return OF_ESTATE;
        double sc = 1.0 / sqrt(pr[collapse]);
        size_t out = 0;
        for (size_t j = 0; j < f->k; j++) {
            if (getb(f->sig + j * W, R) != collapse) continue;
            memmove(f->sig + out * W, f->sig + j * W, 8 * W);
            f->a[out] = f->a[j] * sc;
            out++;
        }
        f->k = out;
    }
    return OF_OK;
}

/* TOF_{c1 c2 t} by cofactors (Eq. 2 and its three steps): COFACTOR on c1
 * and c2, so that M holds the rows Z_c1 (index u) and Z_c2 (index v); then X_t
 * is applied to the states of the c1 c2 = 11 cofactor, the elements whose
 * phase vector is -1 at both u and v.  A Pauli gate leaves M unchanged, so X_t
 * acts on each such state as a frame rotation of that state alone: its
 * phase vector takes the sign flips of the rows that anticommute with X_t and
 * its amplitude the five-step phase factor.  The 11 class maps onto itself
 * (X_t commutes with Z_c1 and Z_c2), so no phase vectors collide.           */
int of_toffoli_cofactor(void* hh, uint32_t c1, uint32_t c2, uint32_t t) {
    ofr* f = (ofr*)hh;
    int n = f->n, W = f->W;
    if ((int)c1 >= n || (int)c2 >= n || (int)t >= n || c1 == c2 || c1 == t || c2 == t) return OF_EINVAL;
    int st = cofactor(f, c1);
    if (!st) st = cofactor(f, c2);
    if (st) return st;
    int u = find_zq_row(f, (int)c1), v = find_zq_row(f, (int)c2);
    if (u < 0 || v < 0) return OF_ESTATE;
    uint64_t* flip = (uint64_t*)calloc(W, 8);
    for (int h = 0; h < n; h++) {
        int l = lit_of(f->x + (size_t)h * W, f->z + (size_t)h * W, (int)t), dummy = 0;
        if (ot_conjugate(3, &l, &dummy)) flipb(flip, h);
    }
    cplx U[4][4];
    int nq;
    gate_matrix(3, U, &nq);
    uint64_t* s = (uint64_t*)malloc(8 * W);
    uint64_t* b = (uint64_t*)malloc(8 * W);
    uint64_t* y = (uint64_t*)malloc(8 * W);
    double scale = pow(2.0, 0.5 * f->r);
    for (size_t j = 0; j < f->k; j++) {
        uint64_t* sj = f->sig + j * W;
        if (!getb(sj, u) || !getb(sj, v)) continue;
        for (int w = 0; w < W; w++) s[w] = sj[w] ^ flip[w];
        anchor(f, s, b);
        int lo = getb(b, (int)t);
        cplx om = 0.0;
        for (int li = 0; li < 2; li++) {
            if (U[lo][li] == 0.0) continue;
            memcpy(y, b, 8 * W);
            setb(y, (int)t, li);
            om += U[lo][li] * amp_at(f, sj, y);
        }
        memcpy(sj, s, 8 * W);
        f->a[j] *= om * scale;
    }
    free(s); free(b); free(y); free(flip);
    return OF_OK;
}

/* R(alpha)_{ct} by cofactors (Eq. 3): COFACTOR on c and t, then the states of
 * the ct = 11 cofactor take the factor e^{i alpha}.                          */
int of_cr_cofactor(void* hh, uint32_t c, uint32_t t, double alpha) {
    ofr* f = (ofr*)hh;
    int W = f->W;
    if ((int)c >= f->n || (int)t >= f->n || c == t) return OF_EINVAL;
    int st = cofactor(f, c);
    if (!st) st = cofactor(f, t);
    if (st) return st;
    int u = find_zq_row(f, (int)c), v = find_zq_row(f, (int)t);
    if (u < 0 || v < 0) return OF_ESTATE;
    const cplx ph = cexp(I * alpha);
    for (size_t j = 0; j < f->k; j++) {
        const uint64_t* sj = f->sig + j * W;
        if (getb(sj, u) && getb(sj, v)) f->a[j] *= ph;
    }
    return OF_OK;
}

/* <y|Psi> summed over elements [lo, hi) (Observation 1 per element) */
typedef struct {
    const ofr* f;
    const uint64_t* y;
    cplx part[OF_MAX_THREADS];
} amp_ctx;

static void amp_range(void* vctx, size_t lo, size_t hi, int part) {
    amp_ctx* cx = (amp_ctx*)vctx;
    cplx acc = 0.0;
    for (size_t j = lo; j < hi; j++) acc += cx->f->a[j] * amp_at(cx->f, cx->f->sig + j * cx->f->W, cx->y);
    cx->part[part] = acc;
}

int of_amplitude(void* hh, const uint64_t* y, double* re, double* im) {
    ofr* f = (ofr*)hh;
    amp_ctx cx;
    cx.f = f; cx.y = y;
    int T = for_ranges(f->k, amp_range, &cx);
    cplx acc = 0.0;
    for (int t = 0; t < T; t++) acc += cx.part[t];
    *re = creal(acc);
    *im = cimag(acc);
    return OF_OK;
}

int of_get_tableau(void* hh, uint64_t* x, uint64_t* z, uint32_t* r) {
    ofr* f = (ofr*)hh;
    memcpy(x, f->x, 8 * (size_t)f->n * f->W);
    memcpy(z, f->z, 8 * (size_t)f->n * f->W);
    *r = (uint32_t)f->r;
    return OF_OK;
}

size_t of_size(void* hh) { return ((ofr*)hh)->k; }

/* frame sorted ascending by phase vector (word W-1 most significant) */
int of_get_frame(void* hh, uint64_t* sig, double* amp, size_t cap, size_t* k) {
    ofr* f = (ofr*)hh;
    merge_frame(f, 0.0); /* sort; equal vectors cannot remain after coalescing */
    *k = f->k;
    if (cap < f->k) return OF_ECAPACITY;
    memcpy(sig, f->sig, 8 * f->k * f->W);
    for (size_t j = 0; j < f->k; j++) {
        amp[2 * j] = creal(f->a[j]);
        amp[2 * j + 1] = cimag(f->a[j]);
    }
    return OF_OK;
}

/* load an explicit frame (for brute-force tests): M must be given in RREF */
int of_set_state(void* hh, const uint64_t* x, const uint64_t* z, const uint64_t* sig,
                 const double* amp, size_t k) {
    ofr* f = (ofr*)hh;
    int n = f->n, W = f->W;
    memcpy(f->x, x, 8 * (size_t)n * W);
    memcpy(f->z, z, 8 * (size_t)n * W);
    gprog prog = {0};
    int st = gauss_jordan(f, &prog);
    int moved = prog.n != 0;
    free(prog.v);
    if (st || moved) return OF_EINVAL;
    if (reserve(f, k ? k : 1)) return OF_ENOMEM;
    memcpy(f->sig, sig, 8 * k * W);
    for (size_t j = 0; j < k; j++) f->a[j] = amp[2 * j] + I * amp[2 * j + 1];
    f->k = k;
    return OF_OK;
}

/* psi_can(M, sigma) at basis point y, for tests that brute-force the basis. */
int of_basis_amp(void* hh, const uint64_t* s, const uint64_t* y, double* re, double* im) {
    cplx v = amp_at((ofr*)hh, s, y);
    *re = creal(v);
    *im = cimag(v);
    return OF_OK;
}

/* 1 if the stored tableau equals its own RREF (Invariant 1) */
int of_is_rref(void* hh) {
    ofr* f = (ofr*)hh;
    ofr* g = clone_tableau(f);
    gprog prog = {0};
    int st = gauss_jordan(g, &prog);
    int ok = (st == 0) && prog.n == 0 && memcmp(g->piv, f->piv, sizeof(int) * f->n) == 0;
    free(prog.v);
    free_tableau(g);
    return ok;
}
