/*
 * sf.h -- C ABI of libsf: a stabilizer-frame simulator that keeps one shared
 * canonical stabilizer tableau and a frame of (phase vector, FP64 amplitude)
 * pairs resident on one GPU (GB300, sm_103a).
 *
 * Model (Garcia & Markov, "Simulation of Quantum Circuits via Stabilizer
 * Frames"):
 *   - A stabilizer frame F = (M, {sigma_j}) (Def. 1, Sec. III) is an n x 2n
 *     binary tableau M of n commuting Pauli rows plus k distinct phase vectors
 *     sigma_j in {+1,-1}^n.  State j is M with the row signs set to sigma_j.
 *     The represented state is Psi = sum_j a_j |psi_j> with FP64 complex a_j.
 *   - M is kept in row-reduced echelon form after every operation
 *     (Invariant 1, Sec. III): columns ordered x_0..x_{n-1}, z_0..z_{n-1};
 *     rows with an X/Y literal first (X-block), then Z/I-only rows (Z-block).
 *   - Pauli literals use two bits per qubit, 00=I 01=Z 10=X 11=Y (Sec. II-B).
 *
 * Conventions shared by every entry point:
 *   - Qubit q is bit q of a basis index (qubit 0 = least significant bit).
 *     W = ceil(n/64) 64-bit words hold one row half or one phase vector; bit r
 *     of word r/64 is row r.  sigma bit r = 1 means the sign of row r is -1.
 *   - Exported amplitudes follow one canonical phase convention: psi_j has
 *     amplitude 2^{-r/2} (real, positive) at its anchor, the basis state in its
 *     support whose bits at every X-block pivot qubit are 0 (r = X-block size).
 *     With this convention the exported frame is unique for a given state.
 *   - Ownership: a handle owns all of its device memory.  Host pointers passed
 *     in are owned by the caller and are only read or written during the call.
 *   - Errors: every entry point returns an sf_status; no C++ exception crosses
 *     the ABI.  sf_last_error() gives a message.
 *   - Asynchrony: calls are stream-ordered on the handle's CUDA stream and
 *     return without waiting for the GPU unless marked "synchronises".
 *     Errors found on the device (capacity exceeded, an internal check) are
 *     deferred: the failing kernel leaves the frame as it was before that
 *     call, every later kernel of the handle does nothing until the error is
 *     reported, and the next synchronising call returns it and clears it.
 *     The frame is then the one from before the failing call; asynchronous
 *     calls made between the failure and the report were dropped.
 *   - Threads: a handle is not thread-safe.  Distinct handles on distinct
 *     streams are independent.
 */
#ifndef SF_ABI_H_
#define SF_ABI_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sf_frame_s* sf_handle;

typedef enum {
    SF_OK = 0,
    SF_EINVAL = 1,     /* bad argument (qubit out of range, q0 == q1, unknown kind, NULL) */
    SF_ENOMEM = 2,     /* device or pinned host allocation failed */
    SF_ECAPACITY = 3,  /* a branch or cofactor would exceed max_elems */
    SF_ECUDA = 4,      /* a CUDA runtime call failed */
    SF_ETIMEOUT = 5,   /* a bounded device wait ran out (hash probe limit) */
    SF_ESTATE = 6,     /* operation invalid in the current state (e.g. collapse onto p = 0) */
    SF_EINTERNAL = 7   /* a device-side consistency check of the tableau algebra failed */
} sf_status;

/* Clifford gate kinds.  H, S (the paper's P) and CNOT are Table 2 of the paper;
 * the rest are products of those. */
enum { SF_H = 0, SF_S = 1, SF_SDG = 2, SF_X = 3, SF_Y = 4, SF_Z = 5,
       SF_CNOT = 6 /* control q0, target q1 */, SF_CZ = 7, SF_SWAP = 8 };

typedef struct { uint32_t kind, q0, q1, pad; } sf_gate; /* q1 ignored for one-qubit kinds */

/* Diagonal non-Clifford kinds (Sec. IV). */
enum { SF_T = 0,      /* diag(1, e^{i pi/4}) on q0 */
       SF_TDG = 1,    /* diag(1, e^{-i pi/4}) on q0 */
       SF_PHASE = 2,  /* diag(1, e^{i theta}) on q0 */
       SF_CPHASE = 3  /* controlled phase R(theta), Eq. 3: diag(1,1,1,e^{i theta}) on (q0, q1) */ };

/* Create a frame for |0...0> (M = RREF{Z_0..Z_{n-1}}, one element sigma = 0,
 * a = 1) on `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 * 1 <= n_qubits <= 1024.  max_elems bounds the number of frame elements that
 * any step may hold, including the children of a branch before coalescing.
 * Device memory: about max_elems * (40 W + 88) bytes plus O(n^2) for the
 * tableau.  Synchronises. */
sf_status sf_create(uint32_t n_qubits, uint64_t max_elems, void* cuda_stream, sf_handle* out);

/* Device bytes that sf_create(n_qubits, max_elems, ...) allocates (0 for
 * arguments sf_create rejects).  For admission control. */
uint64_t sf_footprint_bytes(uint32_t n_qubits, uint64_t max_elems);

/* Free all device and host memory of the handle.  Synchronises. */
sf_status sf_destroy(sf_handle h);

/* Back to |0...0>, discarding any unreported device error.  Asynchronous. */
sf_status sf_reset(sf_handle h);

/* ROTATE(F, U) for each gate in order (Sec. III): the tableau is conjugated
 * (Table 2), restored to RREF (Invariant 1), and every phase vector receives
 * the resulting affine GF(2) update.  `gates` is a host array of n_gates
 * records, copied before return.  Asynchronous. */
sf_status sf_apply_clifford(sf_handle h, const sf_gate* gates, uint64_t n_gates);

/* As sf_apply_clifford, with `dev_gates` already in device memory (it must
 * stay valid until the stream reaches this call).  Suitable for stream
 * capture into a CUDA graph.  Asynchronous. */
sf_status sf_apply_clifford_device(sf_handle h, const sf_gate* dev_gates, uint64_t n_gates);

/* Diagonal non-Clifford gate (Sec. IV): every element branches into at most
 * two (one-qubit kinds) or four (SF_CPHASE) children along the
 * anticommutation masks of the gate's Z-type Pauli terms.  Children are NOT
 * merged: call sf_coalesce afterwards.  theta is used by SF_PHASE and
 * SF_CPHASE only.  Asynchronous; exceeding max_elems is reported by the next
 * synchronising call. */
sf_status sf_apply_nonclifford(sf_handle h, uint32_t kind, uint32_t q0, uint32_t q1, double theta);

/* sf_apply_nonclifford followed by sf_coalesce(h, drop_eps, NULL), done in one
 * pass: the anticommutation masks of the gate's terms form a group U, so each
 * element looks up its partners sigma ^ u (u in U) in an index of the frame and
 * every output element is computed by exactly one thread, summing its parents'
 * contributions in a fixed order.  Same frame as the two calls; asynchronous. */
sf_status sf_apply_nonclifford_coalesce(sf_handle h, uint32_t kind, uint32_t q0, uint32_t q1, double theta,
                                        double drop_eps);

/* TOF_{c1 c2 t} by cofactors (Eq. 2): COFACTOR on c1 and c2 (Sec. III; the
 * frame may double twice, merged as in sf_measure), after which M holds the
 * rows Z_c1 and Z_c2, then X_t applied to the states of the c1 c2 = 11
 * cofactor (the elements whose sign is -1 at both rows): each such phase
 * vector takes the sign flips of the rows that anticommute with X_t, with the
 * exact phase factor, and the amplitude stays in place.  The same state as the
 * Clifford+T decomposition, in fewer passes; M then differs (it holds Z_c1 and
 * Z_c2), so frames are compared after the same sequence of operations.
 * Distinct qubits < n_qubits.  Synchronises (twice, inside the cofactors). */
sf_status sf_apply_toffoli(sf_handle h, uint32_t c1, uint32_t c2, uint32_t t);

/* R(alpha)_{ct} by cofactors (Eq. 3): COFACTOR on c and t, then the states of
 * the ct = 11 cofactor take the factor e^{i alpha}.  Synchronises. */
sf_status sf_apply_cr_cofactor(sf_handle h, uint32_t c, uint32_t t, double alpha);

/* Merge elements with equal phase vectors (summing amplitudes) and drop those
 * with |a| < drop_eps (Def. 1: the phase vectors of a frame are distinct).
 * If out_size is non-NULL the new frame size is written there and the call
 * synchronises; otherwise it is asynchronous. */
sf_status sf_coalesce(sf_handle h, double drop_eps, uint64_t* out_size);

/* Measurement of qubit q in the computational basis (Sec. IV, "Measuring F").
 * If q is random in M the frame is first cofactored on q (COFACTOR, Sec. III):
 * M becomes RREF({rows commuting with Z_q} + {Z_q}), each element splits into
 * its two cofactors, and the frame is coalesced with drop_eps = 1e-12.  Then
 * p0/p1 (nullable) receive the outcome probabilities.  collapse_to = 0 or 1
 * keeps only the consistent states and renormalises; -1 leaves the state
 * as is (it is still cofactored).  Synchronises. */
sf_status sf_measure(sf_handle h, uint32_t q, int32_t collapse_to, double* p0, double* p1);

/* <x|Psi> for the basis state x given as W host words (bit q = qubit q),
 * Observation 1 evaluated on the canonical tableau.  Synchronises. */
sf_status sf_amplitude(sf_handle h, const uint64_t* x_bits, double* re, double* im);

/* Current frame size (number of elements).  Synchronises. */
sf_status sf_size(sf_handle h, uint64_t* k);

/* Wait for all queued work and report any sticky device error.  Synchronises. */
sf_status sf_sync(sf_handle h);

/* Export the canonical tableau: x and z are n*W words each, row-major (row h
 * occupies words [h*W, h*W+W)); n_xblock receives the X-block size r.
 * Synchronises. */
sf_status sf_get_tableau(sf_handle h, uint64_t* x, uint64_t* z, uint32_t* n_xblock);

/* Export the frame in the canonical amplitude convention, sorted ascending by
 * phase vector read as a W-word integer (word W-1 most significant).  sigma
 * receives k*W words (element j at [j*W, j*W+W)), amp receives 2k doubles
 * (re, im).  k receives the frame size; if it exceeds `capacity` nothing is
 * written and SF_ECAPACITY is returned.  Call after sf_coalesce.
 * Synchronises. */
sf_status sf_get_frame(sf_handle h, uint64_t* sigma, double* amp, uint64_t capacity, uint64_t* k);

/* Kernel classes of this library, for sf_time_kernel(). */
enum { SF_K_CLIFFORD = 0,      /* tableau update of a Clifford batch (single CTA) */
       SF_K_AFFINE = 1,        /* per-element affine phase-vector update */
       SF_K_BRANCH = 2,        /* per-element branching, children written unmerged */
       SF_K_BRANCH_MERGE = 3,  /* branching merged through the phase-vector index */
       SF_K_INSERT = 4,        /* generic coalescing: elements hashed into the slot table */
       SF_K_COMPACT = 5,       /* generic coalescing: slot table -> frame, dropping |a| < eps */
       SF_K_INDEX = 6,         /* (re)build of a frame's phase-vector index */
       SF_K_MEASURE_PREP = 7,  /* cofactor planning (single CTA) */
       SF_K_COFACTOR = 8,      /* cofactor split merged through the index */
       SF_K_PROB = 9, SF_K_REDUCE = 10, SF_K_AMP_PREP = 11, SF_K_AMPLITUDE = 12,
       SF_K_FILTER = 13,       /* collapse */
       SF_K_EXPORT = 14, SF_K_RESET = 15,
       SF_K_SEGMENT = 16,      /* sf_apply_program (single CTA) */
       SF_K_COND = 17,         /* the 11-cofactor step of sf_apply_toffoli / sf_apply_cr_cofactor */
       SF_K_GPROG = 18,        /* sf_apply_program_grid (one cooperative launch) */
       SF_K_COUNT_CLASSES = 19 };

/* Number of CUDA kernels this handle has launched since it was created. */
uint64_t sf_kernel_launches(sf_handle h);

/* From now on, bracket every launch of kernel class kernel_id (SF_K_*) with a
 * pair of CUDA events on the handle's stream, forgetting the pairs recorded so
 * far; kernel_id = -1 stops recording and keeps them.  Waits for the stream
 * (so it must not be called while the stream is being captured). */
sf_status sf_time_kernel(sf_handle h, int32_t kernel_id);

/* Device time in milliseconds summed over the event pairs recorded since the
 * last sf_time_kernel, and their number.  Inside a captured CUDA graph each
 * replay records the same pairs again, so read this after every replay.
 * Synchronises. */
sf_status sf_kernel_time(sf_handle h, double* total_ms, uint64_t* launches);

/* The device-side representation, for tests: destabilizer row h is
 * i^{de[h]} P(dx_h, dz_h) (rows laid out as in sf_get_tableau, de has n
 * entries) and g (2 doubles) is the global phase.  Frame element (sigma, a)
 * stands for g a D^sigma phi_0(M), phi_0 being the state stabilized by +M with
 * <0|phi_0> = 2^{-r/2}.  Synchronises. */
sf_status sf_get_internal(sf_handle h, uint64_t* dx, uint64_t* dz, uint32_t* de, double* g);

/* Largest input accepted by sf_coalesce_noalloc. */
#define SF_COALESCE_NOALLOC_MAX_ELEMS 65536u

/* Coalescing of caller-owned device buffers that allocates nothing.  The paper
 * has no counterpart: it is an addition for callers that must not allocate
 * device memory where they merge a frame -- frameworks whose device memory
 * belongs to their own caching pool (little is free outside it, so an extra
 * cudaMalloc may fail, and cudaMalloc/cudaFree may synchronise the device),
 * and serving loops that budget all device memory up front and must not fail
 * half way through a request on an allocation.  It calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *
 * sigma_in: k_in phase vectors of n_words (1..16) 64-bit words each,
 * row-major (element j at [j*n_words, j*n_words+n_words)); amp_in: k_in FP64
 * complex amplitudes (re, im).  Both are device pointers.  Elements with equal
 * phase vectors are merged by summing their amplitudes, and merged elements
 * with |a| < drop_eps are dropped.  Each group is represented by its first
 * element (the smallest input index); the survivors are written to sigma_out /
 * amp_out (device, same layouts, room for k_in elements) in input order, and
 * their number to *k_out (host).  A group's amplitudes are summed with device
 * atomics in an order that depends on scheduling, so two calls on the same
 * input can differ in the last bits of a merged amplitude (far below 1e-10
 * for unit-norm frames).
 *
 * Limits and behaviour: k_in must not exceed SF_COALESCE_NOALLOC_MAX_ELEMS
 * (SF_EINVAL otherwise).  The hash table and accumulators are one fixed
 * __device__ array of about 1.8 MB that every GPU loading this library holds
 * until the process exits; it is shared by all calls on a device and is
 * cleared by each call before use, so calls whose work overlaps on the GPU
 * (different streams or host threads) race and must be ordered by the caller.
 * The first call on each device looks up the array's device address (with that
 * device current) and keeps it; after cudaDeviceReset on that device the
 * entry point must not be called again.  Runs on cuda_stream (a cudaStream_t)
 * and synchronises it to read the output count. */
sf_status sf_coalesce_noalloc(const uint64_t* sigma_in, const double* amp_in, uint64_t k_in, uint32_t n_words,
                              double drop_eps, uint64_t* sigma_out, double* amp_out, uint64_t* k_out,
                              void* cuda_stream);

/* Host-side bookkeeping of the handle: which of its two frame buffers holds
 * the current frame, which buffers carry a valid phase-vector index, what the
 * grid program may assume about the frame's phase vectors, and whether the
 * frame's elements are still where the last grid program left them (a
 * measurement then finds cofactor partners by position).  The token is below
 * 64.  A
 * CUDA graph captured from this handle's stream replays device work only, so
 * read the token right after the capture ends and restore it with
 * sf_set_host_state after every replay, before the next call on the handle. */
uint32_t sf_host_state(sf_handle h);
sf_status sf_set_host_state(sf_handle h, uint32_t token);

/* Words per phase vector / row half used by this handle (ceil(n/64)). */
uint32_t sf_words(sf_handle h);

/* Message for the last error of the handle; NULL handle -> last global error. */
const char* sf_last_error(sf_handle h);

/* ---- Batched campaigns: many small independent circuits in one launch ------
 * The same frame algebra (Sec. III-IV) run on many circuits of n <= 63 qubits
 * at once, one circuit per CTA of a persistent kernel, with the circuit's
 * tableau in registers and its frame in a per-CTA workspace -- for workloads
 * such as fault-injection campaigns, where each circuit is small but there are
 * thousands of them.  Every diagonal gate is merged as in
 * sf_apply_nonclifford_coalesce; measurements are cofactored (COFACTOR,
 * Sec. III), their outcome is drawn from the program and the frame collapsed;
 * classically conditioned Clifford gates read the outcomes so far.
 *
 * A program is an array of sf_op records; circuit c is records
 * [offsets[c], offsets[c+1]).  Op kinds:
 *   0..8        Clifford gate (SF_H..SF_SWAP) on q0 (control) and q1
 *   16 + k      diagonal gate k (SF_T..SF_CPHASE) on q0, q1, angle param;
 *               merged, children with |a| < drop_eps dropped
 *   SF_OP_MEASURE  measure Z on q0 and collapse: outcome 1 iff param < p(1),
 *               param being a uniform draw in [0, 1) made by the caller;
 *               p(1) is the unnormalised probability sum of the frame, and the
 *               survivors are divided by sqrt(p(outcome))
 *   SF_OP_COND  Clifford gate `arg` on q0, q1 applied iff the parity of
 *               (outcome bits & mask) is 1, mask = the 64 bits of param
 *               (bit m = outcome of the circuit's m-th measurement)
 * At most 64 measurements per circuit. */
#define SF_CAMPAIGN_MAX_ELEMS 16384u
enum { SF_OP_DIAG = 16, SF_OP_MEASURE = 32, SF_OP_COND = 33 };

typedef struct {
    uint32_t kind, q0, q1, arg;
    double param; /* angle, draw, or mask bits (memcpy of a uint64_t) */
} sf_op;

/* Largest frame sf_apply_program works on. */
#define SF_SEGMENT_MAX_ELEMS 16384u

/* A program of sf_op records (the record kinds above:
 * Clifford gates, merged diagonal gates, measurements with caller draws,
 * conditional Clifford gates; Sec. III-IV) applied to this handle's frame in
 * ONE launch of a single-CTA kernel, for handles with n_qubits <= 63: the
 * tableau is held in one warp's registers and the frame, while it has at most
 * L = min(max_frame, max_elems, SF_SEGMENT_MAX_ELEMS) elements (max_frame 0:
 * no extra limit), is branched, merged, cofactored and collapsed in place with
 * a shared-memory index.  This replaces one or more grid-wide launches per op
 * while the frame is small; the same frame results as the per-op calls
 * (amplitudes to rounding).  One CTA is faster than the grid-wide kernels only
 * for small frames (a few hundred elements on GB300), hence max_frame.
 *
 * dev_ops: n_ops records in device memory (valid until the stream reaches the
 * call).  The records are checked first (qubits, kinds, at most 64
 * measurements); a bad record fails the call (SF_EINVAL, deferred) with the
 * frame untouched.  The run stops at an op boundary before a diagonal gate or
 * random measurement whose intermediate frame could exceed L.
 * With dev_consumed (device, one uint64) non-NULL the number of records applied
 * is written there and stopping early is not an error: continue with the
 * per-op calls from that record.  With dev_consumed NULL, stopping early is
 * reported as SF_ECAPACITY (deferred), the frame then holding the state after
 * the records that were applied.  dev_meas (device, two uint64, nullable)
 * receives the outcome bits of the program's measurements and their count.
 * Outcomes follow the draw rule of the campaign engine.  Asynchronous. */
sf_status sf_apply_program(sf_handle h, const sf_op* dev_ops, uint64_t n_ops, double drop_eps,
                           uint64_t max_frame, uint64_t* dev_consumed, uint64_t* dev_meas);

/* A program of Clifford and diagonal sf_op records (kinds 0..8 and 16..19;
 * ROTATE and merged branching, Sec. III-IV) applied to this handle's frame, of
 * any size up to max_elems, in ONE cooperative launch over the whole GPU, for
 * handles with n_qubits <= 63.  One persistent CTA per SM walks the records; a
 * Clifford run is applied to the tableau by one warp, a run of diagonal
 * records is planned at once (one CTA per record), and the records are then
 * applied in passes over the frame separated by grid barriers.  A diagonal
 * gate whose anticommutation mask is not spanned by the differences of the
 * frame's phase vectors has no partners: its elements write both children in
 * place, and the following gates that keep those pairs are applied in the same
 * pass; other gates are merged through the phase-vector index as in
 * sf_apply_nonclifford_coalesce.  The same frame results as the per-op calls
 * (amplitudes to rounding; an amplitude between 0 and drop_eps inside a pass
 * is kept to the pass's end, a difference of at most drop_eps).
 *
 * dev_ops: n_ops records in device memory (valid until the stream reaches the
 * call).  The records are checked first (qubits and kinds; measurement and
 * conditional records are accepted); a bad record fails the call (SF_EINVAL,
 * deferred) with the frame untouched.  The run stops before the first
 * measurement or conditional record; dev_consumed (device, one uint64,
 * nullable) receives the number of records applied, so the caller continues
 * with the per-op calls from there.  A frame that would exceed max_elems fails
 * the call (SF_ECAPACITY, deferred), the frame holding the state before the
 * failing record.  A grid barrier that waits longer than the handle's wait
 * limit (sf_set_wait_limit) fails the call with SF_ETIMEOUT (deferred); the
 * tableau and frame are then unspecified until sf_reset.  The frame ends in
 * the handle's current buffer.  Asynchronous; two calls on the same handle are
 * ordered by its stream. */
sf_status sf_apply_program_grid(sf_handle h, const sf_op* dev_ops, uint64_t n_ops, double drop_eps,
                                uint64_t* dev_consumed);

/* A whole program of sf_op records (every kind above: Clifford gates, merged
 * diagonal gates, measurements with caller draws, conditional Clifford gates;
 * Sec. III-IV) from HOST memory, run on this handle.  The records are checked
 * first (SF_EINVAL, nothing applied, for a bad record or more than 64
 * measurements).  For n_qubits <= 63 the library copies them to the device
 * once (through a pinned staging buffer of the handle) and runs each stretch
 * of Clifford and diagonal records as one sf_apply_program_grid launch, a
 * launch that occupies the whole GPU; otherwise it applies them with the
 * per-op calls.  flags = SF_RUN_ONE_CTA is for a GPU shared with other
 * handles' work (e.g. the serving loop below): for n_qubits <= 63 the program
 * then runs from its first record on one CTA (sf_apply_program) while the
 * frame has at most min(max_elems, SF_SEGMENT_MAX_ELEMS) elements, and the
 * per-op calls continue from where it stops, with no whole-GPU launch.  A
 * measurement is made as in the campaign engine: outcome 1 iff the record's
 * draw (param) is below p(1), then the frame is collapsed onto it; a
 * conditional gate applies iff the parity of (outcome bits & mask) is 1.
 * outcomes / n_meas (host, nullable) receive the outcome bits (bit m =
 * measurement m) and their number.  Synchronises at each measurement (the
 * draw needs p(1)) and, with SF_RUN_ONE_CTA, after the one-CTA program;
 * otherwise asynchronous, with deferred device errors as for the calls it
 * makes. */
enum { SF_RUN_ONE_CTA = 1 };
sf_status sf_run_program(sf_handle h, const sf_op* ops, uint64_t n_ops, double drop_eps, uint64_t* outcomes,
                         uint32_t* n_meas, uint32_t flags);

/* Bytes of phase vectors (8 per word) and amplitudes (16) that the passes of
 * the last sf_apply_program_grid launch on this handle read and wrote, each
 * pass counted once: a branch pass reads its k elements and writes 2k, an
 * in-place pass reads k and writes back the amplitudes (and the phase vectors
 * when it applies a Clifford map), a merge reads its input and writes its
 * output, an index build reads the phase vectors; index slots are not
 * counted.  For roofline figures.  Synchronises. */
sf_status sf_grid_program_bytes(sf_handle h, uint64_t* bytes);

/* Tracing of the grid program, for performance analysis.  With on != 0 the
 * next sf_apply_program_grid launches of this handle time each phase (the
 * stretch between two grid barriers) with the GPU's global nanosecond timer.
 * sf_grid_program_trace writes up to cap records of 13 words for the last
 * traced launch, one per phase in order, and their number to *n: what ran
 * (low 4 bits: 3 branch pass along a new direction, 4 in-place pass, 5
 * merge, 6 compaction, 7 index build, 8 Clifford map pass, 10 record check;
 * bits 4..7: records in the pass, mod 16; bits 8..: elements), the time CTA 0
 * began the phase, the time it reached the barrier, the time the last CTA
 * reached it, that CTA's index, then 8 checkpoint times of CTA 0 inside the
 * phase (0 where not reached): Clifford run start and end, planning end, hull
 * update end, pass start, Clifford-map tables end, element loop end, and the
 * time the kept-children counts of the previous pass were read after its
 * barrier.  Synchronises. */
sf_status sf_set_trace(sf_handle h, int32_t on);
sf_status sf_grid_program_trace(sf_handle h, uint64_t* rec, uint32_t cap, uint32_t* n);

/* The planning CTAs of the last traced launch (the tableau CTA applies each
 * step's Clifford run, the plan CTA plans its diagonal records): for planning
 * steps 0..cap-1, 8 times each (global nanosecond timer, 0 where not reached):
 * the tableau CTA's start of the step and its publication; the plan CTA's take
 * of the step's tableau, end of its copy, end of the plans, end of the runs'
 * extents and hull map, end of the hull walk and verdicts, its publication.
 * Synchronises. */
sf_status sf_grid_program_plan_trace(sf_handle h, uint64_t* rec, uint32_t cap);

/* Bounded device waits: a grid barrier of sf_apply_program_grid polls at most
 * `polls` times, about 100 ns apart, before the launch gives up with
 * SF_ETIMEOUT (every CTA leaves at its next barrier; no kernel waits without
 * bound).  The default, SF_WAIT_LIMIT_DEFAULT, is about 0.1 s of waiting; a
 * small value makes a barrier run out on purpose, for tests of the timeout
 * path.  Takes effect at the next launch. */
#define SF_WAIT_LIMIT_DEFAULT 1048576u
sf_status sf_set_wait_limit(sf_handle h, uint32_t polls);

/* Low-rank forms of the per-element maps, for frames of 513..1024 qubits
 * (and 257..512).  The phase-vector map of a Clifford batch (Sec. III, the row
 * operations of Invariant 1) and the cofactor's old-to-new destabilizer map
 * (COFACTOR, Sec. III) differ from the identity by a GF(2) matrix of small rank
 * after one gate or one measurement.  With `on` (the default) a one-CTA kernel
 * factors that difference, and the per-element kernels apply it with
 * 2 r W word operations per element instead of one W-word row per set bit of
 * the phase vector; a rank above 16 falls back to the per-bit form on the
 * device, without a host round trip.  `on` = 0 always takes the per-bit form
 * (the results are identical either way).  Takes effect at the next launch. */
sf_status sf_set_lowrank(sf_handle h, int32_t on);
/* Ranks of the last factorisations: ranks[0] the Clifford batch's map,
 * ranks[1] and ranks[2] the cofactor's U ^ I and V; -1 where the rank exceeded
 * 16, the form was switched off or never computed (always -1 below 257
 * qubits).  ranks[1] is -1 also when V was above the limit.  Synchronises. */
sf_status sf_lowrank_ranks(sf_handle h, int32_t* ranks);

typedef struct sf_campaign_s* sf_campaign;

/* Engine for circuits on n_qubits (1..63) whose frames never exceed
 * max_elems (1..SF_CAMPAIGN_MAX_ELEMS) elements, on cuda_stream.  Allocates a
 * workspace of about (#CTAs x max_elems x 56) bytes, #CTAs = SMs x resident
 * CTAs per SM of the launch shape with the most (see sf_campaign_set_shape).
 * Synchronises. */
sf_status sf_campaign_create(uint32_t n_qubits, uint32_t max_elems, void* cuda_stream, sf_campaign* out);

/* Waits for the engine's stream and frees the workspace. */
sf_status sf_campaign_destroy(sf_campaign c);

/* Runs n_circuits circuits.  All pointers are device pointers, owned by the
 * caller and valid until the stream reaches the launch: dev_ops (sf_op
 * records), dev_offsets (n_circuits + 1 entries).  Per circuit c it writes
 * dev_outcomes[c] (bit m = outcome of measurement m), dev_n_meas[c],
 * dev_k_final[c] (final frame size), dev_norm[c] (sum of |a|^2 of the final
 * frame, times |g|^2 = 1) and dev_status[c] (an sf_status: SF_EINVAL for a bad
 * op, SF_ECAPACITY if a step would exceed max_elems, SF_ESTATE for a collapse
 * onto probability 0, SF_EINTERNAL for a failed tableau check; the circuit
 * stops at its first failing op and the others run on).  If the three export
 * pointers are non-NULL, the final frame of circuit c is written in the
 * canonical convention of sf_get_frame: dev_export_sigma[c * max_elems + j]
 * (one word), dev_export_amp[2 * (c * max_elems + j) + {0, 1}] for
 * j < k_final, in the frame's order (not sorted), and dev_export_tableau[c * 129 + {0..63, 64..127, 128}] = the x
 * words, z words of the canonical rows and the X-block size r.  All three or
 * none.  Results do not depend on the number of CTAs, on the order in which
 * circuits are run or on the other circuits of the batch.  Asynchronous (one
 * memset and one kernel on the stream). */
sf_status sf_campaign_run(sf_campaign c, const sf_op* dev_ops, const uint64_t* dev_offsets, uint32_t n_circuits,
                          double drop_eps, uint64_t* dev_outcomes, uint32_t* dev_n_meas, uint32_t* dev_k_final,
                          double* dev_norm, int32_t* dev_status, uint64_t* dev_export_sigma,
                          double* dev_export_amp, uint64_t* dev_export_tableau);

/* Number of CTAs of the engine's persistent launch in its current shape. */
uint32_t sf_campaign_ctas(sf_campaign c);

/* Shape of the persistent launch: threads per circuit (32, 64, 128 or 256)
 * and where each CTA keeps the hash index of its frame's phase vectors
 * (smem_index = 1: shared memory, fastest probes, fewer CTAs per SM for large
 * max_elems; 0: a per-CTA slice of global memory).  Small threads-per-circuit
 * values run more circuits side by side (the tableau work of a circuit is one
 * warp's); large ones spread big frames over more threads.  For a given shape
 * a circuit's results do not depend on the rest of the batch; across shapes
 * the probability and norm sums are added in a different order, so amplitudes
 * may differ in the last bits.  SF_EINVAL for an unknown shape or one that cannot be
 * resident on this GPU.  The default is 64 threads, index in shared memory
 * when it needs at most 32 KB. */
sf_status sf_campaign_set_shape(sf_campaign c, uint32_t threads_per_circuit, uint32_t smem_index);
sf_status sf_campaign_get_shape(sf_campaign c, uint32_t* threads_per_circuit, uint32_t* smem_index, uint32_t* ctas);

/* Coalescing strategy of the merges (Def. 1: a branch or cofactor output
 * meets the element with the same phase vector): sorted_index = 0 finds it
 * through a hash index of the frame's phase vectors (built with one
 * compare-and-swap per element), 1 through the frame's positions sorted by
 * phase vector (a CTA radix sort over the n phase-vector bits, then binary
 * searches).  Both find the same partners, so the results are bit for bit the
 * same; only the time differs.  The default is the hash index. */
sf_status sf_campaign_set_coalesce(sf_campaign c, uint32_t sorted_index);
uint32_t sf_campaign_get_coalesce(sf_campaign c);

/* Autotuner: runs the given program (device pointers as for sf_campaign_run)
 * once untimed and `reps` (1..16) times timed in every shape (threads per
 * circuit and index location) with each coalescing strategy, keeps the
 * fastest pair, and writes its mean time per run to *best_ms (nullable).  Uses
 * temporary device buffers for the outputs.  Synchronises. */
sf_status sf_campaign_autotune(sf_campaign c, const sf_op* dev_ops, const uint64_t* dev_offsets,
                               uint32_t n_circuits, double drop_eps, uint32_t reps, float* best_ms);

/* ---- Serving: continuous batching of circuits over resident frames ---------
 * A request is one circuit: qubit count, frame capacity, an sf_op program
 * (the record kinds of the campaign engine: Clifford gates, merged diagonal
 * gates, measurements with caller draws, conditional Clifford gates) and up to
 * SF_SERVER_MAX_PROBES basis states whose amplitudes <x|Psi> are returned.
 * sf_server_submit queues it and returns at once.  Up to max_active requests
 * run at a time, each on its own host worker and CUDA stream with its frame
 * resident on the device from the first gate batch to the last; a queued
 * request is admitted as soon as a slot is free and its device footprint
 * (sf_footprint_bytes) fits in the HBM budget next to what the slots hold, in
 * arrival order except that a request that does not fit may be passed by later
 * ones (at most 8 times).  Slots keep their frame handle for the next request
 * of the same qubit count and no larger capacity.  Results are the ones
 * sf_create ... sf_apply_* ... sf_amplitude give for the circuit alone. */
#define SF_SERVER_MAX_PROBES 4

typedef struct {
    uint32_t n_qubits;      /* 1..1024 */
    uint32_t n_probes;      /* 0..SF_SERVER_MAX_PROBES */
    uint64_t max_elems;     /* frame capacity, as for sf_create */
    double drop_eps;        /* merge threshold of every diagonal gate */
    const sf_op* ops;       /* host, n_ops records; copied by sf_server_submit */
    uint64_t n_ops;
    const uint64_t* probes; /* host, n_probes x ceil(n_qubits/64) words; copied */
} sf_request;

typedef struct {
    uint64_t id;
    int32_t status;         /* sf_status of the run */
    uint32_t n_meas;
    uint64_t outcomes;      /* bit m = outcome of measurement m */
    uint64_t k_final;       /* final frame size */
    double t_submit, t_start, t_done;  /* seconds on the server clock */
    uint32_t n_probes;
    uint32_t pad;
    double amp[2 * SF_SERVER_MAX_PROBES];  /* (re, im) of <probe_p|Psi> */
} sf_result;

typedef struct {
    uint32_t queued, active;
    uint64_t bytes_in_use, submitted, completed;
} sf_server_stats;

typedef struct sf_server_s* sf_server;

/* max_active (1..256) slots on the current device, HBM budget in bytes for
 * the frames the slots hold.  Starts the workers. */
sf_status sf_server_create(uint64_t hbm_budget_bytes, uint32_t max_active, sf_server* out);
/* Queue a request (thread-safe, does not wait); *id (nullable) receives its
 * id.  SF_ENOMEM if its footprint exceeds the whole budget. */
sf_status sf_server_submit(sf_server s, const sf_request* r, uint64_t* id);
/* Move up to max_results completed results (in completion order) to out;
 * returns how many.  Does not wait. */
uint32_t sf_server_poll(sf_server s, sf_result* out, uint32_t max_results);
/* Wait until every submitted request has completed (timeout_s < 0: no limit;
 * SF_ETIMEOUT when it runs out). */
sf_status sf_server_wait(sf_server s, double timeout_s);
sf_status sf_server_stats_get(sf_server s, sf_server_stats* st);
/* Seconds since sf_server_create: the clock of t_submit / t_start / t_done. */
double sf_server_clock(sf_server s);
/* Stop the workers after their current request and free every frame. */
sf_status sf_server_destroy(sf_server s);

#ifdef __cplusplus
}
#endif

#endif /* SF_ABI_H_ */
