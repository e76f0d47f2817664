/*
 * sf_multiframe.h -- multiframe simulation (Garcia & Markov, "Simulation of
 * Quantum Circuits via Stabilizer Frames", Sec. IV "Multiframe simulation").
 *
 * A multiframe is a list of stabilizer frames with different stabilizer
 * matrices that together represent one state:
 *     Psi = sum over frames F, over elements (sigma, a) of F, a psi_can(M_F, sigma).
 * Each frame is an sf_handle of libsf (include/sf.h) on the multiframe's
 * stream.  Frames hold one-word phase vectors: n_qubits <= 63.
 *
 * COALESCE(F) (Sec. IV): a Z_k-row is a row of the RREF matrix with no X
 * part and a single Z literal, on qubit k.  Two elements are a candidate pair
 * when their phase vectors differ only on Z_k-rows (the set e, qubits
 * v_1 < ... < v_m) and their canonical amplitudes satisfy a_r = i^d a_j
 * (|a_r - i^d a_j| <= 1e-9 |a_j|).  Step 1 sorts the phase vectors by their
 * entries on the other rows, then on the Z_k-rows, each read as a row vector
 * with the first row most significant; the sorted list is walked once from
 * the front and two neighbours that are candidates form a pair.  sigma_j is
 * the member with qubit v_1 in |0>.  The pair becomes the element
 * (sigma_j, sqrt(2) a_j) of the frame with matrix C M C^dagger,
 * C = CNOT_{v1,v2} ... CNOT_{v1,vm} P^d_{v1} H_{v1}; the pairs sharing (e, d)
 * form one new frame.  Frames with equal stabilizer matrices are merged
 * (union, then Def. 1 coalescing of equal phase vectors), and the two steps
 * repeat until no candidate pair is left (Sec. IV, gates on multiframes).
 *
 * Errors are sf_status codes; no call throws.  A failed call leaves the
 * multiframe in an unspecified but destroyable state.  Calls synchronise the
 * stream unless stated otherwise; an operation over all frames enqueues every
 * frame's work and synchronises once per phase.  Not thread-safe per
 * multiframe.
 */
#ifndef SF_MULTIFRAME_H
#define SF_MULTIFRAME_H

#include "sf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sf_multiframe_s* sf_multiframe;

/* A multiframe of one frame in |0...0>.  max_elems: capacity of every frame
 * (each frame is an sf_handle of that capacity; COALESCE handles frames of up
 * to 8192 elements, larger ones fail with SF_ECAPACITY).  max_frames: the
 * most frames the list may hold (SF_ECAPACITY beyond).  n_qubits in [1, 63]
 * (SF_EINVAL otherwise).  cuda_stream: the stream of every frame, or NULL. */
sf_status sf_mf_create(uint32_t n_qubits, uint64_t max_elems, uint32_t max_frames, void* cuda_stream,
                       sf_multiframe* out);
sf_status sf_mf_destroy(sf_multiframe m);

/* Clifford gates on every frame (host array, sf_apply_clifford per frame).
 * Asynchronous.  An invalid gate fails with SF_EINVAL before any frame
 * changes: every frame has the same n, so the first frame rejects it. */
sf_status sf_mf_apply_clifford(sf_multiframe m, const sf_gate* gates, uint64_t n_gates);

/* A diagonal non-Clifford gate (sf_nonclifford_kind) branched and coalesced
 * (Def. 1) in every frame; frames left empty are dropped (one
 * synchronisation).  No multiframe coalescing. */
sf_status sf_mf_apply_nonclifford(sf_multiframe m, uint32_t kind, uint32_t q0, uint32_t q1, double theta,
                                  double drop_eps);

/* Toffoli by cofactors (Eq. 2) / controlled-R(alpha) by cofactors (Eq. 3) in
 * every frame, each frame coalesced (Def. 1, drop_eps), then the multiframe
 * coalesced as sf_mf_coalesce does. */
sf_status sf_mf_apply_toffoli(sf_multiframe m, uint32_t c1, uint32_t c2, uint32_t t, double drop_eps);
sf_status sf_mf_apply_cr(sf_multiframe m, uint32_t c, uint32_t t, double alpha, double drop_eps);

/* Merge frames with equal matrices, then COALESCE every frame and merge again
 * until no candidate pair is left.  drop_eps: amplitudes below it are dropped
 * when merged frames are coalesced.  Outputs (nullable): frames and total
 * elements afterwards. */
sf_status sf_mf_coalesce(sf_multiframe m, double drop_eps, uint32_t* n_frames, uint64_t* n_states);

/* Number of frames and total elements. */
sf_status sf_mf_count(sf_multiframe m, uint32_t* n_frames, uint64_t* n_states);

/* <x|Psi> = sum over frames of sf_amplitude (x: one word, bit q = qubit q). */
sf_status sf_mf_amplitude(sf_multiframe m, const uint64_t* x_bits, double* re, double* im);

/* Frame i (0 <= i < frames) as a borrowed sf_handle, valid until the next
 * call on m; read it with sf_get_tableau / sf_get_frame / sf_size only. */
sf_status sf_mf_frame(sf_multiframe m, uint32_t i, sf_handle* out);

/* Kernel launches made by the multiframe and all its frames so far. */
uint64_t sf_mf_launches(sf_multiframe m);

/* Message of the last failed call on m; NULL m -> the last global error. */
const char* sf_mf_last_error(sf_multiframe m);

#ifdef __cplusplus
}
#endif

#endif /* SF_MULTIFRAME_H */
