"""sf_coalesce_noalloc against the oracle's coalescing and the library's own.

The allocation-free entry point is for callers that must not allocate device
memory where they merge a frame: frameworks whose device memory belongs to
their own caching pool, and serving loops that budget all memory up front.
This file runs last so that a failure here never hides another test's result.
Every test makes two calls in a row, the second on a smaller input, so stale
scratch contents from the first call would show up in the second.
"""
import numpy as np
import pytest

from paper_1712_03554_gb300 import circuits as c

pytestmark = pytest.mark.gpu
TOL = 1e-10
EPS = 1e-12


def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _unmerged_frame(sfm, n, seed, n_t):
    """A frame with repeated phase vectors: T gates on three random qubits
    (Z_q anticommutes with a row of M), applied without coalescing."""
    g = sfm.Frame(n, 1 << 14)
    c.run(g, [("C", c.H, q, 0) for q in range(n)] + c.random_clifford(n, 60, seed))
    x, _, _ = g.tableau()
    random_q = [q for q in range(n) if np.any(x[:, q // 64] & (np.uint64(1) << np.uint64(q % 64)))]
    assert len(random_q) >= 3
    rng = c.rng_for(seed + 11)
    targets = [random_q[int(i)] for i in rng.choice(len(random_q), size=3, replace=False)]
    for _ in range(n_t):
        g.apply_nonclifford(c.T if rng.random() < 0.5 else c.TDG, targets[int(rng.integers(3))])
    return g


def _noalloc(sfm, torch, sig, amp):
    """One sf_coalesce_noalloc call on host arrays copied to the device."""
    k_in, W = sig.shape
    d_sig = torch.from_numpy(np.ascontiguousarray(sig, dtype=np.uint64).view(np.int64)).cuda()
    d_amp = torch.from_numpy(np.ascontiguousarray(np.stack([amp.real, amp.imag], axis=1))).cuda()
    o_sig = torch.full_like(d_sig, -1)
    o_amp = torch.full_like(d_amp, np.nan)
    stream = torch.cuda.current_stream().cuda_stream
    k_out = sfm.coalesce_noalloc(d_sig.data_ptr(), d_amp.data_ptr(), k_in, W, EPS, o_sig.data_ptr(),
                                 o_amp.data_ptr(), stream)
    got_sig = o_sig[:k_out].cpu().numpy().view(np.uint64)
    got_amp = o_amp[:k_out].cpu().numpy()
    return got_sig, got_amp[:, 0] + 1j * got_amp[:, 1]


def _oracle_coalesce(n, x, z, sig, amp):
    """The oracle's sort-and-merge (Def. 1) on the same elements."""
    import oracle
    o = oracle.FrameOracle(n)
    o.set_state(x, z, sig, amp)
    o.coalesce(EPS)
    return o.frame()


def _first_occurrence_order(sig, keep):
    seen, order = set(), []
    for s in sig:
        key = tuple(int(w) for w in s)
        if key not in seen:
            seen.add(key)
            if key in keep:
                order.append(key)
    return order


def _check(got_sig, got_amp, ref_sig, ref_amp, in_sig, what):
    got = {tuple(int(w) for w in s): a for s, a in zip(got_sig, got_amp)}
    assert len(got) == len(got_sig), what  # no phase vector twice
    assert len(got_sig) == len(ref_sig), (what, len(got_sig), len(ref_sig))
    for s, a in zip(ref_sig, ref_amp):
        key = tuple(int(w) for w in s)
        assert key in got, (what, key)
        assert abs(got[key] - a) <= TOL, (what, key, got[key], a)
    # survivors come out in the order of their group's first input element
    assert [tuple(int(w) for w in s) for s in got_sig] == _first_occurrence_order(in_sig, set(got)), what


@pytest.mark.parametrize("cases", [[(12, 3, 9), (7, 5, 6)], [(150, 4, 10), (100, 8, 7)], [(200, 6, 8), (64, 2, 5)]])
def test_noalloc_coalesce_matches_oracle_and_handle(cases):
    """Frames with duplicates made by unmerged T branches (one to four words per
    phase vector): the same survivors and sums as the oracle's coalescing and as
    sf_coalesce on the handle."""
    torch = _need_cuda()
    from paper_1712_03554_gb300 import sf

    for call, (n, seed, n_t) in enumerate(cases):
        g = _unmerged_frame(sf, n, seed, n_t)
        sig, amp = g.frame()            # every element, duplicates included
        k_in = len(sig)
        assert 2 <= k_in <= 2 ** n_t
        assert len({tuple(int(w) for w in s) for s in sig}) < k_in  # there is something to merge
        x, z, _ = g.tableau()
        got_sig, got_amp = _noalloc(sf, torch, sig, amp)
        o_sig, o_amp = _oracle_coalesce(n, x, z, sig, amp)
        _check(got_sig, got_amp, o_sig, o_amp, sig, ("oracle", call, n))
        g.coalesce(EPS)
        ref_sig, ref_amp = g.frame()
        _check(got_sig, got_amp, ref_sig, ref_amp, sig, ("handle", call, n))
        g.close()


def _synthetic(n, k_in, n_groups, n_cancel, seed):
    """k_in elements over n_groups distinct phase vectors of n bits (random
    multiplicities), plus n_cancel further phase vectors that occur exactly
    twice with opposite amplitudes, so their sums are exactly zero."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W = (n + 63) // 64
    top = (1 << (n - 64 * (W - 1))) - 1 if n % 64 else (1 << 64) - 1
    pool = rng.integers(0, 1 << 63, size=(n_groups + n_cancel, W), dtype=np.uint64) * np.uint64(2)
    pool ^= rng.integers(0, 2, size=pool.shape, dtype=np.uint64)
    pool[:, W - 1] &= np.uint64(top)
    pool = np.unique(pool, axis=0)
    rng.shuffle(pool)
    groups, cancel = pool[:n_groups], pool[n_groups:n_groups + n_cancel]
    m = k_in - 2 * len(cancel)
    pick = np.concatenate([np.arange(len(groups)), rng.integers(0, len(groups), size=m - len(groups))])
    sig = np.concatenate([groups[pick], cancel, cancel])
    amp = (rng.standard_normal(m) + 1j * rng.standard_normal(m)) / np.sqrt(2.0 * k_in)
    ca = (rng.standard_normal(len(cancel)) + 1j * rng.standard_normal(len(cancel))) / np.sqrt(2.0 * k_in)
    amp = np.concatenate([amp, ca, -ca])
    perm = rng.permutation(len(sig))
    return sig[perm], amp[perm]


def test_noalloc_full_size_with_cancellations():
    """Inputs at the stated maximum (three words per phase vector) and a second,
    smaller call after it: duplicates of random multiplicity, and groups whose
    amplitudes cancel exactly and must vanish, against the oracle."""
    torch = _need_cuda()
    from paper_1712_03554_gb300 import sf

    n = 150
    W = (n + 63) // 64
    x = np.zeros((n, W), dtype=np.uint64)
    z = np.zeros((n, W), dtype=np.uint64)
    for h in range(n):  # M = RREF{Z_0..Z_{n-1}}: every phase vector is a valid state
        z[h, h // 64] = np.uint64(1) << np.uint64(h % 64)
    for call, (k_in, n_groups, n_cancel, seed) in enumerate([(sf.COALESCE_NOALLOC_MAX_ELEMS, 20000, 3000, 1),
                                                             (5000, 1500, 200, 2)]):
        sig, amp = _synthetic(n, k_in, n_groups, n_cancel, seed)
        assert len(sig) == k_in
        got_sig, got_amp = _noalloc(sf, torch, sig, amp)
        o_sig, o_amp = _oracle_coalesce(n, x, z, sig, amp)
        assert len(o_sig) <= n_groups  # every cancelling group is gone
        _check(got_sig, got_amp, o_sig, o_amp, sig, ("synthetic", call))


def test_noalloc_rejects_oversized_input():
    _need_cuda()
    from paper_1712_03554_gb300 import sf
    with pytest.raises(sf.SFError) as ei:
        sf.coalesce_noalloc(1, 1, sf.COALESCE_NOALLOC_MAX_ELEMS + 1, 1, 1e-12, 1, 1)
    assert ei.value.code == sf.SF_EINVAL
