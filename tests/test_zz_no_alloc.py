"""sf_coalesce_noalloc against the library's ordinary coalescing.

The allocation-free entry point exists for callers that cannot allocate device
memory where they merge a frame (stream capture into a CUDA graph, frameworks
that own the device memory pool, serving loops with pre-planned memory).  This
file runs last so that a failure here never hides another test's result.  Two
calls are made in a row, the second on a smaller input, so stale scratch
contents from the first call would show up in the second.
"""
import numpy as np
import pytest

from paper_1712_03554_gb300 import circuits as c

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _unmerged_frame(sfm, n, seed, n_t):
    """A frame with repeated phase vectors: T gates applied without coalescing."""
    g = sfm.Frame(n, 1 << 14)
    c.run(g, c.random_clifford(n, 60, seed))
    rng = c.rng_for(seed + 11)
    for _ in range(n_t):
        g.apply_nonclifford(c.T if rng.random() < 0.5 else c.TDG, int(rng.integers(3)))
    return g


def test_noalloc_coalesce_matches_handle_coalesce():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03554_gb300 import sf

    for call, (n, seed, n_t) in enumerate([(12, 3, 9), (7, 5, 6)]):
        g = _unmerged_frame(sf, n, seed, n_t)
        sig, amp = g.frame()            # every element, duplicates included
        k_in = len(sig)
        assert 2 <= k_in <= 2 ** n_t
        assert len({tuple(int(w) for w in s) for s in sig}) < k_in  # there is something to merge
        W = sig.shape[1]
        d_sig = torch.from_numpy(sig.astype(np.uint64).view(np.int64).copy()).cuda()
        d_amp = torch.from_numpy(np.stack([amp.real, amp.imag], axis=1).copy()).cuda()
        o_sig = torch.zeros_like(d_sig)
        o_amp = torch.zeros_like(d_amp)
        stream = torch.cuda.current_stream().cuda_stream
        k_out = sf.coalesce_noalloc(d_sig.data_ptr(), d_amp.data_ptr(), k_in, W, 1e-12, o_sig.data_ptr(),
                                    o_amp.data_ptr(), stream)
        got_sig = o_sig[:k_out].cpu().numpy().view(np.uint64)
        got_amp = o_amp[:k_out].cpu().numpy()
        got = {tuple(int(w) for w in s): complex(a[0], a[1]) for s, a in zip(got_sig, got_amp)}
        assert len(got) == k_out

        # the ordinary entry point on the same frame
        g.coalesce(1e-12)
        ref_sig, ref_amp = g.frame()
        assert k_out == len(ref_sig), (call, k_out, len(ref_sig))
        for s, a in zip(ref_sig, ref_amp):
            key = tuple(int(w) for w in s)
            assert key in got, (call, key)
            assert abs(got[key] - a) <= TOL, (call, key, got[key], a)


def test_noalloc_rejects_oversized_input():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03554_gb300 import sf
    with pytest.raises(sf.SFError) as ei:
        sf.coalesce_noalloc(1, 1, sf.COALESCE_NOALLOC_MAX_ELEMS + 1, 1, 1e-12, 1, 1)
    assert ei.value.code == sf.SF_EINVAL
