"""The serving loop (sf_server_*): each request's result is the one the
one-circuit library path gives for it alone, whether it ran alone or in a mix
of concurrently admitted requests; admission keeps the frames within the HBM
budget; errors stay with their request."""
import time

import numpy as np
import pytest

import oracle
from paper_1712_03554_gb300 import circuits as c

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def sfm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03554_gb300 import sf
    sf.load()
    return sf


def small_stream(seed, count=12, qubits=(8, 70, 130)):
    g = c.rng_for(seed)
    reqs = []
    for i in range(count):
        n = int(qubits[i % len(qubits)])
        ops = c.serving_circuit(seed * 100 + i, n, int(g.integers(200, 600)), int(g.integers(0, 6)))
        # a measurement with a draw and a conditional gate on its outcome
        q = int(g.integers(n))
        ops += [("C", c.H, q, 0), ("M", q, float(g.random())), ("Q", c.X, (q + 1) % n, 0, 1)]
        probes = [0] + [int(g.integers(1 << min(n, 62))) for _ in range(3)]
        reqs.append({"n": n, "ops": ops, "max_elems": 1 << 8, "probes": probes})
    return reqs


def single_path(sfm, r):
    f = sfm.Frame(r["n"], r["max_elems"])
    res = c.run(f, r["ops"])
    amps = [f.amplitude(x) for x in r["probes"]]
    out = {"k_final": f.size(), "amps": amps, "outcomes": sum(x[3] << m for m, x in enumerate(res))}
    f.close()
    return out


def run_server(sfm, reqs, max_active, budget=8 << 30):
    srv = sfm.Server(budget, max_active)
    ids = [srv.submit(r["n"], r["ops"], r["max_elems"], r["probes"]) for r in reqs]
    srv.wait(120.0)
    res = {x["id"]: x for x in srv.poll()}
    srv.close()
    return [res[i] for i in ids]


def test_results_match_single_circuit_path(sfm):
    reqs = small_stream(1)
    got = run_server(sfm, reqs, max_active=4)
    for r, g in zip(reqs, got):
        assert g["status"] == 0
        ref = single_path(sfm, r)
        assert g["k_final"] == ref["k_final"] and g["outcomes"] == ref["outcomes"] and g["n_meas"] == 1
        assert np.max(np.abs(np.array(g["amps"]) - np.array(ref["amps"]))) <= TOL


def test_results_match_oracle(sfm):
    reqs = small_stream(2, count=6, qubits=(8, 12))
    got = run_server(sfm, reqs, max_active=3)
    for r, g in zip(reqs, got):
        o = oracle.FrameOracle(r["n"])
        res = c.run(o, r["ops"])
        assert g["outcomes"] == sum(x[3] << m for m, x in enumerate(res))
        assert g["k_final"] == o.size()
        for a, x in zip(g["amps"], r["probes"]):
            assert abs(a - o.amplitude(x)) <= TOL


def test_alone_equals_mixed(sfm):
    """One slot (each request alone on the GPU) and eight slots (requests
    overlapping on the GPU) give the same results: frame sizes and outcomes
    exactly, amplitudes within 1e-10 (element order inside a frame follows CTA
    scheduling, so sums may differ in the last bits)."""
    reqs = small_stream(3, count=16)
    alone = run_server(sfm, reqs, max_active=1)
    mixed = run_server(sfm, reqs, max_active=8)
    for a, m in zip(alone, mixed):
        assert a["status"] == m["status"] == 0
        assert a["k_final"] == m["k_final"] and a["outcomes"] == m["outcomes"]
        assert np.max(np.abs(np.array(a["amps"]) - np.array(m["amps"]))) <= TOL
    # the mix really overlapped: some request started before another finished
    spans = sorted((m["t_start"], m["t_done"]) for m in mixed)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


def test_admission_respects_budget(sfm):
    """With room for two frames only, at most two are held at any time and
    every request still completes."""
    n, cap = 70, 1 << 14
    fp = sfm.footprint_bytes(n, cap)
    assert fp > 0
    reqs = [{"n": n, "ops": c.serving_circuit(50 + i, n, 300, 4), "max_elems": cap, "probes": [0]}
            for i in range(8)]
    srv = sfm.Server(2 * fp + fp // 2, 8)
    for r in reqs:
        srv.submit(r["n"], r["ops"], r["max_elems"], r["probes"])
    peak = 0
    t0 = time.time()
    while srv.stats()["completed"] < len(reqs) and time.time() - t0 < 120:
        st = srv.stats()
        assert st["bytes_in_use"] <= 2 * fp + fp // 2
        peak = max(peak, st["active"])
        time.sleep(0.001)
    srv.wait(60.0)
    res = srv.poll()
    assert len(res) == len(reqs) and all(x["status"] == 0 for x in res)
    assert peak <= 2
    with pytest.raises(sfm.SFError):  # larger than the whole budget
        srv.submit(n, [], 1 << 24)
    srv.close()


def test_errors_stay_with_their_request(sfm):
    reqs = small_stream(4, count=4)
    bad = {"n": 8, "ops": [("C", c.CNOT, 0, 9)], "max_elems": 16, "probes": [0]}
    over = {"n": 8, "ops": [("C", c.H, q, 0) for q in range(5)] + [x for q in range(5) for x in
                                                                    (("N", c.T, q, 0, 0.0), ("K",))],
            "max_elems": 4, "probes": [0]}
    got = run_server(sfm, reqs[:2] + [bad, over] + reqs[2:], max_active=3)
    assert [g["status"] for g in got] == [0, 0, sfm.SF_EINVAL, sfm.SF_ECAPACITY, 0, 0]
    for r, g in zip(reqs, got[:2] + got[4:]):
        ref = single_path(sfm, r)
        assert g["k_final"] == ref["k_final"]
        assert np.max(np.abs(np.array(g["amps"]) - np.array(ref["amps"]))) <= TOL
