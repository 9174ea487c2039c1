"""Serving loop: requests of mixed size arriving over time run through batched
launches (small) and concurrent streams (large); each result is the same as the
request served alone, and agrees with the plain sequential path."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07187_gb300 import qk, serve

    return qk, serve, torch


def test_each_result_is_the_same_alone_and_in_the_mix(env):
    qk, serve, torch = env
    reqs = [workloads.serving_request(900 + i, n_min=4, n_max=18) for i in range(20)]
    arr = workloads.poisson_arrivals(len(reqs), 400.0, seed=3)
    server = serve.Server(qk, torch, keep_states=True)
    mixed = server.run(reqs, arr)
    assert {r.path for r in mixed} == {"batch", "stream"}
    for i, c in enumerate(reqs):
        alone = serve.Server(qk, torch, keep_states=True).run([c], [0.0])[0]
        assert list(alone.cbits) == list(mixed[i].cbits), c.name
        assert np.max(np.abs(alone.state - mixed[i].state)) <= 1e-6, c.name
    plain = serve.serve_plain(qk, torch, reqs, [0.0] * len(reqs), keep_states=True)
    for i, c in enumerate(reqs):
        assert list(plain[i].cbits) == list(mixed[i].cbits), c.name
        assert np.max(np.abs(plain[i].state - mixed[i].state)) <= 1e-4, c.name
    s = serve.summarize(mixed)
    assert s["requests"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0
