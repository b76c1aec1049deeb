"""Continuous batching (GPU): answers of the native server are the same as
each query computed alone, and as the oracle, however the queries were
batched; the server really runs several batches at once."""
import math

import numpy as np
import pytest

import oracle
import paper_1108_0135_gb300 as pm
from paper_1108_0135_gb300 import serve, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pm.load()
    yield


def test_mixed_stream_same_alone_and_in_the_mix():
    rng = np.random.default_rng(11)
    ns = [int(10 ** e) for e in rng.uniform(4, 12, size=48)]
    ns += [ns[3], ns[3], 1, 2, 3, 10**12]          # duplicates and the smallest n
    res = serve.run_stream(ns, max_inflight=4, max_batch=8)
    assert res["stats"]["answered"] == len(ns) and res["stats"]["failed"] == 0
    assert res["stats"]["batches"] >= 4
    assert res["stats"]["max_inflight"] >= 2        # batches overlapped on the device
    table = oracle.mertens_table(2 * 10**7)
    for n, m in zip(ns, res["answers"]):
        assert m == pm.mertens(n), n                # alone
        if n <= 2 * 10**7:
            assert m == table[n], n                 # oracle
    assert res["answers"][-1] == oracle.mertens(10**12, L=10**8)


def test_server_on_resident_table_same_answers():
    """With a resident table attached, batches are planned on it (no sieve);
    answers equal each query alone without a table; targets above the
    table's n_max still get ordinary plans."""
    rng = np.random.default_rng(23)
    ns = [int(10 ** e) for e in rng.uniform(6, 13, size=40)] + [10**13 + 5, 3, 10**6]
    table = pm.mertens_table_create(2**27, 10**13)
    try:
        res = serve.run_stream(ns, max_inflight=4, max_batch=8, table=table)
    finally:
        pm.mertens_table_destroy(table)
    assert res["stats"]["answered"] == len(ns) and res["stats"]["failed"] == 0
    for n, m in zip(ns, res["answers"]):
        assert m == pm.mertens(n), n


def test_open_loop_poisson_arrivals():
    t, n = workloads.serving_stream(seed=5, count=30, lo_exp=8.0, hi_exp=12.0, rate_per_s=200.0)
    res = serve.run_stream(list(n), arrivals_s=t, max_inflight=3, max_batch=16)
    for v, m in zip(n, res["answers"]):
        assert m == pm.mertens(int(v)), int(v)
    assert res["p99_s"] >= res["p50_s"] > 0


def test_server_rejects_bad_queries():
    srv = pm.mertens_server_create(0)
    try:
        with pytest.raises(pm.MertensError):
            pm.mertens_server_submit(srv, 0)
        with pytest.raises(pm.MertensError) as ei:
            pm.mertens_server_submit(srv, 2**63)
        assert ei.value.code == pm.MERTENS_ENOTSUP
        t = pm.mertens_server_submit(srv, 10**9)
        assert pm.mertens_server_wait(srv, t, 60.0) == -222 == oracle.mertens(10**9)
        with pytest.raises(pm.MertensError):
            pm.mertens_server_poll(srv, 987654321)
    finally:
        pm.mertens_server_destroy(srv)
