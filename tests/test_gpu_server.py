"""Serving: many requests in flight on one GPU through ssa_server_*.

A request's results must not depend on what else is in flight: each request
is run alone (a server that admits one request at a time) and again inside a
mixed stream whose memory budget forces queueing, and the two results are
compared.  A few requests are also checked against the oracle, and the
admission rules (budget, arrival order, per-request failures) are checked on
the server's own counters.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_5050_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402
from oracle import ssa_oracle as O  # noqa: E402
from paper_1309_5050_gb300 import _lib as LL  # noqa: E402

GROUPS = [[0], [1, 2]]


def submit(srv, q, seed):
    if q.kind == "1d":
        return srv.submit_series(q.data, q.L, q.rank, groups=GROUPS, residual=True, seed=seed)
    if q.kind == "mssa":
        return srv.submit_multi(q.data, q.L, q.rank, groups=GROUPS, residual=True, seed=seed)
    return srv.submit_image(q.data, q.window[0], q.window[1], q.rank, mask=q.mask, groups=GROUPS,
                            residual=True, seed=seed)


def flat(outs):
    parts = []
    for o in outs:
        if isinstance(o, list):
            parts.extend(np.ravel(v) for v in o)
        else:
            parts.append(np.ravel(o, order="F"))
    return np.concatenate(parts)


def scale(q):
    if q.kind == "mssa":
        return max(float(np.nanmax(np.abs(v))) for v in q.data)
    return float(np.nanmax(np.abs(q.data)))


@pytest.fixture(scope="module")
def stream_requests():
    return W.serving_requests(n=18, rate_hz=1000.0, seed=13, n_max=4000, side_lo=40, side_hi=80)


@pytest.fixture(scope="module")
def alone(stream_requests):
    srv = pkg.Server(max_live=1)
    res = []
    for i, q in enumerate(stream_requests):
        t = submit(srv, q, seed=100 + i)
        srv.drain()
        res.append(srv.take(t))
    srv.close()
    return res


def test_same_alone_and_in_the_mix(stream_requests, alone):
    ests = [r["estimated_bytes"] for r in alone]
    budget = int(3 * np.median(ests))
    srv = pkg.Server(memory_budget=budget)
    tickets = []
    # the stream arrives in three waves while earlier requests are in flight
    waves = np.array_split(np.arange(len(stream_requests)), 3)
    seen_queue_and_live = False
    max_live = 0
    for w in waves:
        for i in w:
            tickets.append(submit(srv, stream_requests[i], seed=100 + i))
        for _ in range(2):
            srv.step()
            st = srv.stats()
            assert st["bytes_live"] <= budget
            max_live = max(max_live, st["live"])
            seen_queue_and_live |= st["queued"] > 0 and st["live"] >= 2
    while True:
        st = srv.stats()
        assert st["bytes_live"] <= budget
        max_live = max(max_live, st["live"])
        seen_queue_and_live |= st["queued"] > 0 and st["live"] >= 2
        if st["queued"] == 0 and st["live"] == 0:
            break
        srv.step()
    assert sorted(srv.finished()) == sorted(tickets)
    mixed = [srv.take(t) for t in tickets]
    assert srv.finished() == []
    srv.close()
    assert max_live >= 2, "requests never shared the GPU"
    assert seen_queue_and_live, "the budget never held a request back"
    # admission in arrival order
    adm = [m["t_admit"] for m in mixed]
    assert all(a <= b for a, b in zip(adm, adm[1:]))
    for q, a, m in zip(stream_requests, alone, mixed):
        assert a["status"] == 0 and m["status"] == 0, (q.rid, a["status"], m["status"])
        assert m["estimated_bytes"] >= m["device_bytes"], (q.rid, m["estimated_bytes"], m["device_bytes"])
        np.testing.assert_allclose(m["sigma"], a["sigma"], rtol=1e-6, atol=0)
        fa, fm = flat(a["outputs"]), flat(m["outputs"])
        ok = ~np.isnan(fa)
        assert np.array_equal(ok, ~np.isnan(fm))
        assert np.max(np.abs(fa[ok] - fm[ok])) <= 1e-5 * scale(q), q.rid


def test_server_matches_oracle(stream_requests, alone):
    kinds_done = set()
    for q, a in zip(stream_requests, alone):
        if q.kind in kinds_done:
            continue
        kinds_done.add(q.kind)
        if q.kind == "1d":
            P = O.Problem.series(q.data, q.L)
        elif q.kind == "mssa":
            P = O.Problem.multi([np.asarray(v, np.float32) for v in q.data], q.L)
        else:
            P = O.Problem.image(q.data, q.window[0], q.window[1], mask=q.mask)
        sig, U, V = O.decompose(P, q.rank)
        # per value 1e-5 relative, plus the Lanczos residual bound 1e-7 sigma_1
        # that limits trailing values of a noise cluster
        assert np.all(np.abs(a["sigma"] - sig) <= 1e-5 * sig + 1e-7 * sig[0]), q.rid
        # reconstruction of the leading component when it is separated by a gap
        if sig[0] / sig[1] >= 1.1:
            ref = O.reconstruct(P, sig, U, V, [[0]])[0]
            got = a["outputs"][0]
            if q.kind == "mssa":
                got = [np.asarray(g).reshape(-1, 1) for g in got]
            elif q.kind == "1d":
                got = [np.asarray(got).reshape(-1, 1)]
            else:
                got = [got]
            for gc, rc in zip(got, ref):
                ok = ~np.isnan(rc)
                assert np.array_equal(ok, ~np.isnan(gc))
                assert np.max(np.abs(gc[ok] - rc[ok])) <= 1e-4 * scale(q)
    assert kinds_done == {"1d", "mssa", "2d"}


def test_request_failures_stay_local():
    budget = 8 << 20
    srv = pkg.Server(memory_budget=budget)
    x = W.series_1d(600, seed=3)
    good = srv.submit_series(x, 300, 6, groups=[[0]], seed=1)
    bad_rank = srv.submit_series(x, 300, 400, groups=[[0]], seed=1)         # rank > min(L, K) = 300
    huge = srv.submit_series(W.series_1d(16000, seed=4), 8000, 50, seed=1)  # larger than the whole budget
    after = srv.submit_series(x, 300, 6, groups=[[0]], seed=1)
    srv.drain()
    rg, rb, rh, ra = srv.take(good), srv.take(bad_rank), srv.take(huge), srv.take(after)
    assert rg["status"] == 0 and rg["sigma"][0] > 0
    assert rb["status"] == LL.SSA_ERANK
    assert rh["estimated_bytes"] > budget and rh["status"] == LL.SSA_ENOMEM
    assert ra["status"] == 0
    np.testing.assert_array_equal(ra["sigma"], rg["sigma"])
    with pytest.raises(pkg.SSAError):
        srv.take(good)           # already taken
    srv.close()


def test_server_fp64():
    srv = pkg.Server(prec="fp64")
    x = W.series_1d(1000, seed=1)
    t = srv.submit_series(x, 500, 10, groups=[[0, 1], [2, 3]], residual=True, seed=5)
    srv.drain()
    r = srv.take(t)
    srv.close()
    sig, U, V = O.decompose(O.Problem.series(x, 500), 10)
    np.testing.assert_allclose(r["sigma"], sig, rtol=1e-9, atol=0)
