"""GPU tests of the serving handle and of the full-size batched workload.

Serving: requests of mixed sizes and distributions submitted from the host
come back identical to the oracle's hulls, whether collected by polling or
waiting and in any order; a request larger than the memory budget is
refused; statistics are reported.  Batched: the 4096-set workload (sizes
log-uniform in [64, 1e6], about 424M points) in one call, checked exactly
against the oracle on a sample of sets and by the complete verifier on
every set of the sample's complement that the time allows.
"""
import time

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_09417_gb300 as v
    v.load()
    return v


def test_server_matches_oracle(vq):
    reqs = synth.serving_requests(40, rate_per_s=1000.0, lo=100, hi=2_000_000)
    pts = [synth.points(r["dist"], int(r["n"]), int(r["seed"])) for r in reqs]
    with vq.Server(mem_budget_bytes=8 << 30, max_inflight=16) as srv:
        tickets = [srv.submit(x, y) for x, y in pts]
        got = {}
        # collect half by polling (in reverse order), the rest by waiting
        deadline = time.time() + 120
        pending = list(reversed(tickets[: len(tickets) // 2]))
        while pending and time.time() < deadline:
            t = pending.pop()
            res = srv.poll(t, len(pts[tickets.index(t)][0]))
            if res is None:
                pending.insert(0, t)
                time.sleep(0.001)
            else:
                got[t] = res
        assert not pending
        for t in tickets[len(tickets) // 2:]:
            res = srv.wait(t, len(pts[tickets.index(t)][0]), timeout_ms=120_000)
            assert res is not None
            got[t] = res
        st = srv.stats()
    for t, (x, y) in zip(tickets, pts):
        assert np.array_equal(got[t], oracle.hull(x, y)), t
    assert st["hulls_per_s"] > 0
    assert 0 < st["p50_ms"] <= st["p99_ms"]


def test_server_continuous_batching(vq):
    """Requests that arrive while another batch is on the GPU are admitted by
    another lane at once (not after the running batch), finish before it,
    and each result is the same as the request's hull computed alone (and
    the oracle's)."""
    big = synth.points("circle", 40_000_000, 51)   # hull-dense: its batch runs for a while
    small = [synth.points(synth.DISTRIBUTIONS[i % 4], 1000 + 4321 * i, 60 + i) for i in range(20)]
    budget = 6 << 30
    with vq.Server(mem_budget_bytes=budget, max_inflight=64, lanes=3) as srv:
        tb = srv.submit(*big)
        time.sleep(0.02)
        ts = [srv.submit(x, y) for x, y in small]
        done = [srv.wait_any(len(big[0]), timeout_ms=120_000) for _ in range(21)]
        info = srv.info()
    assert all(d is not None for d in done)
    order = [d[0] for d in done]
    res = {d[0]: d[1] for d in done}
    assert sorted(order) == sorted([tb] + ts)
    assert info["admitted_while_busy"] >= 1
    assert info["max_busy_lanes"] >= 2
    assert info["batches"] >= 2
    assert 0 < info["peak_bytes"] <= budget
    assert info["completed"] == 21
    # the first request to finish is one that arrived after the big one
    assert order[0] != tb
    got = [res[t] for t in ts]
    got_big = res[tb]
    for (x, y), g in zip(small, got):
        alone = vq.vq_hull2d(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).cpu().numpy()
        assert np.array_equal(g, alone)
        assert np.array_equal(g, oracle.hull(x, y))
    alone = vq.vq_hull2d(torch.from_numpy(big[0]).cuda(), torch.from_numpy(big[1]).cuda()).cpu().numpy()
    assert np.array_equal(got_big, alone)
    code, bad = oracle.verify(big[0], big[1], got_big)
    assert code == 0, (oracle.VERIFY_CODES.get(code), bad)


def test_server_budget(vq):
    with vq.Server(mem_budget_bytes=64 << 20, max_inflight=4) as srv:
        x, y = synth.points("disk", 2_000_000, 1)  # about 136 MB of device memory: above the budget
        with pytest.raises(vq.VQError) as e:
            srv.submit(x, y)
        assert e.value.status == -7
        x, y = synth.points("square", 10_000, 2)   # fits
        t = srv.submit(x, y)
        assert np.array_equal(srv.wait(t, 10_000, timeout_ms=60_000), oracle.hull(x, y))


@pytest.mark.slow
def test_batched_full_size(vq):
    x, y, offs, dists = synth.batched_sets()  # 4096 sets, seed 5
    nsets = len(offs) - 1
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    hi, ho = vq.vq_hull2d_batched(xd, yd, torch.from_numpy(offs).cuda())
    hi, ho = hi.cpu().numpy(), ho.cpu().numpy()
    del xd, yd
    rng = np.random.default_rng(7)
    exact = set(rng.choice(nsets, 48, replace=False).tolist()) | {0, nsets - 1}
    circle = {s for s in range(nsets) if dists[s] == "circle"}
    for s in sorted(exact):
        a, b = offs[s], offs[s + 1]
        assert np.array_equal(hi[ho[s]:ho[s + 1]], oracle.hull(x[a:b], y[a:b])), s
    # the complete verifier on further sets, circle sets first (hull-dense)
    more = [s for s in sorted(circle) if s not in exact][:32] + [s for s in range(0, nsets, 64) if s not in exact]
    for s in more:
        a, b = offs[s], offs[s + 1]
        code, bad = oracle.verify(x[a:b], y[a:b], hi[ho[s]:ho[s + 1]])
        assert code == 0, (s, oracle.VERIFY_CODES.get(code), bad)
