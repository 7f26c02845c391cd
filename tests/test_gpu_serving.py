"""The serving runtime (continuous batching): requests of uneven size and parameters are
admitted by an HBM budget, prepared by setup workers and swept together; each result must
be bit-identical to bltc_solve of the same request alone, and the runtime's memory must
stay within its budget."""
import numpy as np
import pytest

import oracle
import paper_2003_01836_gb300 as b
from gpu_helpers import gpu_solve, system

pytestmark = pytest.mark.gpu


def _requests(k, seed, nmax_exp=5.0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(round(10 ** rng.uniform(3.0, nmax_exp)))
        kind = "cube" if rng.random() < 0.5 else "plummer"
        ker = int(rng.random() < 0.5)
        kappa = float(rng.uniform(0.1, 1.0)) if ker else 0.0
        theta = float(rng.uniform(0.5, 0.8))
        deg = int(rng.choice([4, 6, 8, 10]))
        leaf = int(rng.choice([500, 1000, 2000]))
        x, y, z, q = system(kind, n, 20031840 + 10000 * i + seed)
        out.append((x, y, z, q, b.params(deg, theta, leaf, leaf, ker, kappa, b.BLTC_PRECISION_MIXED)))
    return out


def test_served_results_equal_solo(gpu):
    reqs = _requests(24, 1)
    solo = [gpu_solve(gpu, *r) for r in reqs]
    # a batching window long enough that requests prepared together are swept together
    srv = b.Server(0, setup_workers=3, max_batch=16, linger_us=200_000)
    try:
        tickets = [srv.submit(*r) for r in reqs]
        outs = [srv.wait(t) for t in tickets]
        for i, ((st, phi, info), ref) in enumerate(zip(outs, solo)):
            assert st == b.BLTC_OK, (i, st)
            assert np.array_equal(phi, ref), f"request {i} differs from its solo solve"
            assert info["t_submit"] <= info["t_admit"] <= info["t_ready"] <= info["t_swept"]
            assert info["t_swept"] <= info["t_copy"] <= info["t_done"]
        s = srv.stats()
        assert s["completed"] == 24 and s["failed"] == 0
        assert s["max_batch"] > 1, "requests were never swept together"
        assert s["peak_live_bytes"] <= s["budget_bytes"]
        assert s["live_bytes"] == 0 and s["reserved_bytes"] == 0
    finally:
        srv.close()


def test_more_requests_in_a_sweep_than_one_launch_holds(gpu):
    # 80 small requests ready together with max_batch 100: the merged sweep runs them in
    # launches of at most 64 argument sets, and every result is still its solo solve's bits
    reqs = _requests(80, 5, nmax_exp=3.3)
    solo = [gpu_solve(gpu, *r) for r in reqs]
    srv = b.Server(0, setup_workers=4, max_batch=100, linger_us=2_000_000, slice_us=0)
    try:
        tickets = [srv.submit(*r) for r in reqs]
        for i, (t, ref) in enumerate(zip(tickets, solo)):
            st, phi, _ = srv.wait(t)
            assert st == b.BLTC_OK and np.array_equal(phi, ref), i
        assert srv.stats()["max_batch"] > 64
    finally:
        srv.close()


@pytest.mark.parametrize("in_flight,setup_blocks", [(1, 0), (2, 0), (1, 8)],
                         ids=["one-slice", "two-slices", "one-slice-free-blocks"])
def test_sliced_sweeps_let_small_requests_pass_a_large_one(gpu, in_flight, setup_blocks):
    # With slices of 2 ms, small requests that become ready while a large sweep runs are
    # swept at the next slice (least remaining work first) and finish before the large one;
    # every result is still its solo solve's bits, with one or two slices enqueued at a time
    # and with block slots left free for the setup workers' kernels.
    big = system("cube", 600000, 20031911) + (b.params(10, 0.5, 2000),)
    small = [system("plummer", 3000, 20031912 + i) + (b.params(6, 0.7, 500),) for i in range(6)]
    solo = [gpu_solve(gpu, *r) for r in [big] + small]
    srv = b.Server(0, setup_workers=2, max_batch=16, slice_us=2000, setup_blocks=setup_blocks,
                   slices_in_flight=in_flight)
    try:
        tb = srv.submit(*big)
        import time
        time.sleep(0.02)                 # the large request is being prepared or swept
        ts = [srv.submit(*r) for r in small]
        outs = [srv.wait(t) for t in [tb] + ts]
        for (st, phi, _), ref in zip(outs, solo):
            assert st == b.BLTC_OK and np.array_equal(phi, ref)
        t_big = outs[0][2]["t_done"]
        assert all(o[2]["t_done"] < t_big for o in outs[1:]), [o[2]["t_done"] - t_big for o in outs]
        assert srv.stats()["sweep_launches"] > 2
    finally:
        srv.close()


def test_served_small_requests_match_oracle(gpu):
    reqs = [r for r in _requests(10, 2, nmax_exp=3.7)][:6]
    srv = b.Server(0, setup_workers=2, max_batch=8)
    try:
        tickets = [srv.submit(*r) for r in reqs]
        for (x, y, z, q, p), t in zip(reqs, tickets):
            st, phi, _ = srv.wait(t)
            assert st == b.BLTC_OK
            ref, _, _ = oracle.bltc(x, y, z, q, p.theta, p.degree, p.leaf_size, p.batch_size,
                                    p.kernel, p.kappa)
            assert oracle.rel_err(ref, phi) <= 1e-6
    finally:
        srv.close()


def test_budget_admission_and_cancel(gpu):
    reqs = _requests(8, 3, nmax_exp=4.5)
    # a budget that holds about one request at a time: admission serialises them
    big = max(400 * r[0].shape[0] for r in reqs) + (40 << 20)
    srv = b.Server(0, setup_workers=2, max_batch=8, hbm_budget_bytes=big * 1.3)
    try:
        tickets = [srv.submit(*r) for r in reqs]
        cancelled = False
        try:
            srv.cancel(tickets[-1])
            cancelled = True
        except b.BltcError as e:
            assert e.status == b.BLTC_ERR_STATE       # already admitted
        for i, t in enumerate(tickets):
            st, phi, info = srv.wait(t)
            if i == len(tickets) - 1 and cancelled:
                assert st == b.BLTC_ERR_CANCELLED
                continue
            assert st == b.BLTC_OK
            assert np.array_equal(phi, gpu_solve(gpu, *reqs[i]))
        s = srv.stats()
        assert s["peak_reserved_bytes"] <= s["budget_bytes"]
        assert s["peak_live_bytes"] <= s["budget_bytes"]
        # a request larger than the whole budget is refused at submission
        x, y, z, q = system("cube", 2_000_000, 5)
        with pytest.raises(b.BltcError) as e:
            srv.submit(x, y, z, q, b.params(8, 0.7, 2000))
        assert e.value.status == b.BLTC_ERR_OOM
    finally:
        srv.close()


def test_submit_rejects_bad_parameters(gpu):
    srv = b.Server(0, setup_workers=1, max_batch=2)
    try:
        x, y, z, q = system("cube", 100, 1)
        for bad in (b.params(0, 0.7, 10), b.params(8, 1.2, 10), b.params(8, 0.7, 10, precision=0)):
            with pytest.raises(b.BltcError) as e:
                srv.submit(x, y, z, q, bad)
            assert e.value.status == b.BLTC_ERR_ARG
        st, _ = b.bltc_server_wait(srv.h, 12345)    # unknown ticket
        assert st == b.BLTC_ERR_ARG
    finally:
        srv.close()


def test_concurrent_setup_of_different_degrees(gpu):
    # Setup workers prepare requests of very different degrees at the same time; the upward
    # kernels' shared-memory limits must not be lowered by one worker while another launches.
    reqs = []
    for i in range(16):
        deg = (2, 16, 10, 4)[i % 4]
        n = 40000 if deg == 16 else 12000
        x, y, z, q = system("cube" if i % 2 else "plummer", n, 20031890 + i)
        reqs.append((x, y, z, q, b.params(deg, 0.6, 6000 if deg == 16 else 1000,
                                          kernel=i % 2, kappa=0.5 if i % 2 else 0.0)))
    srv = b.Server(0, setup_workers=6, max_batch=8)
    try:
        tickets = [srv.submit(*r) for r in reqs]
        for t, r in zip(tickets, reqs):
            st, phi, _ = srv.wait(t)
            assert st == b.BLTC_OK, srv.last_error()
            assert np.array_equal(phi, gpu_solve(gpu, *r))
        assert srv.last_error() == ""
    finally:
        srv.close()
