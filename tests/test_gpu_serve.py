"""Serving: continuous batching of mixed requests (results vs the oracle,
bitwise the same alone and in the mix, admission by free HBM, cancellation,
bounded waits)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import BTCS, EXPLICIT, F32
from paper_2601_12204_b300 import _lib as L
from paper_2601_12204_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_12204_b300.api import Context
    c = Context(0)
    yield c
    c.close()


def _requests(count, seed, nmax=20000, smax=300, nmin=3):
    reqs = W.serving_trace(rate=1e6, duration=1.0, seed=seed, nmin=nmin, nmax=nmax, smin=0,
                           smax=smax, max_requests=count)
    out = []
    for q in reqs:
        dt = oracle.cfl_dt(q.u0, q.dx, q.nu, 0.4) * (1.0 if q.scheme == EXPLICIT else 6.0)
        out.append((q, dt))
    return out


def _oracle(q, dt):
    f = oracle.explicit if q.scheme == EXPLICIT else oracle.btcs
    return f(q.u0, q.bc, q.dx, q.nu, dt, q.nsteps)


def test_serve_mixed_matches_oracle_and_alone(ctx):
    from paper_2601_12204_b300.api import Server
    ctx.set(L.BURGERS_OPT_RESIDENT_MAX, 2048)  # exercise streaming and multi-level rows too
    try:
        sv = Server(ctx, F32, hbm_budget=512 << 20, slice_steps=64)
        reqs = _requests(48, seed=5)
        tickets = [sv.submit(q.scheme, q.bc, q.u0, q.dx, q.nu, dt, q.nsteps) for q, dt in reqs]
        mixed = []
        for (q, dt), t in zip(reqs, tickets):
            rc, out, st = sv.wait(t, q.n, timeout_s=120)
            assert rc == L.BURGERS_OK, L.last_error()
            mixed.append(out.astype(np.float64))
            ref = _oracle(q, dt)
            assert oracle.rel_l2(mixed[-1], ref) <= 1e-5, (q.scheme, q.bc, q.n, q.nsteps)
            assert st.t_submit <= st.t_admit <= st.t_done
        # each request alone gives bitwise the same result
        for (q, dt), m in zip(reqs[:16], mixed[:16]):
            t = sv.submit(q.scheme, q.bc, q.u0, q.dx, q.nu, dt, q.nsteps)
            rc, out, _ = sv.wait(t, q.n, timeout_s=120)
            assert rc == L.BURGERS_OK
            assert np.array_equal(out.astype(np.float64), m)
        s = sv.stats()
        assert s["completed"] == len(reqs) + 16 and s["pool_used_max"] <= s["pool_bytes"]
        assert sv.close() == 0
    finally:
        ctx.set(L.BURGERS_OPT_RESIDENT_MAX, 0)


def test_serve_admission_by_free_memory(ctx):
    """With a pool far smaller than the total state, requests wait for slots
    to free up and still all complete; a request that can never fit is
    refused at submission."""
    from paper_2601_12204_b300.api import Server
    sv = Server(ctx, F32, hbm_budget=4 << 20, slice_steps=32)  # 2 MiB pool
    reqs = _requests(24, seed=6, nmin=20000, nmax=60000, smax=120)
    tickets = [sv.submit(q.scheme, q.bc, q.u0, q.dx, q.nu, dt, q.nsteps) for q, dt in reqs]
    total = sum(q.n * 4 for q, _ in reqs)
    assert total > sv.stats()["pool_bytes"]
    for (q, dt), t in zip(reqs, tickets):
        rc, out, _ = sv.wait(t, q.n, timeout_s=120)
        assert rc == L.BURGERS_OK
        assert oracle.rel_l2(out.astype(np.float64), _oracle(q, dt)) <= 1e-5
    s = sv.stats()
    assert s["pool_used_max"] <= s["pool_bytes"]
    big = np.zeros(1 << 20, np.float32)
    with pytest.raises(Exception):
        sv.submit(EXPLICIT, 0, big, 0.01, 0.01, 1e-4, 10)
    sv.close()


def test_serve_late_arrivals_join_running_work(ctx):
    """A request that arrives while another is on the GPU is admitted before
    the first finishes (continuous batching, not a queue)."""
    from paper_2601_12204_b300.api import Server
    sv = Server(ctx, F32, hbm_budget=256 << 20, slice_steps=16)
    x, dx = W.grid(4096, 0, 0.0, W.TWO_PI)
    u0 = np.sin(x)
    dt = oracle.cfl_dt(u0, dx, 0.05, 0.4)
    ta = sv.submit(BTCS, 0, u0, dx, 0.05, dt * 5, 3000)
    import time
    t0 = time.time()
    while sv.stats()["active"] == 0 and time.time() - t0 < 10:
        time.sleep(0.001)
    tb = sv.submit(EXPLICIT, 0, u0, dx, 0.05, dt, 50)
    rb, _, sb = sv.wait(tb, 4096, timeout_s=120)
    ra, _, sa = sv.wait(ta, 4096, timeout_s=120)
    assert ra == rb == L.BURGERS_OK
    assert sb.t_admit < sa.t_done and sb.t_done < sa.t_done
    sv.close()


def test_serve_cancel_timeout_and_bad_requests(ctx):
    from paper_2601_12204_b300.api import Server
    sv = Server(ctx, F32, hbm_budget=64 << 20, slice_steps=8)
    x, dx = W.grid(2048, 0, 0.0, W.TWO_PI)
    u0 = np.sin(x)
    dt = oracle.cfl_dt(u0, dx, 0.05, 0.4)
    t = sv.submit(BTCS, 0, u0, dx, 0.05, dt, 1_000_000)
    rc, out, _ = sv.wait(t, 2048, timeout_s=0.05)
    assert rc == L.BURGERS_ETIMEOUT and out is None
    assert sv.cancel(t) == L.BURGERS_OK
    rc, out, st = sv.wait(t, 2048, timeout_s=60)
    assert rc == L.BURGERS_ECANCELED and st.status == L.BURGERS_ECANCELED
    rc, _, _ = sv.poll(t, 2048)
    assert rc == L.BURGERS_ENOTFOUND
    with pytest.raises(Exception):
        sv.submit(EXPLICIT, 0, np.zeros(2, np.float32), dx, 0.05, dt, 10)  # n < 3
    with pytest.raises(Exception):
        sv.submit(EXPLICIT, 0, u0, dx, -1.0, dt, 10)  # nu < 0
    t2 = sv.submit(EXPLICIT, 1, u0, dx, 0.05, dt, 0)  # zero steps: returns u0
    rc, out, _ = sv.wait(t2, 2048, timeout_s=60)
    assert rc == L.BURGERS_OK and np.array_equal(out, u0.astype(np.float32))
    assert sv.close() == 0


def test_serve_concurrent_submitters(ctx):
    """Four client threads submit and collect at once (the page-locked arena
    is taken outside the server lock); every result matches the oracle and
    the tickets are distinct."""
    import threading

    from paper_2601_12204_b300.api import Server
    sv = Server(ctx, F32, hbm_budget=256 << 20, slice_steps=32)
    reqs = _requests(96, seed=23, nmax=40000, smax=200)
    parts = [reqs[i::4] for i in range(4)]
    results, errors = [None] * 4, []

    def client(k):
        try:
            mine = [(q, dt, sv.submit(q.scheme, q.bc, q.u0, q.dx, q.nu, dt, q.nsteps))
                    for q, dt in parts[k]]
            outs = []
            for q, dt, t in mine:
                rc, out, _ = sv.wait(t, q.n, timeout_s=120)
                outs.append((q, dt, t, rc, out))
            results[k] = outs
        except Exception as e:  # noqa: BLE001
            errors.append(repr(e))

    try:
        ths = [threading.Thread(target=client, args=(k,)) for k in range(4)]
        for th in ths:
            th.start()
        for th in ths:
            th.join(300)
        assert not errors, errors
        tickets = [t for r in results for (_, _, t, _, _) in r]
        assert len(tickets) == len(reqs) == len(set(tickets))
        for r in results:
            for q, dt, _, rc, out in r:
                assert rc == L.BURGERS_OK, L.last_error()
                assert oracle.rel_l2(out.astype(np.float64), _oracle(q, dt)) <= 1e-5, \
                    (q.scheme, q.bc, q.n, q.nsteps)
    finally:
        sv.close()


def test_serve_submit_timed_replays_a_trace(ctx):
    """burgers_serve_submit_timed submits each request once its arrival time
    has passed, from native code: every request completes (oracle parity),
    the server saw the submissions spread over the trace's 50 ms, each
    lateness is non-negative, and a NULL array is EINVAL."""
    import ctypes
    from paper_2601_12204_b300.api import Server
    sv = Server(ctx, F32, hbm_budget=512 << 20, slice_steps=64)
    reqs = _requests(24, seed=9, nmax=5000)
    u0s = [np.ascontiguousarray(q.u0, dtype=np.float32) for q, _ in reqs]
    arr = (L.burgers_request * len(reqs))()
    for i, ((q, dt), u) in enumerate(zip(reqs, u0s)):
        arr[i] = L.burgers_request(int(q.scheme), int(q.bc), int(q.n), 0, float(q.dx),
                                   float(q.nu), float(dt), int(q.nsteps), u.ctypes.data)
    t_arr = np.linspace(0.0, 0.05, len(reqs))
    tickets, late = sv.submit_timed(arr, t_arr)
    assert len(set(tickets.tolist())) == len(reqs) and np.all(tickets > 0)
    assert np.all(late >= 0.0)
    subs = []
    for (q, dt), t in zip(reqs, tickets.tolist()):
        rc, out, st = sv.wait(t, q.n, timeout_s=120)
        assert rc == L.BURGERS_OK, L.last_error()
        assert oracle.rel_l2(out.astype(np.float64), _oracle(q, dt)) <= 1e-5
        subs.append(st.t_submit)
    assert max(subs) - min(subs) >= 0.045
    rc = sv._lib.burgers_serve_submit_timed(sv.h, None, None, ctypes.c_int64(1), None, None)
    assert rc == L.BURGERS_EINVAL
    assert sv.close() == 0
