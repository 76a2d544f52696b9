"""GPU tests of the continuous-batching server: a request's result is
bit-identical alone and in a mix of geometries, weights, budgets and arrival
times when its group has the same number of slots (within 1e-6 when the
demand-sized groups differ), and matches the FP64 oracle (relative l2 <=
1e-4); admission keeps the device bytes within the HBM budget."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1812_01307_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_01307_gb300 import build
    build.build_library()
    from paper_1812_01307_gb300 import bsgdtv
    bsgdtv.load()
    torch.cuda.set_device(0)
    return bsgdtv


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


GEOMS = {"g64": (64, 60, 91, 10), "g37": (37, 11, 55, 4)}
K = 12
_geo = {}


def geometry(name):
    if name not in _geo:
        n, na, nb, ne = GEOMS[name]
        A = synth.parallel_beam_csr(n, na, nb)
        u, _ = oracle.power_iteration(A)
        _geo[name] = (A, n, ne, 0.9 / (2 * u))
    return _geo[name]


def request(name, seed):
    A, n, ne, _ = geometry(name)
    x = synth.phantom(n, ne, seed)
    return synth.noisy_projections(A, x, seed).astype(np.float32)


# (geometry, seed, lambda, epochs)
MIX = [("g64", 1, 0.05, 14), ("g37", 2, 0.02, 9), ("g64", 3, 0.1, 23), ("g64", 4, 0.03, 5),
       ("g37", 5, 0.08, 17), ("g64", 6, 0.05, 11), ("g37", 7, 0.04, 3), ("g64", 8, 0.07, 19),
       ("g64", 9, 0.02, 8), ("g37", 10, 0.06, 12)]


def _serve(B, reqs, slots=3, max_tick=4, budget=1 << 34, stagger=0, pack=1, priority=1):
    """Runs the requests through one server; submits `stagger` at a time from
    a second thread while the first ones run; pack > 1 lets groups take that
    many geometries.  Returns {index: x}."""
    with B.Server(budget, K, max_tick) as srv:
        srv.set_priority(priority)
        if pack > 1:
            srv.set_packing(pack, 1e9)
            srv.hold(True)   # the whole burst is queued before the first group is made
        gid = {}
        for name in sorted({r[0] for r in reqs}):
            A, n, _, mu = geometry(name)
            gid[name] = srv.add_geometry(A, (n, n), mu, slots=slots, prewarm=0 if pack > 1 else 1)
        ids = {}

        def submit(lo, hi):
            for i in range(lo, hi):
                name, seed, lam, ep = reqs[i]
                ids[i] = srv.submit(gid[name], request(name, seed), lam, ep)

        if stagger:
            assert pack == 1
            submit(0, stagger)
            t = threading.Thread(target=lambda: (time.sleep(0.01), submit(stagger, len(reqs))))
            t.start()
            t.join()
        else:
            submit(0, len(reqs))
        if pack > 1:
            srv.hold(False)
        out = {}
        for i, rid in ids.items():
            x, lat, q = srv.wait(rid, gid[reqs[i][0]], timeout_s=120)
            assert lat >= q >= 0
            out[i] = x
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    return out, st


def test_server_alone_equals_mixed_and_oracle(B):
    mixed, st = _serve(B, MIX, stagger=4)
    assert st["max_running"] >= 2                  # requests did share the device
    for i in (0, 2, 4, 9):
        alone, _ = _serve(B, [MIX[i]])
        assert np.array_equal(alone[0], mixed[i]), i
    for i in (1, 2, 6):
        name, seed, lam, ep = MIX[i]
        A, n, _, mu = geometry(name)
        x_ref, _ = oracle.run(A, request(name, seed).astype(np.float64), (n, n), 1, 1, lam, mu, ep, K)
        assert rel(mixed[i], x_ref) <= 1e-4, i


def test_server_slots_by_l2_rule(B):
    """slots = 0 lets the server size groups by its L2 rule (32 for these small
    images): the mix runs and matches the oracle."""
    out, st = _serve(B, MIX[:6], slots=0)
    assert st["completed"] == 6
    for i in (0, 1, 4):
        name, seed, lam, ep = MIX[i]
        A, n, _, mu = geometry(name)
        x_ref, _ = oracle.run(A, request(name, seed).astype(np.float64), (n, n), 1, 1, lam, mu, ep, K)
        assert rel(out[i], x_ref) <= 1e-4, i


def test_server_priority_changes_no_result(B):
    """Stream priorities by size (the default) and equal priorities give the
    same results bit for bit (two geometries of different sizes)."""
    with_prio, _ = _serve(B, MIX[:6], stagger=3)
    equal, _ = _serve(B, MIX[:6], stagger=3, priority=0)
    for i in range(6):
        assert np.array_equal(with_prio[i], equal[i]), i


def _op_bytes(B, A):
    return (B.bsgdtv_batch_device_bytes(A.rows, A.cols_n, A.nnz, 1)
            - B.bsgdtv_batch_device_bytes(A.rows, A.cols_n, 0, 1))


def test_server_admission_by_hbm_budget(B):
    """A budget that holds both geometries' A but one group's vectors at a
    time: the geometries take turns (idle groups are released), every
    request completes with the same bits."""
    A64, A37 = geometry("g64")[0], geometry("g37")[0]
    vec = max(B.bsgdtv_batch_device_bytes(A.rows, A.cols_n, 0, 3) for A in (A64, A37))
    budget = _op_bytes(B, A64) + _op_bytes(B, A37) + vec + 4096
    reqs = MIX[:6]
    out, st = _serve(B, reqs, budget=budget)
    assert st["groups_made"] >= 3 and st["device_bytes"] <= budget
    ref, _ = _serve(B, reqs)
    for i in out:
        assert np.array_equal(out[i], ref[i])


def test_server_groups_sized_by_demand(B):
    """With up to 16 slots per group, groups are made with as many slots as
    requests wait (4 .. 16); a request's result then depends on its group's
    size only through FP32 rounding: alone vs in the mix <= 1e-6, and both
    match the oracle."""
    mixed, st = _serve(B, MIX, slots=16, stagger=0)
    for i in (0, 3, 7):
        alone, _ = _serve(B, [MIX[i]], slots=16)
        assert rel(alone[0], mixed[i]) <= 1e-6, i
        name, seed, lam, ep = MIX[i]
        A, n, _, mu = geometry(name)
        x_ref, _ = oracle.run(A, request(name, seed).astype(np.float64), (n, n), 1, 1, lam, mu, ep, K)
        assert rel(mixed[i], x_ref) <= 1e-4


def test_server_errors(B):
    A, n, _, mu = geometry("g64")
    with pytest.raises(B.BsgdtvError) as e:       # A and one group exceed the budget
        with B.Server(1 << 20, K) as srv:
            srv.add_geometry(A, (n, n), mu, slots=3)
    assert e.value.code == -2
    with B.Server(1 << 34, K) as srv:
        gid = srv.add_geometry(A, (n, n), mu, slots=2, prewarm=0)
        y = request("g64", 1)
        with pytest.raises(B.BsgdtvError):
            srv.submit(gid + 5, y, 0.05, 3)
        with pytest.raises(B.BsgdtvError):
            srv.submit(gid, y, 0.05, 0)
        bad = y.copy()
        bad[7] = np.nan
        with pytest.raises(B.BsgdtvError) as e:
            srv.submit(gid, bad, 0.05, 3)
        assert e.value.code == -6
        rid = srv.submit(gid, y, 0.05, 400)
        with pytest.raises(B.BsgdtvError) as e:
            srv.wait(rid, gid, timeout_s=0.0)     # still running: timeout, request kept
        assert e.value.code == -5
        x, lat, _ = srv.wait(rid, gid, timeout_s=120)
        assert np.all(np.isfinite(x)) and lat > 0


def _poll_until(srv, rid, state, limit_s=60.0):
    t0 = time.time()
    while srv.poll(rid) != state:
        assert time.time() - t0 < limit_s, (rid, srv.poll(rid))
        time.sleep(0.001)


def test_server_cancel(B):
    """A budget for one group of one slot: a long request runs, a second one
    queues.  Cancelling the queued one takes effect at once, the running one
    at its group's next epoch boundary (the device's slot scheduler reads the
    cancellation from the slot's mailbox); both then wait with
    BSGDTV_ERR_CANCELLED and are forgotten, and the next request reuses the
    slot with the bits it gets alone."""
    A, n, _, mu = geometry("g64")
    budget = _op_bytes(B, A) + B.bsgdtv_batch_device_bytes(A.rows, A.cols_n, 0, 1) + 4096
    with B.Server(budget, K, 4) as srv:
        gid = srv.add_geometry(A, (n, n), mu, slots=1, prewarm=0)
        long_id = srv.submit(gid, request("g64", 1), 0.05, 1 << 30)
        queued_id = srv.submit(gid, request("g64", 2), 0.05, 5)
        _poll_until(srv, long_id, 1)
        assert srv.poll(queued_id) == 0
        srv.cancel(queued_id)
        assert srv.poll(queued_id) == 4
        with pytest.raises(B.BsgdtvError) as e:
            srv.cancel(queued_id)                  # already cancelled
        assert e.value.code == -4
        with pytest.raises(B.BsgdtvError) as e:
            srv.wait(queued_id, gid, timeout_s=1.0)
        assert e.value.code == -8
        with pytest.raises(B.BsgdtvError) as e:
            srv.poll(queued_id)                    # forgotten after the wait
        assert e.value.code == -1
        srv.cancel(long_id)
        with pytest.raises(B.BsgdtvError) as e:
            srv.wait(long_id, gid, timeout_s=60.0)
        assert e.value.code == -8
        rid = srv.submit(gid, request("g64", 3), 0.05, 7)
        x, _, _ = srv.wait(rid, gid, timeout_s=120)
        with pytest.raises(B.BsgdtvError) as e:
            srv.cancel(rid)                        # waited for: unknown
        assert e.value.code == -1
        st = srv.stats()
    assert st["cancelled"] == 2 and st["completed"] == 1 and st["failed"] == 0
    assert st["device_bytes"] <= budget and st["groups_made"] == 1
    alone, _ = _serve(B, [("g64", 3, 0.05, 7)], slots=1)
    assert np.array_equal(x, alone[0])


def test_server_admits_and_retires_between_epochs_of_a_running_group(B):
    """Admission and retirement happen on the device at epoch boundaries: a
    short request submitted while a long one keeps its group running (runs of
    up to 200 epochs) joins that group and completes while the long one is
    still running; its result equals the same request served alone."""
    A, n, _, mu = geometry("g64")
    with B.Server(1 << 34, K, 200) as srv:
        gid = srv.add_geometry(A, (n, n), mu, slots=4, prewarm=1)
        long_id = srv.submit(gid, request("g64", 1), 0.05, 1 << 30)
        _poll_until(srv, long_id, 1)
        time.sleep(0.05)                           # the group is mid-run now
        short_id = srv.submit(gid, request("g64", 4), 0.03, 9)
        x, lat, _ = srv.wait(short_id, gid, timeout_s=120)
        assert srv.poll(long_id) == 1               # the long request is still running
        st = srv.stats()
        assert st["groups_made"] == 1 and st["max_running"] == 2
        srv.cancel(long_id)
        with pytest.raises(B.BsgdtvError) as e:
            srv.wait(long_id, gid, timeout_s=60.0)
        assert e.value.code == -8
    alone, _ = _serve(B, [("g64", 4, 0.03, 9)], slots=4)
    assert np.array_equal(x, alone[0])
    x_ref, _ = oracle.run(A, request("g64", 4).astype(np.float64), (n, n), 1, 1, 0.03, mu, 9, K)
    assert rel(x, x_ref) <= 1e-4


def test_server_armed_wait_times_out(B):
    """An armed epoch whose device-side wait sees no request ends it after the
    limit and reports BSGDTV_ERR_TIMEOUT; the server stays usable."""
    A, n, _, mu = geometry("g37")
    with B.Server(1 << 34, K, 4) as srv:
        gid = srv.add_geometry(A, (n, n), mu, slots=4, prewarm=1)
        t0 = time.time()
        with pytest.raises(B.BsgdtvError) as e:
            srv.arm(gid, 0.05)
        assert e.value.code == -5
        assert time.time() - t0 >= 0.05
        st = srv.stats()
        assert st["armed_epochs"] == 1 and st["wait_timeouts"] == 1
        with pytest.raises(B.BsgdtvError) as e:
            srv.arm(gid, 2.0)                       # beyond the 1 s limit
        assert e.value.code == -1
        rid = srv.submit(gid, request("g37", 2), 0.02, 9)
        x, _, _ = srv.wait(rid, gid, timeout_s=120)
    alone, _ = _serve(B, [("g37", 2, 0.02, 9)], slots=4)
    assert np.array_equal(x, alone[0])


def test_server_armed_wait_admits_a_request(B):
    """A request submitted while an armed epoch waits on the device starts in
    that epoch: the arm reports success, and the result equals the request
    served alone."""
    A, n, _, mu = geometry("g37")
    with B.Server(1 << 34, K, 4) as srv:
        gid = srv.add_geometry(A, (n, n), mu, slots=4, prewarm=1)
        res = {}

        def arm():
            try:
                srv.arm(gid, 0.9)
                res["rc"] = 0
            except B.BsgdtvError as err:
                res["rc"] = err.code

        th = threading.Thread(target=arm)
        th.start()
        t0 = time.time()
        while srv.stats()["armed_epochs"] < 1:     # the armed epoch is on the device
            assert time.time() - t0 < 30
            time.sleep(0.001)
        rid = srv.submit(gid, request("g37", 5), 0.05, 11)
        th.join()
        x, _, _ = srv.wait(rid, gid, timeout_s=120)
        assert res["rc"] == 0
        assert srv.stats()["wait_timeouts"] == 0
    alone, _ = _serve(B, [("g37", 5, 0.05, 11)], slots=4)
    assert np.array_equal(x, alone[0])


def test_server_packs_two_geometries_into_one_group(B):
    """With packing, requests of two geometries waiting together share one
    group (one packed batch): every epoch stage is one launch for both
    (scheduler pair, two passes, two transposes, one FGP launch), and each
    result is bit-identical to the request served alone in an unpacked group
    of the same slot count, and within 1e-4 of the oracle."""
    reqs = MIX[:6]
    mixed, st = _serve(B, reqs, slots=3, pack=2)
    assert st["packed_groups"] >= 1 and st["max_parts"] == 2
    assert st["packed_launches"] == 2 + 2 + 2 + 1
    for i in range(len(reqs)):
        alone, _ = _serve(B, [reqs[i]], slots=3)
        assert np.array_equal(alone[0], mixed[i]), i
    for i in (0, 1):
        name, seed, lam, ep = reqs[i]
        A, n, _, mu = geometry(name)
        x_ref, _ = oracle.run(A, request(name, seed).astype(np.float64), (n, n), 1, 1, lam, mu, ep, K)
        assert rel(mixed[i], x_ref) <= 1e-4, i
