"""Serving with continuous batching (dbm_submit / dbm_poll): requests that
arrive while others run join the batch, every result equals the result of
running that request alone (bit for bit), and queue limits, cancellation and
poll timeouts behave as documented (all failures made on the host)."""
import time

import numpy as np
import pytest

from paper_1308_0653_gb300 import dbm
from paper_1308_0653_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)


def _alone(w, nsteps, precision="fp32"):
    sim = dbm.Simulation(dict(w.params, precision=precision))
    sim.init_state(w.fields)
    sim.step(nsteps)
    out = sim.moments(totals=True)
    sim.close()
    return out


def test_results_in_the_mix_equal_results_alone():
    reqs = [(w, n) for w, n in zip(W.batch(7, seed=21, nsteps=0, nmin=48, nmax=260),
                                  [150, 40, 300, 0, 97, 64, 211])]
    srv = dbm.Server(pool_bytes=1 << 30, max_slots=4, quantum=32)
    tickets = []
    for k, (w, n) in enumerate(reqs):
        tickets.append(srv.submit(dict(w.params, precision="fp32"), w.fields, n))
        if k == 3:
            time.sleep(0.05)  # later requests arrive while the first ones run
    for (w, n), t in zip(reqs, tickets):
        st, res = srv.poll(t, timeout_us=60_000_000)
        assert st == dbm.DBM_OK and res["status"] == dbm.DBM_OK
        assert res["steps"] == n
        ref = _alone(w, n)
        for k in dbm.FIELDS:
            assert np.array_equal(res[k], ref[k]), (w.name, k)
        assert np.array_equal(res["totals"], ref["totals"])
        assert res["t_submit"] <= res["t_start"] <= res["t_end"]
    stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["failed"] == 0 and stats["status"] == 0
    srv.close()


def test_queue_limit_cancel_and_poll_timeouts():
    w = W.explosion(256, 256, nsteps=0, seed=22)
    srv = dbm.Server(pool_bytes=1 << 28, max_slots=1, max_queue=2, quantum=32)
    t1 = srv.submit(dict(w.params, precision="fp32"), w.fields, 200000)  # long: occupies the slot
    time.sleep(0.1)
    t2 = srv.submit(dict(w.params, precision="fp32"), w.fields, 10)
    t3 = srv.submit(dict(w.params, precision="fp32"), w.fields, 10)
    with pytest.raises(dbm.DbmError) as e:
        srv.submit(dict(w.params, precision="fp32"), w.fields, 10)   # queue holds 2
    assert e.value.status == dbm.DBM_EBUSY
    assert srv.poll(t2, timeout_us=0)[0] == dbm.DBM_ENOTREADY
    assert srv.poll(t2, timeout_us=1000)[0] == dbm.DBM_ETIMEOUT
    srv.cancel(t3)                                   # queued -> cancelled
    st, res = srv.poll(t3, timeout_us=10_000_000)
    assert st == dbm.DBM_OK and res["status"] == dbm.DBM_ECANCELLED and res["rho"] is None
    srv.cancel(t1)                                   # running -> leaves the batch
    st, res = srv.poll(t1, timeout_us=10_000_000)
    assert st == dbm.DBM_OK and res["status"] == dbm.DBM_ECANCELLED
    assert 0 < res["steps"] < 200000
    st, res = srv.poll(t2, timeout_us=60_000_000)   # the freed slot runs t2
    assert st == dbm.DBM_OK and res["status"] == dbm.DBM_OK and res["steps"] == 10
    assert srv.poll(t2, timeout_us=0)[0] == dbm.DBM_ENOTFOUND  # consumed
    srv.close()


def test_oversized_and_invalid_requests_are_rejected():
    srv = dbm.Server(pool_bytes=1 << 24, max_slots=2)
    big = W.explosion(512, 512, nsteps=0)
    with pytest.raises(dbm.DbmError) as e:
        srv.submit(dict(big.params, precision="fp32"), big.fields, 5)
    assert e.value.status == dbm.DBM_ENOMEM
    w = W.explosion(32, 32, nsteps=0)
    with pytest.raises(dbm.DbmError) as e:
        srv.submit(dict(w.params, precision="fp64"), w.fields, 5)   # precision differs
    assert e.value.status == dbm.DBM_EINVAL
    with pytest.raises(dbm.DbmError) as e:
        srv.submit(dict(w.params, precision="fp32", dt=1.0), w.fields, 5)
    assert e.value.status == dbm.DBM_ECFL
    srv.close()


def test_destroy_with_work_in_flight_cancels_it():
    w = W.explosion(128, 128, nsteps=0, seed=23)
    srv = dbm.Server(pool_bytes=1 << 28, max_slots=2, quantum=32)
    for _ in range(4):
        srv.submit(dict(w.params, precision="fp32"), w.fields, 100000)
    time.sleep(0.05)
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 30


def test_a_failed_batched_step_ends_every_unfinished_request_with_its_error(monkeypatch):
    """Failure injected on the host: the third quantum reports DBM_ECUDA
    instead of launching.  The request that finished in the first quantum
    keeps its result (equal to running it alone); the resident and queued
    ones end with DBM_ECUDA and no arrays, the server refuses new work with
    that status, and it still shuts down."""
    monkeypatch.setenv("DBM_SERVER_FAIL_QUANTUM", "2")
    w = W.explosion(128, 128, nsteps=0, seed=24)
    prm = dict(w.params, precision="fp32")
    srv = dbm.Server(pool_bytes=1 << 28, max_slots=2, quantum=32)
    monkeypatch.delenv("DBM_SERVER_FAIL_QUANTUM")
    short = srv.submit(prm, w.fields, 32)            # all its steps are in quantum 0
    others = [srv.submit(prm, w.fields, 100000) for _ in range(3)]
    st, res = srv.poll(short, timeout_us=60_000_000)
    assert st == dbm.DBM_OK and res["status"] == dbm.DBM_OK and res["steps"] == 32
    ref = _alone(w, 32)
    for k in dbm.FIELDS:
        assert np.array_equal(res[k], ref[k]), k
    for t in others:
        st, res = srv.poll(t, timeout_us=60_000_000)
        assert st == dbm.DBM_OK and res["status"] == dbm.DBM_ECUDA and res["rho"] is None
    stats = srv.stats()
    assert stats["status"] == dbm.DBM_ECUDA
    assert (stats["completed"], stats["failed"], stats["running"], stats["queued"]) == (1, 3, 0, 0)
    with pytest.raises(dbm.DbmError) as e:
        srv.submit(prm, w.fields, 10)
    assert e.value.status == dbm.DBM_ECUDA
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 30
