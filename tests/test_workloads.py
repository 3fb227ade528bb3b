"""Pins of the input recipe (paper_1308_0653_gb300/workloads.py): the seeded
generator against SplitMix64's published output, and each workload against
the shapes its docstring states (the paper's runs and the configurations the
benchmark and the parity tests use)."""
import math

import numpy as np
import pytest

from paper_1308_0653_gb300 import workloads as W


def test_splitmix64_finaliser_gives_the_published_sequence():
    """SplitMix64 from state 0: the first two outputs of the reference
    implementation are 0xe220a8397b1dcdaf and 0x6e789e6aa1b965f4."""
    g = 0x9E3779B97F4A7C15
    z = W._mix64(np.array([g, (2 * g) & ((1 << 64) - 1)], dtype=np.uint64))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_uniform_streams_are_reproducible_independent_and_uniform():
    a = W.uniform(0, 1, 100000)
    assert np.array_equal(a, W.uniform(0, 1, 100000))
    assert not np.array_equal(a[:100], W.uniform(0, 2, 100)) and not np.array_equal(a[:100], W.uniform(1, 1, 100))
    assert 0.0 <= a.min() and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.005 and abs(a.var() - 1 / 12) < 0.002
    assert all(W.uniform_at(3, 7, i) == W.uniform(3, 7, i + 1)[-1] for i in (0, 1, 17, 999))


def test_explosion_recipe():
    w = W.explosion(128, 64, nsteps=10, seed=0)
    r, _ = W.grid(128, 64, w.params["r_in"], w.params["r_out"])
    hot = r < 0.2
    assert np.all(w.fields["T"][hot] == 1.6) and np.all(w.fields["T"][~hot] == 1.0)
    assert np.all(w.fields["lam"][hot] == 1.0) and np.all(w.fields["lam"][~hot] == 0.0)
    base = np.where(hot, 1.4, 1.0)
    noise = w.fields["rho"] / base - 1.0
    assert np.abs(noise).max() <= 0.01 and np.abs(noise).max() > 0.009  # 1 % white noise
    assert np.all(w.fields["ur"] == 0) and np.all(w.fields["uth"] == 0)
    assert (w.params["omega1"], w.params["omega2"], w.params["tau"], w.params["dt"]) == (2.0, 2.0, 1e-3, 1e-5)


def test_implosion_recipe():
    w = W.implosion(256, 256, nsteps=10, seed=0)
    r, _ = W.grid(256, 256, w.params["r_in"], w.params["r_out"])
    out = w.fields["lam"] == 1.0
    # the shocked ring lies outside r_s(theta) = 0.9 (1 +- 0.5 %)
    assert np.all(r[out] > 0.9 * 0.995) and np.all(r[~out] <= 0.9 * 1.005)
    assert np.all(w.fields["ur"][out] == -0.5) and np.all(w.fields["rho"][out] == 1.4)
    assert np.all(w.fields["T"][~out] == 1.0)
    # the front really is perturbed (modes 4..16): its radius varies with theta
    front = [r[m][out[m]].min() for m in range(256)]
    assert max(front) - min(front) >= r[0, 1] - r[0, 0]


@pytest.mark.parametrize("nr,ntheta,seed", [(256, 256, 0), (200, 96, 3), (33, 7, 5)])
def test_implosion_front_follows_its_formula_at_every_site(nr, ntheta, seed):
    """The shocked region is exactly r > r_s(theta) with r_s = 0.9 [1 + 0.005
    sum_q a_q cos(q theta + phi_q) / sum a_q], q = 4..16, a_q from stream 2 and
    phi_q / 2 pi from stream 3, evaluated here site by site."""
    w = W.implosion(nr, ntheta, nsteps=0, seed=seed)
    r, th = W.grid(nr, ntheta, w.params["r_in"], w.params["r_out"])
    a = W.uniform(seed, 2, 13)
    phi = 2.0 * math.pi * W.uniform(seed, 3, 13)
    q = np.arange(4, 17)
    rs = np.empty((ntheta, nr))
    for m in range(ntheta):
        for j in range(nr):
            rs[m, j] = 0.9 * (1.0 + 0.005 * (a * np.cos(q * th[m, j] + phi)).sum() / a.sum())
    assert np.array_equal(w.fields["lam"] == 1.0, r > rs)


def test_batch_recipe():
    ws = W.batch(64, seed=0, nsteps=5)
    sides = [w.params["nr"] for w in ws]
    assert all(w.params["nr"] == w.params["ntheta"] for w in ws)
    assert min(sides) >= 128 and max(sides) <= 1024 and len(set(sides)) > 40
    assert sum("explosion" in w.name for w in ws) == 32
    for w in ws:
        s, n = w.meta["ratio"], w.params["nr"]
        assert 1.2 <= s <= 3.0 and 0.5 <= w.params["omega1"] <= 8.0
        # Courant: 0.4 of the limit set by the fastest ring at the innermost radius
        assert w.params["dt"] == pytest.approx(0.4 * min(1.0 / n, 0.05 * 2 * math.pi / n) / 12.5)


def test_arrivals_are_a_poisson_process():
    t = np.array(W.arrivals(20.0, 600.0, seed=0))
    assert np.all(np.diff(t) > 0) and t[-1] < 600.0
    assert len(t) == pytest.approx(12000, rel=0.03)        # rate 20/s
    gaps = np.diff(t)
    assert gaps.mean() == pytest.approx(0.05, rel=0.03)
    assert gaps.std() == pytest.approx(0.05, rel=0.05)      # exponential: std = mean


def test_serving_requests_span_the_stated_ranges():
    ws = []
    for k in range(0, 400, 7):  # keep the metadata only (fields of 2048^2 sides are 168 MB)
        w = W.serving_request(k, seed=0)
        w.fields = None
        ws.append(w)
    sides = np.array([w.params["nr"] for w in ws])
    steps = np.array([w.nsteps for w in ws])
    assert sides.min() >= 128 and sides.max() <= 2048 and np.all(sides % 32 == 0)
    assert 1000 <= steps.min() and steps.max() <= 20000
    assert np.median(np.log(sides)) == pytest.approx(math.log(512), abs=0.5)   # log-uniform
    assert {w.params["omega1"] for w in ws} == {1.0, 2.0, 4.0}
    kinds = ["explosion" in w.name for w in ws]
    assert 0.25 < np.mean(kinds) < 0.75


def test_paper_disc_runs_use_the_printed_shock_state():
    """Sec. III.C-D: the implosion ring and the explosion driver are the
    printed state (rho, T, |u_r|) = (1.5, 1.55556, 0.666667) into gas at rest
    (1, 1, 0), which for gamma = 2 (P = rho T, c0 = sqrt 2) is the normal
    shock of speed 2, Mach^2 = 2: rho1 = (g+1) M^2 / ((g-1) M^2 + 2) = 3/2,
    P1 = 1 + 2g (M^2 - 1) / (g+1) = 7/3, u1 = D (1 - 1/rho1) = 2/3."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_numbers.json")))["implosion_shock_state"]
    g, D = 2.0, 2.0
    M2 = D * D / g
    rho1 = (g + 1) * M2 / ((g - 1) * M2 + 2)
    P1 = 1 + 2 * g * (M2 - 1) / (g + 1)
    u1 = D * (1 - 1 / rho1)
    assert (gold["rho"], gold["T"], -gold["u_r"]) == pytest.approx((rho1, P1 / rho1, u1), abs=1e-5)
    imp = W.paper_implosion(nr=200)
    ring = imp.fields["lam"] == 1.0
    r, _ = W.grid(200, 1, 0.0, 0.1)
    assert np.array_equal(ring, r > 0.098) and ring.sum() == 4
    exp_ = W.paper_explosion(0.015, 0.3, 600)
    core = exp_.fields["lam"] == 1.0
    for w, sel, sign in ((imp, ring, -1.0), (exp_, core, 1.0)):
        assert np.all(w.fields["rho"][sel] == gold["rho"]) and np.all(w.fields["T"][sel] == gold["T"])
        assert np.all(w.fields["ur"][sel] == sign * abs(gold["u_r"]))
        assert np.all(w.fields["rho"][~sel] == 1.0) and np.all(w.fields["T"][~sel] == 1.0)
        assert np.all(w.fields["ur"][~sel] == 0.0) and np.all(w.fields["uth"] == 0.0)
