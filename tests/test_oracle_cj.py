"""Whole-method pin of the oracle: the steady planar detonation of the
paper's validation run (Sec. III.B) against Chapman-Jouguet theory and the
paper's own printed numbers (tests/golden/paper_numbers.json).

The paper runs nr = 20000 on r in [1000, 1000.1]; the CPU run here uses
nr = 500 (dt = 1e-5, the same Courant numbers) on a full 2 pi grid with
ntheta = 8, which for axisymmetric data is the paper's one-cell pi/4 sector.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1308_0653_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_numbers.json")))


def cj_state(gamma=2.0, Q=1.0, rho0=1.0, P0=1.0):
    """Chapman-Jouguet detonation of an ideal gas with heat release Q
    (textbook closed form; gamma = (D + 2)/D = 2 for the D = 2 model)."""
    c0sq = gamma * P0 / rho0
    D = math.sqrt(c0sq + (gamma ** 2 - 1) * Q / 2) + math.sqrt((gamma ** 2 - 1) * Q / 2)
    rho1 = rho0 * (gamma + 1) * D ** 2 / (gamma * D ** 2 + c0sq)
    u1 = D * (1 - rho0 / rho1)
    P1 = P0 + rho0 * D * u1
    return D, rho1, P1 / rho1, u1


def test_cj_closed_form_matches_the_papers_numbers():
    """The paper's CJ state and speed follow from the closed form with gamma = 2
    and Q = 1 (the paper does not print Q; Q = 1 is the value its numbers need)."""
    D, rho, T, u = cj_state()
    g = GOLD["cj_initial_burnt_state"]
    assert rho == pytest.approx(g["rho"], abs=1e-5)
    assert T == pytest.approx(g["T"], abs=1e-5)
    assert u == pytest.approx(g["u_r"], abs=1e-5)
    assert D == pytest.approx(GOLD["cj_speed"]["value"], abs=1e-5)


@pytest.fixture(scope="module")
def detonation(orc):
    nr, dt = 500, 1e-5
    w = W.planar_cj(nr=nr, dt=dt, t_end=0.025)
    p = orc.make_params(**{k: v for k, v in w.params.items() if k != "precision"})
    f, lam = orc.init(p, w.fields)
    r = 1000.0 + (np.arange(nr) + 0.5) * 0.1 / nr
    n = w.nsteps
    marks = {}
    for s in range(1, n + 1):
        f, lam, _ = orc.step(p, f, lam)
        if s in (int(0.8 * n), n):
            marks[s] = _front(r, lam[0])
    m = orc.macro(p, f, lam)
    D = (marks[n] - marks[int(0.8 * n)]) / ((n - int(0.8 * n)) * dt)
    return dict(r=r, m=m, front=marks[n], D=D)


def _front(r, lam):
    """Position of the lambda = 1/2 crossing (linear interpolation); nan if none."""
    idx = np.nonzero(lam < 0.5)[0]
    if idx.size == 0 or idx[0] == 0 or not np.isfinite(lam).all():
        return float("nan")
    j = int(idx[0])
    return r[j - 1] + (0.5 - lam[j - 1]) / (lam[j] - lam[j - 1]) * (r[j] - r[j - 1])


@pytest.mark.slow
def test_post_front_state_matches_chapman_jouguet(detonation):
    """Behind the reaction zone (0.015 behind the lambda = 1/2 front) the
    burnt state is within 1 % of CJ in rho, T, u_r and P = rho T; the paper
    reports 0.1-0.3 % at 40x finer resolution."""
    D_cj, rho, T, u = cj_state()
    r, m = detonation["r"], detonation["m"]
    assert np.isfinite(detonation["front"]), "no detonation front"
    j = int(np.searchsorted(r, detonation["front"] - 0.015))
    assert m["lam"][0, j] > 0.9999
    assert m["rho"][0, j] == pytest.approx(rho, rel=0.01)
    assert m["T"][0, j] == pytest.approx(T, rel=0.01)
    assert m["ur"][0, j] == pytest.approx(u, rel=0.01)
    assert m["rho"][0, j] * m["T"][0, j] == pytest.approx(rho * T, rel=0.01)
    # axisymmetric data stay axisymmetric: no azimuthal flow, identical rows
    assert np.abs(m["uth"]).max() < 1e-10
    assert np.ptp(m["rho"], axis=0).max() < 1e-10


@pytest.mark.slow
def test_detonation_speed_matches_chapman_jouguet(detonation):
    """The front speed over the last fifth of the run is within 3 % of
    D_CJ = 3.09557 (the paper reports 3.152, 1.8 % above)."""
    assert detonation["D"] == pytest.approx(cj_state()[0], rel=0.03)


@pytest.mark.slow
def test_peak_order_matches_the_paper(detonation):
    """Sec. III.B.2: the maxima of T, P and rho, u_r do not coincide; the paper
    prints R_T < R_P < R_u ~ R_rho with R_rho - R_T = 8.6e-4.  The oracle
    gives the same order and a spacing within 30 % of the paper's."""
    r, m = detonation["r"], detonation["m"]
    assert all(np.isfinite(m[k]).all() for k in m)
    P = m["rho"][0] * m["T"][0]
    R_T, R_P = r[np.argmax(m["T"][0])], r[np.argmax(P)]
    R_rho, R_u = r[np.argmax(m["rho"][0])], r[np.argmax(m["ur"][0])]
    assert R_T < R_P < R_rho
    assert abs(R_u - R_rho) <= 2 * (r[1] - r[0])
    assert (R_rho - R_T) == pytest.approx(1000.08740 - 1000.08654, rel=0.3)
