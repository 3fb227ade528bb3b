"""Mutation check of the oracle's pins: plant one plausible mistake at a time
(a dropped term, a wrong sign, factor or index) in a temporary copy of the
oracle source (the C oracle, or the ZND solver), rebuild it, and require the
pin suite to fail.

Only the temporary copy is changed; the oracle in the tree is untouched.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = [
    ("F_k last-term sign", "- 0.25 * a * b * c * T", "+ 0.25 * a * b * c * T"),
    ("F_0 factor", "F[0] = 1.0 - 8.0 * sum;", "F[0] = 1.0 - sum;"),
    ("f^eq linear term sign", "double term1 = vu / T *", "double term1 = -vu / T *"),
    ("f^eq linear term factor", "double term1 = vu / T * (1.0 - u2 / (2.0 * T));",
     "double term1 = vu / T * (1.0 - u2 / (1.0 * T));"),
    ("f^eq cubic term factor", "(6.0 * T * T * T)", "(2.0 * T * T * T)"),
    ("f^eq quartic term dropped", "(term0 + term1 + term2 + term3 + term4)",
     "(term0 + term1 + term2 + term3)"),
    ("f^eq u^4 factor", "+ u2 * u2 / (8.0 * T * T);", "+ u2 * u2 / (4.0 * T * T);"),
    ("temperature half dropped", "e += 0.5 * f[q * stride]", "e += f[q * stride]"),
    ("u_theta moment index", "jt += fq * vth[q];", "jt += fq * vr[q];"),
    ("M: D T -> T", "(-DIM * T + c2)", "(-T + c2)"),
    ("M: 2Q/D -> 2Q", "(2.0 * Q / DIM)", "(2.0 * Q)"),
    ("M: T^2 -> T", "/ (2.0 * T * T) * (2.0 * Q", "/ (2.0 * T) * (2.0 * Q"),
    ("M dt doubled", "+ M[q] * dt;", "+ M[q] * dt * 2.0;"),
    ("rate a uses omega2", "aa = p->omega1 * pow(P, p->m);", "aa = p->omega2 * pow(P, p->m);"),
    ("rate P = rho", "double P = rho * T;", "double P = rho;"),
    ("ignition gate inverted", "if (T > p->T_th) {", "if (T < p->T_th) {"),
    ("lambda: printed denominator", "((a + b * lam) * E + b * (1.0 - lam))",
     "((a + b * lam) * E + a * (1.0 - lam))"),
    ("lambda: E sign", "double E = exp((a + b) * dt);", "double E = exp(-(a + b) * dt);"),
    ("streaming sign (both)", "- fr_star - ft_star", "+ fr_star + ft_star"),
    ("streaming sign (theta)", "- fr_star - ft_star", "- fr_star + ft_star"),
    ("upwind side swapped (r)", "if (Cr >= 0.0)\n                    fr_star",
     "if (Cr < 0.0)\n                    fr_star"),
    ("C_theta without r", "double Ct = vth[q] * dt / (r * dth);", "double Ct = vth[q] * dt / (dth);"),
    ("C_r scale", "double Cr = vr[q] * dt / dr;", "double Cr = vr[q] * dt / (1.5 * dr);"),
    ("BGK sign", "(fs[q] - feq[q]) * decay", "(feq[q] - fs[q]) * decay"),
    ("BGK rate", "const double decay = exp(-dt / p->tau);",
     "const double decay = exp(-2.0 * dt / p->tau);"),
    ("lambda advection sign", "lr_star = -ur * (lam[s] - l_inner(p, lam, m, j)) / dr * dt;",
     "lr_star = ur * (lam[s] - l_inner(p, lam, m, j)) / dr * dt;"),
    ("lambda theta advection without r",
     "lt_star = -uth * (lam[s] - l_below(p, lam, m, j)) / (r * dth) * dt;",
     "lt_star = -uth * (lam[s] - l_below(p, lam, m, j)) / (dth) * dt;"),
    ("velocity angle sign", "double ang = i * PI / 4.0 - theta;", "double ang = theta - i * PI / 4.0;"),
    ("v_r and v_theta swapped", "vr[vindex(k, i)] = v[k - 1] * cos(ang);\n            vth[vindex(k, i)] = v[k - 1] * sin(ang);",
     "vr[vindex(k, i)] = v[k - 1] * sin(ang);\n            vth[vindex(k, i)] = v[k - 1] * cos(ang);"),
    ("theta wrap", "return f[at(p, N, p->sector ? vrot(q, 1) : q, p->ntheta - 1, j)];",
     "return f[at(p, N, p->sector ? vrot(q, 1) : q, 0, j)];"),
    ("sector wrap rotates the wrong way", "return f[at(p, N, p->sector ? vrot(q, 1) : q, p->ntheta - 1, j)];",
     "return f[at(p, N, p->sector ? vrot(q, -1) : q, p->ntheta - 1, j)];"),
    ("centre rule rotation", "if (p->sector) return f[at(p, N, vrot(q, 4), m, 0)];",
     "if (p->sector) return f[at(p, N, vrot(q, 2), m, 0)];"),
    ("full-disc centre mirror", "return f[at(p, N, q, (m + p->ntheta / 2) % p->ntheta, 0)];",
     "return f[at(p, N, q, m, 0)];"),
    ("r not cell-centred", "return p->r_in + (j + 0.5) * dr;", "return p->r_in + (j) * dr;"),
    ("theta grid shifted", "return m * dtheta_of(p); }", "return (m + 0.5) * dtheta_of(p); }"),
    ("sector span", "return (p->sector ? PI / 4.0 : 2.0 * PI) / p->ntheta;",
     "return (p->sector ? PI / 2.0 : 2.0 * PI) / p->ntheta;"),
    ("lambda clamp bound", "if (ln > 1.0) { ln = 1.0; ++clamped; }", "if (ln > 0.9) { ln = 0.9; ++clamped; }"),
    ("outer ghost reflects", "return f[at(p, N, q, m, j < p->nr - 1 ? j + 1 : p->nr - 1)];",
     "return f[at(p, N, q, m, j < p->nr - 1 ? j + 1 : p->nr - 2)];"),
    ("M*_{3,1} component", "out[7] += 0.5 * gq * s2 * a;", "out[7] += 0.5 * gq * s2 * b;"),
    ("M*_{4,2} factor", "out[9] += 0.5 * gq * s2 * a * a;", "out[9] += gq * s2 * a * a;"),
    ("M*_3 index", "out[5] += gq * a * b * b;", "out[5] += gq * a * a * b;"),
    ("upwind side swapped (theta)", "if (Ct >= 0.0)\n                    ft_star",
     "if (Ct < 0.0)\n                    ft_star"),
    ("lambda upwind side swapped (r)", "if (ur >= 0.0)\n                lr_star",
     "if (ur < 0.0)\n                lr_star"),
    ("lambda upwind side swapped (theta)", "if (uth >= 0.0)\n                lt_star",
     "if (uth < 0.0)\n                lt_star"),
    ("rate b uses exponent m", "bb = p->omega2 * pow(P, p->n);", "bb = p->omega2 * pow(P, p->m);"),
    ("rate b term without (1 - lambda)", "bb * lam * (1.0 - lam)", "bb * lam"),
    ("lambda step numerator sign", "- a * (1.0 - lam)) / ((a + b * lam) * E",
     "+ a * (1.0 - lam)) / ((a + b * lam) * E"),
    ("lambda step E without b", "double E = exp((a + b) * dt);", "double E = exp(a * dt);"),
    ("totals area without r", "double w = r_of(p, j) * dr * dth;", "double w = dr * dth;"),
    ("totals p_y sign of u_theta", "py += rho * (ur * sin(th) + uth * cos(th)) * w;",
     "py += rho * (ur * sin(th) - uth * cos(th)) * w;"),
    ("totals energy without kinetic part", "en += (rho * T + 0.5 * rho * (ur * ur + uth * uth)) * w;",
     "en += (rho * T) * w;"),
    ("f^eq quadratic term factor", "double term2 = vu * vu / (2.0 * T * T) * (1.0 - u2 / (2.0 * T));",
     "double term2 = vu * vu / (2.0 * T * T) * (1.0 - u2 / (4.0 * T));"),
    ("f^eq zeroth term u^2 sign", "double term0 = 1.0 - u2 / (2.0 * T)", "double term0 = 1.0 + u2 / (2.0 * T)"),
    ("f^eq rest weight index", "feq[q] = rho * F[k] *", "feq[q] = rho * F[k == 0 ? 1 : k] *"),
    ("moments: u_r from theta momentum", "double u_r = jr / r, u_t = jt / r;",
     "double u_r = jt / r, u_t = jt / r;"),
    ("moments: T about the origin", "double dr_ = vr[q] - u_r, dt_ = vth[q] - u_t;\n        e +=",
     "double dr_ = vr[q], dt_ = vth[q];\n        e +="),
    ("M: (v - u)^2 without u", "double dr_ = vr[q] - ur, dt_ = vth[q] - uth;\n        double c2",
     "double dr_ = vr[q], dt_ = vth[q];\n        double c2"),
    ("ignition gate not strict", "if (T > p->T_th) {", "if (T >= p->T_th) {"),
    ("consistent R without 1/dt", "R = (lam_react - lam[s]) / dt;", "R = (lam_react - lam[s]);"),
    ("init: lambda not copied", "lam_f[s] = lam[s];", "lam_f[s] = 0.0;"),
    ("inner ghost reflects", "return f[at(p, N, q, m, 0)];\n}", "return f[at(p, N, q, m, 1)];\n}"),
    ("ring speed index", "vr[vindex(k, i)] = v[k - 1] * cos(ang);", "vr[vindex(k, i)] = v[k % 4] * cos(ang);"),
    ("noneq: v* about the origin", "double a = vr[q] - ur, b = vth[q] - uth;  /* v* in polar components */",
     "double a = vr[q], b = vth[q];  /* v* in polar components */"),
    ("noneq: M*_2 r-theta component", "out[1] += gq * a * b;", "out[1] += gq * a * a;"),
    ("noneq: M*_3 rrr factor", "out[3] += gq * a * a * a;", "out[3] += gq * a * a * a * 0.5;"),
    ("noneq: M*_{3,1} theta", "out[8] += 0.5 * gq * s2 * b;", "out[8] += 0.5 * gq * s2 * a;"),
    ("noneq: M*_{4,2} theta-theta", "out[11] += 0.5 * gq * s2 * b * b;", "out[11] += 0.5 * gq * s2 * a * b;"),
    ("noneq: equilibrium part from f", "central_with_velocities(vr, vth, feq, 1, ur, uth, me);",
     "central_with_velocities(vr, vth, f + s, N, ur, uth, me);"),
    ("noneq: sign", "out[c * N + s] = mf[c] - me[c];", "out[c * N + s] = me[c] - mf[c];"),
    ("run: f buffers not swapped", "double *tf = fa; fa = fb; fb = tf;", "/* no swap */"),
    ("run: lambda buffers not swapped", "double *tl = la; la = lb; lb = tl;", "/* no swap */"),
    ("sector wrap above rotates the wrong way", "return f[at(p, N, p->sector ? vrot(q, -1) : q, 0, j)];",
     "return f[at(p, N, p->sector ? vrot(q, 1) : q, 0, j)];"),
    ("theta wrap above to the last row", "return f[at(p, N, p->sector ? vrot(q, -1) : q, 0, j)];",
     "return f[at(p, N, p->sector ? vrot(q, -1) : q, p->ntheta - 1, j)];"),
    ("lambda centre mirror missing",
     "if (p->r_bc_inner == 1 && !p->sector) return lam[(long)((m + p->ntheta / 2) % p->ntheta) * p->nr];",
     "if (p->r_bc_inner == 1 && !p->sector) return lam[(long)m * p->nr];"),
    ("lambda outer ghost reflects", "return lam[(long)m * p->nr + (j < p->nr - 1 ? j + 1 : p->nr - 1)];",
     "return lam[(long)m * p->nr + (j < p->nr - 1 ? j + 1 : p->nr - 2)];"),
    ("lambda inner ghost reflects", "    return lam[(long)m * p->nr];\n}", "    return lam[(long)m * p->nr + 1];\n}"),
    ("lambda theta wrap below", "return lam[(long)(m > 0 ? m - 1 : p->ntheta - 1) * p->nr + j];",
     "return lam[(long)(m > 0 ? m - 1 : 0) * p->nr + j];"),
    ("lambda theta wrap above", "return lam[(long)(m < p->ntheta - 1 ? m + 1 : 0) * p->nr + j];",
     "return lam[(long)(m < p->ntheta - 1 ? m + 1 : p->ntheta - 1) * p->nr + j];"),
    ("F_k T^4 coefficient", "double num = 48.0 * T * T * T * T", "double num = 24.0 * T * T * T * T"),
    ("F_k T^3 coefficient", "- 6.0 * (a + b + c) * T * T * T", "- 8.0 * (a + b + c) * T * T * T"),
    ("F_k T^2 term sign", "+ (a * b + b * c + c * a) * T * T", "- (a * b + b * c + c * a) * T * T"),
    ("F_k denominator without x_k", "double den = x[k] * (x[k] - a)", "double den = (x[k] - a)"),
    ("F_k cyclic index", "int k3 = k + 3 > 4 ? k + 3 - 4 : k + 3;", "int k3 = k + 3 > 4 ? k + 2 - 4 : k + 3;"),
    ("x = v instead of v^2", "x[k] = v[k - 1] * v[k - 1];", "x[k] = v[k - 1];"),
    ("macro: lambda output not copied", "if (lam_out) lam_out[s] = lam[s];", "if (lam_out) lam_out[s] = 0.0;"),
    ("macro: u_r and u_theta swapped", "if (ur) ur[s] = b;\n            if (uth) uth[s] = c;",
     "if (ur) ur[s] = c;\n            if (uth) uth[s] = b;"),
]

ZND_MUTANTS = [
    ("omega1 term uses n", "omega1 * P ** m", "omega1 * P ** n"),
    ("omega2 term without lambda", "omega2 * P ** n * lm)", "omega2 * P ** n)"),
    ("left-point rule", "lm = 0.5 * (lam[i - 1] + lam[i])", "lm = lam[i - 1]"),
    ("larger Hugoniot root", "v = (b - math.sqrt(", "v = (b + math.sqrt("),
    ("enthalpy factor", "g = gamma / (gamma - 1.0)", "g = gamma / (gamma + 1.0)"),
    ("CJ bisection keeps the wrong half", "            hi = mid\n        else:\n            lo = mid",
     "            lo = mid\n        else:\n            hi = mid"),
]

PIN_FILES = ["tests/test_oracle_equilibrium.py", "tests/test_oracle_reaction.py",
             "tests/test_oracle_step.py", "tests/test_oracle_noneq.py", "tests/test_oracle_sector.py",
             "tests/test_oracle_cj.py"]


def _run_pins(name, old, new, source="dbm_oracle.c", pins=PIN_FILES):
    """Run the pin suite on a copy of the oracle with `old` replaced by `new`
    in oracle/<source>; returns pytest's summary line."""
    src = open(os.path.join(ROOT, "oracle", source)).read()
    assert src.count(old) >= 1, f"mutation pattern not found: {name}"
    tmp = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(tmp, "oracle"),
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
        shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(tmp, "tests"),
                        ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutations.py"))
        os.makedirs(os.path.join(tmp, "paper_1308_0653_gb300"))
        for fn in ("__init__.py", "workloads.py"):
            shutil.copy(os.path.join(ROOT, "paper_1308_0653_gb300", fn),
                        os.path.join(tmp, "paper_1308_0653_gb300", fn))
        with open(os.path.join(tmp, "oracle", source), "w") as fh:
            fh.write(src.replace(old, new, 1))
        env = dict(os.environ, ORACLE_THREADS="2")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            *pins], cwd=tmp, capture_output=True, text=True, timeout=900,
                           env=env)
        lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
        return lines[-1] if lines else r.stderr[-200:]
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin():
    control = _run_pins("control", "#include <math.h>", "#include <math.h>")
    assert "passed" in control and "failed" not in control and "error" not in control, control
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        res = dict(zip([m[0] for m in MUTANTS], ex.map(lambda m: _run_pins(*m), MUTANTS)))
    # caught = a pin assertion failed (a build or collection error does not count)
    survivors = {k: v for k, v in res.items() if "failed" not in v}
    assert not survivors, f"mutations not caught by any pin: {survivors}"


def test_every_planted_znd_mistake_fails_a_pin():
    pins = ["tests/test_oracle_znd.py"]
    control = _run_pins("control", "import math", "import math", "znd.py", pins)
    assert "passed" in control and "failed" not in control and "error" not in control, control
    res = {m[0]: _run_pins(*m, "znd.py", pins) for m in ZND_MUTANTS}
    survivors = {k: v for k, v in res.items() if "failed" not in v}
    assert not survivors, f"mutations not caught by any pin: {survivors}"
