"""Pins of the oracle's artificial viscosity and limiter by hand-worked two-particle cases.

The expected dv/dt and du/dt of every case in tests/golden/hydro_viscosity_hand_worked.json
are derived by hand (each step written out there; sound speeds, pressures, mu, Q and the
limiter value phi as the numbers the derivation gives), with the corrections switched
off (A = 1, B = 0, grad A = grad B = 0) so that the pair force reduces to a closed form.
The cases isolate each term: beta mu^2 alone, alpha cbar mu alone, a receding pair,
eta^2 dominating at small r, an oblique pair, and the van Leer limiter at gradient
ratios 1/2, 2, 1 and -1 (Sec. 5: the Acceleration and Energy kernels).

The second test plants plausible slips in a copy of the oracle's C source (a sum
instead of a mean, eta^2 on r^2, another limiter, ...) and checks that each one fails
at least one case, so the cases do pin those terms.
"""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hydro_viscosity_hand_worked.json")
with open(GOLDEN) as fh:
    DATA = json.load(fh)
CASES = DATA["cases"]


def _expected(case):
    ns = {"pi": math.pi, "sqrt": math.sqrt}
    for name, _why, expr in case["derivation"]:
        ns[name] = eval(expr, {"__builtins__": {}}, ns)
    dv = np.array([[eval(e, {"__builtins__": {}}, ns) for e in row] for row in case["dv"]], dtype=np.float64)
    du = np.array([eval(e, {"__builtins__": {}}, ns) for e in case["du"]], dtype=np.float64)
    return dv, du


def _run(orc, case):
    c = DATA["common"]
    pos = np.array(case["pos"], dtype=np.float64)
    n = pos.shape[0]
    I = orc.Inputs(pos, np.zeros(n, np.uint8), case["m"], case["h"], case["u"], case["v"], c["L"], 3.0, 0.1,
                   np.zeros(6))
    A = np.ones(n)
    B = np.zeros((n, 3))
    gA = np.zeros((n, 3))
    gB = np.zeros((n, 9))
    dvg = np.array(case["dvg"], dtype=np.float64) if "dvg" in case else None
    dv, du, _ = orc.hydro(I, np.array(case["V"], np.float64), np.array(case["rho"], np.float64), A, B, gA, gB,
                          c["gamma"], case["alpha"], case["beta"], c["eta2"], dvg=dvg, brute=True)
    return dv, du


def _mismatch(orc, case):
    dv, du = _run(orc, case)
    edv, edu = _expected(case)
    scale = max(np.abs(edv).max(), 1e-300)
    return max(np.abs(dv - edv).max() / scale, np.abs(du - edu).max() / max(np.abs(edu).max(), 1e-300))


@pytest.mark.parametrize("case", CASES, ids=[c["name"].split(":")[0] for c in CASES])
def test_viscosity_hand_worked(orc, case):
    assert _mismatch(orc, case) < 1e-12, case["name"]


def test_hand_worked_values_are_not_degenerate():
    """Every case moves both particles and heats or cools them: no pin compares zeros."""
    for case in CASES:
        dv, du = _expected(case)
        assert np.all(np.abs(dv).max(axis=1) > 1e-3) and np.all(np.abs(du) > 1e-4), case["name"]


SLIPS = [
    ("cbar as a sum", "0.5 * (ci + cj)", "(ci + cj)"),
    ("rhobar as a sum", "0.5 * (rho[i] + rho[j])", "(rho[i] + rho[j])"),
    ("eta^2 on r^2", "(r2 + eta2 * hij * hij)", "(r2 + eta2 * r2)"),
    ("beta |mu|", "beta * mu * mu", "beta * fabs(mu)"),
    ("beta mu^3", "beta * mu * mu", "beta * fabs(mu * mu * mu)"),
    ("h_i in mu", "hij * vx", "h[i] * vx"),
    ("switch on receding pairs", "vx < 0.0 ? hij", "vx > 0.0 ? hij"),
    ("limiter min(1, r)", "4.0 * rr / ((1.0 + rr) * (1.0 + rr))", "(rr < 1.0 ? rr : 1.0)"),
    ("limiter 2r/(1+r)", "4.0 * rr / ((1.0 + rr) * (1.0 + rr))", "2.0 * rr / (1.0 + rr)"),
    ("reconstruction to the far end", "0.5 * phi * (si[a] + sj[a])", "phi * (si[a] + sj[a])"),
    ("equal split on the reconstructed velocity", "E += -0.5 * (vij[0] * f[0] + vij[1] * f[1] + vij[2] * f[2]);",
     "E += -0.5 * (vs[0] * f[0] + vs[1] * f[1] + vs[2] * f[2]);"),
]


@pytest.mark.parametrize("slip", SLIPS, ids=[s[0] for s in SLIPS])
def test_planted_slip_fails_a_case(orc, slip, tmp_path, monkeypatch):
    """A copy of the oracle with one plausible mistake in the viscosity fails at least one case."""
    name, old, new = slip
    src = open(orc.SRC).read()
    assert src.count(old) >= 1, f"slip anchor not found: {old}"
    path = tmp_path / "crk_oracle_slip.c"
    path.write_text(src.replace(old, new))
    lib = orc.load(orc.compile_c(str(path), str(tmp_path / "liborc_slip.so")))
    monkeypatch.setattr(orc, "_lib", lib)
    worst = max(_mismatch(orc, case) for case in CASES)
    assert worst > 1e-6, f"slip '{name}' passes every hand-worked case"
