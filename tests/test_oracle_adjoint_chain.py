"""Pins of the oracle's reverse modes of Corrections and of the hydro pair force.

Both adjoints are hand-written FP64 reverse modes; what fixes them is the
derivative of the forward oracle itself, taken by central differences:

* the kernel's second radial derivative (d[(dW/dr)/r]/dr)/r against a central
  difference of (dW/dr)/r, and its closed value at r = 0;
* corrections: the gradient of L = sum Abar A + Bbar.B + gAbar.gA + gBbar:gB in
  the positions and the volumes;
* hydro: the gradient of L = sum dvbar.dv + dubar.du in every input of the pair
  force (positions, velocities, u, m, V, rho, A, B, gA, gB) held independent;
* the chain: the gradient of the hydro loss in the positions through geometry,
  corrections and hydro together (hydro adjoint -> corrections adjoint ->
  geometry adjoint), against a central difference of the whole forward chain.

Random cotangents make a dropped term, a transposed index or a wrong sign show
up in at least one sampled derivative.
"""
import numpy as np
import pytest

from paper_2310_16122_gb300 import workloads as W

G, ALPHA, BETA, ETA2 = W.GAMMA, W.AV_ALPHA, W.AV_BETA, W.AV_ETA2
HP = (G, ALPHA, BETA, ETA2)


def _box(orc, seed=71):
    b = W.lattice_box(6, 0.25, seed, h=1.35, leaf_mode=0, cells=2)
    I = orc.from_box(b)
    rng = np.random.default_rng(seed)
    gas = I.species == 0
    v = np.where(gas[:, None], rng.normal(0.0, 0.3, I.v.shape), 0.0)
    u = np.where(gas, rng.uniform(0.6, 1.6, I.n), 0.0)
    return orc.Inputs(I.pos, I.species, I.m, I.h, u, v, I.L, I.r_cut, I.eps, I.poly)


def _with(orc, I, pos=None, v=None, u=None, m=None):
    return orc.Inputs(I.pos if pos is None else pos, I.species, I.m if m is None else m, I.h,
                      I.u if u is None else u, I.v if v is None else v, I.L, I.r_cut, I.eps, I.poly)


def _cd(f, x0, eps):
    return (f(x0 + eps) - f(x0 - eps)) / (2.0 * eps)


def test_kernel_second_derivative(orc):
    h = 1.3
    r = np.linspace(0.05, 2.55, 40)
    _, dWr, ddWr = orc.wendland2(r, h)
    e = 1e-6
    _, dp, _ = orc.wendland2(r + e, h)
    _, dm, _ = orc.wendland2(r - e, h)
    fd = (dp - dm) / (2 * e) / r
    np.testing.assert_allclose(ddWr, fd, rtol=1e-6, atol=1e-9 * np.abs(ddWr).max())
    W0, dW0, ddW0 = orc.wendland2(np.array([0.0]), h)
    s = 495.0 / (256.0 * np.pi)
    assert ddW0[0] == pytest.approx(s * 35.0 / h ** 7, rel=1e-14)
    assert dW0[0] == pytest.approx(-s * 14.0 / 3.0 / h ** 5, rel=1e-14)


def _corr_loss(orc, I, V, cb):
    A, B, gA, gB, nsing = orc.corrections(I, V)
    assert nsing == 0
    return float(np.sum(cb[0] * A) + np.sum(cb[1] * B) + np.sum(cb[2] * gA) + np.sum(cb[3] * gB))


def test_corrections_adjoint_matches_central_differences(orc):
    I = _box(orc)
    gas = I.species == 0
    V, _, _ = orc.geometry(I)
    rng = np.random.default_rng(2)
    cb = [np.where(gas, rng.normal(size=I.n), 0.0), np.where(gas[:, None], rng.normal(size=(I.n, 3)), 0.0),
          np.where(gas[:, None], rng.normal(size=(I.n, 3)), 0.0), np.where(gas[:, None], rng.normal(size=(I.n, 9)), 0.0)]
    xbar, Vbar, nsing = orc.corrections_adjoint(I, V, *cb)
    assert nsing == 0
    idx = rng.choice(np.nonzero(gas)[0], 6, replace=False)
    for k in idx:
        for c in range(3):
            def f(t, k=k, c=c):
                p = I.pos.copy()
                p[k, c] = t
                return _corr_loss(orc, _with(orc, I, pos=p), V, cb)
            fd = _cd(f, I.pos[k, c], 1e-5)
            assert xbar[k, c] == pytest.approx(fd, rel=2e-6, abs=1e-8 * np.abs(xbar).max())

        def fv(t, k=k):
            V2 = V.copy()
            V2[k] = t
            return _corr_loss(orc, I, V2, cb)
        fd = _cd(fv, V[k], 1e-6 * V[k])
        assert Vbar[k] == pytest.approx(fd, rel=2e-6, abs=1e-8 * np.abs(Vbar).max())
    # dark matter takes no part
    assert np.all(xbar[~gas] == 0) and np.all(Vbar[~gas] == 0)


def _hydro_loss(orc, I, ins, cb):
    dv, du, _ = orc.hydro(I, *ins, *HP)
    return float(np.sum(cb[0] * dv) + np.sum(cb[1] * du))


def test_hydro_adjoint_matches_central_differences(orc):
    I = _box(orc, 72)
    gas = I.species == 0
    V, rho, _ = orc.geometry(I)
    A, B, gA, gB, _ = orc.corrections(I, V)
    rng = np.random.default_rng(3)
    cb = [np.where(gas[:, None], rng.normal(size=(I.n, 3)), 0.0), np.where(gas, rng.normal(size=I.n), 0.0)]
    ins = [V, rho, A, B, gA, gB]
    g = orc.hydro_adjoint(I, *ins, *HP, cb[0], cb[1])
    idx = rng.choice(np.nonzero(gas)[0], 5, replace=False)
    scale = {k: np.abs(v).max() for k, v in g.items()}

    def check(name, k, c, fd):
        got = g[name][k, c] if g[name].ndim == 2 else g[name][k]
        assert got == pytest.approx(fd, rel=5e-6, abs=1e-8 * scale[name]), (name, k, c)

    for k in idx:
        for c in range(3):
            def fx(t):
                p = I.pos.copy()
                p[k, c] = t
                return _hydro_loss(orc, _with(orc, I, pos=p), ins, cb)
            check("x", k, c, _cd(fx, I.pos[k, c], 1e-6))

            def fvel(t):
                v = I.v.copy()
                v[k, c] = t
                return _hydro_loss(orc, _with(orc, I, v=v), ins, cb)
            check("v", k, c, _cd(fvel, I.v[k, c], 1e-6))
        for name, arr, pos in (("u", I.u, "u"), ("m", I.m, "m")):
            def fs(t, arr=arr, pos=pos):
                a = arr.copy()
                a[k] = t
                return _hydro_loss(orc, _with(orc, I, **{pos: a}), ins, cb)
            check(name, k, 0, _cd(fs, arr[k], 1e-6 * arr[k]))
        for j, name in enumerate(("V", "rho", "A", "B", "gA", "gB")):
            arr = ins[j]
            comps = range(arr.shape[1]) if arr.ndim == 2 else [None]
            for c in comps:
                def fi(t, j=j, c=c):
                    a = arr.copy()
                    if c is None:
                        a[k] = t
                    else:
                        a[k, c] = t
                    ins2 = list(ins)
                    ins2[j] = a
                    return _hydro_loss(orc, I, ins2, cb)
                x0 = arr[k] if c is None else arr[k, c]
                # the pair force is linear in each of these inputs: a large step has no truncation error
                check(name, k, 0 if c is None else c, _cd(fi, x0, 1e-3 * max(abs(x0), np.abs(arr[gas]).mean())))


def test_chain_adjoint_matches_central_differences(orc):
    """d/dx and d/dm of the hydro loss through geometry -> corrections -> hydro."""
    I = _box(orc, 73)
    gas = I.species == 0
    rng = np.random.default_rng(4)
    cb = [np.where(gas[:, None], rng.normal(size=(I.n, 3)), 0.0), np.where(gas, rng.normal(size=I.n), 0.0)]

    def loss(J):
        V, rho, _ = orc.geometry(J)
        A, B, gA, gB, _ = orc.corrections(J, V)
        return _hydro_loss(orc, J, [V, rho, A, B, gA, gB], cb)

    V, rho, _ = orc.geometry(I)
    A, B, gA, gB, _ = orc.corrections(I, V)
    gh = orc.hydro_adjoint(I, V, rho, A, B, gA, gB, *HP, cb[0], cb[1])
    xc, Vc, _ = orc.corrections_adjoint(I, V, gh["A"], gh["B"], gh["gA"], gh["gB"])
    gx, gm = orc.geometry_adjoint(I, gh["rho"], gh["V"] + Vc)
    xbar = gh["x"] + xc + gx
    mbar = gh["m"] + gm
    idx = rng.choice(np.nonzero(gas)[0], 5, replace=False)
    for k in idx:
        for c in range(3):
            def fx(t):
                p = I.pos.copy()
                p[k, c] = t
                return loss(_with(orc, I, pos=p))
            fd = _cd(fx, I.pos[k, c], 1e-6)
            assert xbar[k, c] == pytest.approx(fd, rel=5e-6, abs=1e-8 * np.abs(xbar).max())

        def fm(t):
            m = I.m.copy()
            m[k] = t
            return loss(_with(orc, I, m=m))
        fd = _cd(fm, I.m[k], 1e-6 * I.m[k])
        assert mbar[k] == pytest.approx(fd, rel=5e-6, abs=1e-8 * np.abs(mbar).max())
