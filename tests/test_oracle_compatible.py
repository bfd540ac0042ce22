"""Pins of the oracle's compatible energy split, signal velocity, timestep and integrator.

Sec. 5 names Acceleration and Energy as separate kernels and Sec. 5.4 calls
each twice per timestep; Sec. 5.1 uses a floating-point atomic max.  The paper
prints no formula for any of them; the readings (compatible differencing of
the pair work on time-centred velocities, shared toward thermal equilibrium;
Monaghan's signal speed with a Courant factor; a two-stage kick-drift step)
are pinned here by what the mathematics fixes:

* the share w_ij is in (0, 1), w_ij + w_ji = 1, it is 1/2 for equal u, and
  heating goes preferentially to the colder particle (cooling to the hotter);
* with equal u and v* = v the compatible du is the equal-split du;
* sum_i m_i du_i = -sum_i m_i v*_i.dv_i for any u and v* (no heat is made or
  lost beyond the work), so one hydro-only step conserves kinetic plus
  thermal energy to FP64 rounding;
* in a two-temperature box every cold particle gains at least, and every hot
  one at most, what the equal split gives it;
* the signal speed of a static gas is 2c; of a uniform compression
  v = -k x it is 2c + 3 k r_max (r_max: the farthest neighbour in range);
  of a uniform expansion 2c;
* a static lattice stays put; a uniform translation only drifts;
* the step is second order: over a fixed time, halving dt divides the
  error against a finely resolved run by about 4 (a first-order step: 2).
"""
import numpy as np
import pytest

from paper_2310_16122_gb300 import workloads as W

G, ALPHA, BETA, ETA2 = W.GAMMA, W.AV_ALPHA, W.AV_BETA, W.AV_ETA2
HP = (G, ALPHA, BETA, ETA2)


def _with(orc, I, pos=None, v=None, u=None):
    return orc.Inputs(I.pos if pos is None else pos, I.species, I.m, I.h, I.u if u is None else u,
                      I.v if v is None else v, I.L, I.r_cut, I.eps, I.poly)


def _chain(orc, I):
    V, rho, _ = orc.geometry(I)
    A, B, gA, gB, nsing = orc.corrections(I, V)
    assert nsing == 0
    return V, rho, A, B, gA, gB


def _two_temperature(I, seed, lo=1.0, hi=4.0):
    rng = np.random.default_rng(seed)
    gas = I.species == 0
    hot = gas & (rng.random(I.n) < 0.5)
    u = np.where(gas, np.where(hot, hi, lo), 0.0)
    return u, hot


def _interior(I, margin):
    return (I.species == 0) & np.all((I.pos > margin) & (I.pos < I.L - margin), axis=1)


def test_energy_share_values_and_symmetry(orc):
    assert orc.energy_share(1.0, 3.0, 1.0) == pytest.approx(0.75, abs=1e-15)   # i colder, heating: 3/4 to i
    assert orc.energy_share(1.0, 3.0, -1.0) == pytest.approx(0.25, abs=1e-15)  # i colder, cooling: 1/4 from i
    assert orc.energy_share(2.0, 2.0, 5.0) == 0.5
    assert orc.energy_share(2.0, 2.0, -5.0) == 0.5
    rng = np.random.default_rng(3)
    for _ in range(200):
        ui, uj = rng.uniform(0.0, 5.0, 2)
        dE = rng.normal()
        wi, wj = orc.energy_share(ui, uj, dE), orc.energy_share(uj, ui, dE)
        assert 0.0 < wi < 1.0
        assert wi + wj == pytest.approx(1.0, abs=1e-15)
        if ui < uj:  # the colder one takes the larger part of heat and the smaller part of cooling
            assert (wi > 0.5) == (dE > 0)


@pytest.mark.parametrize("limited", [False, True])
def test_compatible_with_equal_u_and_vstar_v_is_equal_split(orc, limited):
    I = orc.from_box(W.clustered_box(12, 1, 51))
    gas = I.species == 0
    I = _with(orc, I, u=np.where(gas, 1.3, 0.0))
    V, rho, A, B, gA, gB = _chain(orc, I)
    dvg = orc.extras(I, V, A, B, gA, gB)[1] if limited else None
    dv0, du0, _ = orc.hydro(I, V, rho, A, B, gA, gB, *HP, dvg=dvg)
    dv1, du1, vsig = orc.hydro_compatible(I, V, rho, A, B, gA, gB, *HP, vstar=I.v, dvg=dvg)
    np.testing.assert_array_equal(dv1, dv0)
    np.testing.assert_allclose(du1, du0, rtol=1e-13, atol=1e-15 * np.abs(du0).max())
    assert np.all(vsig[gas] > 0) and np.all(vsig[~gas] == 0)


def test_compatible_heat_balances_work(orc):
    """sum m du = -sum m v*.dv for any u and any v*: a transposed or dropped share fails this."""
    I = orc.from_box(W.clustered_box(12, 1, 52))
    u, _ = _two_temperature(I, 5)
    I = _with(orc, I, u=u)
    V, rho, A, B, gA, gB = _chain(orc, I)
    rng = np.random.default_rng(9)
    vstar = I.v + rng.normal(0.0, 0.03, I.v.shape)
    dv, du, _ = orc.hydro_compatible(I, V, rho, A, B, gA, gB, *HP, vstar=vstar)
    gas = I.species == 0
    work = float(np.sum(I.m[gas, None] * vstar[gas] * dv[gas]))
    heat = float(np.sum(I.m[gas] * du[gas]))
    scale = float(np.sum(np.abs(I.m[gas, None] * vstar[gas] * dv[gas])))
    assert abs(heat + work) < 1e-13 * scale
    assert np.max(np.abs((I.m[gas, None] * dv[gas]).sum(axis=0))) < 1e-13 * np.abs(I.m[gas, None] * dv[gas]).sum()


def test_compatible_split_drives_toward_equilibrium(orc):
    I = orc.from_box(W.clustered_box(12, 1, 53))
    u, hot = _two_temperature(I, 6)
    I = _with(orc, I, u=u)
    gas = I.species == 0
    V, rho, A, B, gA, gB = _chain(orc, I)
    _, du_e, _ = orc.hydro(I, V, rho, A, B, gA, gB, *HP)
    _, du_c, _ = orc.hydro_compatible(I, V, rho, A, B, gA, gB, *HP, vstar=I.v)
    tol = 1e-12 * np.abs(du_e[gas]).max()
    cold = gas & ~hot
    assert np.all(du_c[cold] >= du_e[cold] - tol)
    assert np.all(du_c[hot] <= du_e[hot] + tol)
    assert np.max(du_c[cold] - du_e[cold]) > 1e-3 * np.abs(du_e[gas]).max()
    # the total heat is the same: only its distribution changed
    assert abs(np.sum(I.m * du_c) - np.sum(I.m * du_e)) < 1e-12 * np.sum(np.abs(I.m * du_e))


def test_signal_velocity_static_compression_expansion(orc):
    I = orc.from_box(W.lattice_box(10, 0.2, 54, h=1.3, leaf_mode=0, cells=2))
    gas = I.species == 0
    I = _with(orc, I, u=np.where(gas, 1.1, 0.0), v=np.zeros_like(I.v))
    V, rho, A, B, gA, gB = _chain(orc, I)
    c = np.sqrt(G * (G - 1.0) * 1.1)
    _, _, vs = orc.hydro_compatible(I, V, rho, A, B, gA, gB, *HP, vstar=I.v)
    np.testing.assert_allclose(vs[gas], 2.0 * c, rtol=1e-15)
    k = 0.07
    inner = _interior(I, 2.0 * I.h[gas].max() + 0.01)
    assert inner.sum() > 20
    for sign in (-1.0, 1.0):
        J = _with(orc, I, v=sign * k * I.pos)
        _, _, vs = orc.hydro_compatible(J, V, rho, A, B, gA, gB, *HP, vstar=J.v)
        for i in np.nonzero(inner)[0]:
            d = I.pos[gas] - I.pos[i]  # no wrap needed: i is two supports inside the box
            r = np.sqrt(np.sum(d * d, axis=1))
            hs = I.h[i] + I.h[gas]
            rmax = r[r < hs].max()
            want = 2.0 * c + (3.0 * k * rmax if sign < 0 else 0.0)
            assert vs[i] == pytest.approx(want, rel=1e-13)
    # receding pairs add no approach term: a two-temperature expanding gas has
    # vsig_i = c_i + max_j c_j over the neighbours in range
    u, _ = _two_temperature(I, 8, 0.5, 3.0)
    J = _with(orc, I, v=k * I.pos, u=u)
    _, _, vs = orc.hydro_compatible(J, V, rho, A, B, gA, gB, *HP, vstar=J.v)
    cs = np.sqrt(G * (G - 1.0) * u)
    gi = np.nonzero(gas)[0]
    for i in np.nonzero(inner)[0]:
        d = I.pos[gi] - I.pos[i]
        r = np.sqrt(np.sum(d * d, axis=1))
        near = r < I.h[i] + I.h[gi]
        assert vs[i] == pytest.approx(cs[i] + cs[gi][near].max(), rel=1e-13)


def test_timestep_closed_form(orc):
    I = orc.from_box(W.lattice_box(8, 0.0, 55, h=1.25, leaf_mode=0, cells=2))
    gas = I.species == 0
    I = _with(orc, I, u=np.where(gas, 0.8, 0.0), v=np.zeros_like(I.v))
    c = np.sqrt(G * (G - 1.0) * 0.8)
    vsig = np.where(gas, 2.0 * c, 0.0)
    assert orc.timestep(I, vsig, 0.3, 10.0) == pytest.approx(0.3 * 1.25 / (2.0 * c), rel=1e-15)
    assert orc.timestep(I, vsig, 0.3, 0.01) == 0.01
    # the full step picks the same dt and leaves a static uniform lattice where it was
    J, dt = orc.advance(I, *HP, cfl=0.3, dt_max=10.0)
    assert dt == pytest.approx(0.3 * 1.25 / (2.0 * c), rel=1e-15)
    np.testing.assert_allclose(J.pos, I.pos, atol=1e-12)
    np.testing.assert_allclose(J.v, 0.0, atol=1e-12)
    np.testing.assert_allclose(J.u, I.u, atol=1e-12)


def test_uniform_translation_only_drifts(orc):
    I = orc.from_box(W.lattice_box(8, 0.0, 56, h=1.25, leaf_mode=0, cells=2))
    gas = I.species == 0
    v0 = np.array([0.3, -0.2, 0.45])
    I = _with(orc, I, u=np.where(gas, 1.0, 0.0), v=np.tile(v0, (I.n, 1)))
    J, dt = orc.advance(I, *HP, cfl=0.3, dt_max=0.5)
    d = J.pos - I.pos
    d -= I.L * np.rint(d / I.L)
    np.testing.assert_allclose(d, np.tile(dt * v0, (I.n, 1)), atol=1e-12)
    np.testing.assert_allclose(J.v, I.v, atol=1e-12)
    np.testing.assert_allclose(J.u, I.u, atol=1e-12)


@pytest.mark.parametrize("limited", [False, True])
def test_step_conserves_total_energy(orc, limited):
    """Hydro only: kinetic + thermal energy after one step equals the start, to FP64 rounding."""
    I = orc.from_box(W.clustered_box(12, 1, 57))
    u, _ = _two_temperature(I, 7, 0.5, 2.0)
    rng = np.random.default_rng(11)
    gas = I.species == 0
    v = np.where(gas[:, None], rng.normal(0.0, 0.3, I.v.shape), 0.0)
    I = _with(orc, I, u=u, v=v)
    J, dt = orc.advance(I, *HP, cfl=0.25, dt_max=1.0, limited=limited)
    assert dt > 0
    e0 = 0.5 * np.sum(I.m[:, None] * I.v ** 2) + np.sum(I.m * I.u)
    e1 = 0.5 * np.sum(J.m[:, None] * J.v ** 2) + np.sum(J.m * J.u)
    assert abs(e1 - e0) < 1e-13 * e0
    # momentum too
    p0, p1 = np.sum(I.m[:, None] * I.v, axis=0), np.sum(J.m[:, None] * J.v, axis=0)
    np.testing.assert_allclose(p1, p0, atol=1e-13 * np.sum(np.abs(I.m[:, None] * I.v)))
    # something happened: the step moved energy between kinetic and thermal
    assert abs(np.sum(J.m * J.u) - np.sum(I.m * I.u)) > 1e-6 * e0


def test_step_is_second_order(orc):
    """Inviscid, smooth flow: the one-step error against a resolved step falls ~8x per halving of dt."""
    I = orc.from_box(W.lattice_box(8, 0.15, 58, h=1.3, leaf_mode=0, cells=2))
    gas = I.species == 0
    kx = 2.0 * np.pi / I.L
    v = np.zeros_like(I.v)
    v[:, 0] = 0.2 * np.sin(kx * I.pos[:, 1])
    v[:, 1] = 0.15 * np.cos(kx * I.pos[:, 2])
    v[~gas] = 0.0
    u = np.where(gas, 1.0 + 0.2 * np.sin(kx * I.pos[:, 0]), 0.0)
    I = _with(orc, I, u=u, v=v)
    hp = (G, 0.0, 0.0, ETA2)

    def run(dt, k):
        J = I
        for _ in range(k):
            J, _ = orc.advance(J, *hp, cfl=1.0, dt_max=1.0, dt=dt)
        return J

    def err(a, b):
        d = a.pos - b.pos
        d -= I.L * np.rint(d / I.L)
        return np.sqrt(np.sum(d ** 2) + np.sum((a.v - b.v) ** 2) + np.sum((a.u - b.u) ** 2))

    T = 0.2
    ref = run(T / 16, 16)
    e1 = err(run(T, 1), ref)
    e2 = err(run(T / 2, 2), ref)
    e4 = err(run(T / 4, 4), ref)
    # global error over a fixed time: ~4x per halving for a second-order method (2x for first order)
    assert e1 / e2 > 3.0 and e2 / e4 > 3.0, (e1, e2, e4)
