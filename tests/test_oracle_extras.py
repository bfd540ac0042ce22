"""Pins of the oracle's Extras stage and limited viscosity against mathematics.

Extras (Sec. 5: the density and state gradients) is read as the
corrected-kernel density rhoR_i = sum_j m_j W^R_ij and the velocity gradient
dv^a/dx^b = sum_j V_j (v_j^a - v_i^a) (grad_i W^R_ij)^b; the limited
viscosity reconstructs both velocities to the pair midpoint with a van Leer
limiter.  What fixes each expected value:

* reproduction of a constant: masses m_j = rho0 V_j give rhoR = rho0 on any
  layout (linear CRK reproduces constants exactly);
* reproduction of a linear field: v = v0 + G x gives dv/dx = G exactly, for a
  non-symmetric G (a transposed index fails);
* on a perfect lattice with equal masses rhoR equals the geometry density m/V;
* a zero gradient switches the limiter off (phi = 0): the unlimited hydro;
* the limited pair force is still antisymmetric: momentum and energy are
  conserved to FP64 rounding;
* a linear velocity field with its exact gradient reconstructs to equal
  midpoint velocities, so the viscosity vanishes: the result equals the
  inviscid one (alpha = beta = 0), while the unlimited viscosity does not.
"""
import numpy as np
import pytest

from paper_2310_16122_gb300 import workloads as W

G, ALPHA, BETA, ETA2 = W.GAMMA, W.AV_ALPHA, W.AV_BETA, W.AV_ETA2


def lattice(side=8, sigma=0.0, h=1.2, seed=7):
    return W.lattice_box(side, sigma, seed, h=h, leaf_mode=0, cells=2)


def _chain(orc, I):
    V, rho, _ = orc.geometry(I)
    A, B, gA, gB, nsing = orc.corrections(I, V)
    assert nsing == 0
    return V, rho, A, B, gA, gB


def _with_v(orc, I, v):
    return orc.Inputs(I.pos, I.species, I.m, I.h, I.u, v, I.L, I.r_cut, I.eps, I.poly)


def _interior(I, margin):
    return (I.species == 0) & np.all((I.pos > margin) & (I.pos < I.L - margin), axis=1)


@pytest.mark.parametrize("box", ["perturbed", "clustered"])
def test_extras_density_reproduces_constant(orc, box):
    b = lattice(8, 0.3, h=1.4, seed=21) if box == "perturbed" else W.clustered_box(12, 1, 22)
    I = orc.from_box(b)
    V, _, A, B, gA, gB = _chain(orc, I)
    gas = I.species == 0
    rho0 = 2.5
    m = np.where(gas, rho0 * V, I.m)
    rhoR, _ = orc.extras(I.with_m(m), V, A, B, gA, gB)
    np.testing.assert_allclose(rhoR[gas], rho0, rtol=1e-11)
    assert np.all(rhoR[~gas] == 0.0)


def test_extras_perfect_lattice_density_is_geometry_density(orc):
    I = orc.from_box(lattice(8, 0.0, h=1.3))
    V, rho, A, B, gA, gB = _chain(orc, I)
    gas = I.species == 0
    rhoR, dvg = orc.extras(I, V, A, B, gA, gB)
    np.testing.assert_allclose(rhoR[gas], rho[gas], rtol=1e-12)


@pytest.mark.parametrize("box", ["perturbed", "clustered"])
def test_extras_velocity_gradient_exact_for_linear_field(orc, box):
    b = lattice(10, 0.3, h=1.4, seed=23) if box == "perturbed" else W.clustered_box(14, 1, 24)
    I = orc.from_box(b)
    V, _, A, B, gA, gB = _chain(orc, I)
    Gm = np.array([[0.3, -0.7, 0.2], [0.5, -0.1, 0.9], [-0.4, 0.6, 0.25]])  # not symmetric
    v0 = np.array([0.1, -0.2, 0.05])
    v = v0 + I.pos @ Gm.T  # v^a = v0^a + G[a, b] x^b
    J = _with_v(orc, I, v)
    _, dvg = orc.extras(J, V, A, B, gA, gB)
    hmax = I.h[I.species == 0].max()
    inner = _interior(I, 2.0 * hmax + 0.01)
    assert inner.sum() > 50
    np.testing.assert_allclose(dvg[inner], np.tile(Gm.ravel(), (inner.sum(), 1)), atol=1e-10)


def test_extras_brute_equals_cells(orc):
    I = orc.from_box(W.clustered_box(12, 1, 25))
    V, _, A, B, gA, gB = _chain(orc, I)
    r1, g1, p1 = orc.extras(I, V, A, B, gA, gB, with_pairs=True)
    r2, g2, p2 = orc.extras(I, V, A, B, gA, gB, brute=True, with_pairs=True)
    assert p1 == p2
    np.testing.assert_allclose(r1, r2, rtol=1e-13)
    np.testing.assert_allclose(g1, g2, atol=1e-12 * np.abs(g1).max())


def test_limited_hydro_with_zero_gradient_is_unlimited(orc):
    I = orc.from_box(W.clustered_box(12, 1, 26))
    V, rho, A, B, gA, gB = _chain(orc, I)
    d0 = orc.hydro(I, V, rho, A, B, gA, gB, G, ALPHA, BETA, ETA2)
    d1 = orc.hydro(I, V, rho, A, B, gA, gB, G, ALPHA, BETA, ETA2, dvg=np.zeros((I.n, 9)))
    np.testing.assert_array_equal(d0[0], d1[0])
    np.testing.assert_array_equal(d0[1], d1[1])


def test_limited_hydro_conserves_momentum_and_energy(orc):
    I = orc.from_box(W.clustered_box(12, 1, 27))
    V, rho, A, B, gA, gB = _chain(orc, I)
    rhoR, dvg = orc.extras(I, V, A, B, gA, gB)
    dv, du, _ = orc.hydro(I, V, rhoR, A, B, gA, gB, G, ALPHA, BETA, ETA2, dvg=dvg)
    d0, _, _ = orc.hydro(I, V, rhoR, A, B, gA, gB, G, ALPHA, BETA, ETA2)
    assert np.max(np.abs(dv - d0)) > 0  # the limiter changed something
    cons = orc.conservation(I, dv, du)
    gas = I.species == 0
    scale_p = np.abs(I.m[gas, None] * dv[gas]).sum()
    scale_e = np.abs(I.m[gas] * du[gas]).sum() + np.abs(I.m[gas, None] * I.v[gas] * dv[gas]).sum()
    assert np.max(np.abs(cons[:3])) < 1e-13 * scale_p
    assert abs(cons[3]) < 1e-13 * scale_e


def test_limited_viscosity_vanishes_for_linear_flow(orc):
    """Compressive shear v = G x: the limited viscosity is zero where the gradient is exact."""
    b = lattice(18, 0.25, h=1.3, seed=28)
    I = orc.from_box(b)
    gas = I.species == 0
    Gm = np.array([[-0.20, 0.05, 0.00], [0.10, -0.15, 0.02], [0.00, -0.03, -0.10]])
    J = _with_v(orc, I, I.pos @ Gm.T)
    V, rho, A, B, gA, gB = _chain(orc, J)
    _, dvg = orc.extras(J, V, A, B, gA, gB)
    hmax = I.h[gas].max()
    # particles whose every neighbour has an exact gradient: two support radii from the wrap
    inner = _interior(I, 4.0 * hmax + 0.02)
    assert inner.sum() > 30
    dv_l, du_l, _ = orc.hydro(J, V, rho, A, B, gA, gB, G, ALPHA, BETA, ETA2, dvg=dvg)
    dv_0, du_0, _ = orc.hydro(J, V, rho, A, B, gA, gB, G, 0.0, 0.0, ETA2)
    dv_u, du_u, _ = orc.hydro(J, V, rho, A, B, gA, gB, G, ALPHA, BETA, ETA2)
    np.testing.assert_allclose(dv_l[inner], dv_0[inner], atol=1e-12 * np.abs(dv_0[inner]).max())
    np.testing.assert_allclose(du_l[inner], du_0[inner], atol=1e-12 * np.abs(du_0[inner]).max())
    # the unlimited viscosity heats the same compressive flow
    assert np.max(du_u[inner] - du_0[inner]) > 1e-3 * np.abs(du_0[inner]).max()
