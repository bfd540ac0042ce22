"""Adjoint path (gravity and geometry): autograd through grav_short and crk_geometry on GB300.

Loss = sum_i |a_grav,i|^2 + sum_gas rho_i on the clustered 2x32^3 box (25
halos).  The gradients with respect to positions and masses come from the
hand-written adjoint kernels behind torch.autograd.Function.  They are
checked against the oracle's analytic gradient (whole box) and against FP64
central differences of the oracle's forward pass (step 1e-4) at 64 seeded
coordinates and 16 seeded masses.  A central difference only needs the loss
terms that move: a_i for i within r_c of the moved particle and rho_i for gas
within its smoothing range, so the oracle evaluates just those.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2310_16122_gb300 import workloads as W
from tests._errors import check, cut_boundary_particles

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(np.sum((a - b) ** 2) / max(np.sum(b * b), 1e-300)))


@pytest.fixture(scope="module")
def run():
    from paper_2310_16122_gb300 import api, autograd as AG
    from paper_2310_16122_gb300.build import build_library

    build_library()
    b = W.adjoint_box()
    ctx = api.Context(0)
    db = api.DeviceBox(b)
    # the leaves are built from the rows of the positions tensor the loss differentiates
    pos3 = torch.stack([db.x, db.y, db.z]).contiguous()
    lv = api.build_leaves(ctx, pos3[0], pos3[1], pos3[2], db.species, db.h, db.L, db.lp)
    pos3.requires_grad_(True)
    m = db.m.clone().requires_grad_(True)
    a = AG.gravity(pos3, m, ctx, lv, db.gp)
    V, rho = AG.geometry(pos3, m, ctx, lv)
    gas = db.species == 0
    loss = (a * a).sum() + rho[gas].sum()
    loss.backward()
    torch.cuda.synchronize()
    return b, pos3.grad.detach().cpu().numpy().T, m.grad.detach().cpu().numpy(), float(loss.detach())


def local_loss(I, pos, k, mass=None):
    J = I.with_pos(pos) if mass is None else I.with_m(mass)
    ng = O.neighbour_closure(I, [k], hydro=False)
    acc, _ = O.gravity(J, sub=ng)
    L = float(np.sum(acc[ng] ** 2))
    if I.species[k] == 0:
        nh = O.neighbour_closure(I, [k], hydro=True)
        _, rho, _ = O.geometry(J, sub=nh)
        L += float(np.sum(rho[nh][I.species[nh] == 0]))
    return L


def test_gradient_matches_oracle_analytic(run):
    b, gx, gm, loss = run
    I = O.from_box(b)
    acc, _ = O.gravity(I)
    gas = (b.species == 0).astype(np.float64)
    ogx1, ogm1 = O.gravity_adjoint(I, 2.0 * acc)
    ogx2, ogm2 = O.geometry_adjoint(I, gas)
    _, rho, _ = O.geometry(I)
    ref_loss = float(np.sum(acc * acc) + rho[b.species == 0].sum())
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss)
    check("adjoint/config3", "gx", gx, ogx1 + ogx2, exclude=cut_boundary_particles(I.pos, b.L, b.r_cut))
    check("adjoint/config3", "gm", gm, ogm1 + ogm2)


def test_gradient_matches_fp64_central_differences(run):
    b, gx, gm, _ = run
    I = O.from_box(b)
    rng = np.random.default_rng(W.SEEDS["adjoint"] + 64)
    step = 1e-4
    sx = np.sqrt(np.mean(gx * gx))
    errs = []
    for _ in range(64):
        k, c = int(rng.integers(b.n)), int(rng.integers(3))
        p = I.pos.copy()
        p[k, c] += step
        lp = local_loss(I, p, k)
        p[k, c] -= 2 * step
        lm = local_loss(I, p, k)
        fd = (lp - lm) / (2 * step)
        errs.append(abs(gx[k, c] - fd) / (abs(fd) + 1e-3 * sx))
    sm = np.sqrt(np.mean(gm * gm))
    for _ in range(16):
        k = int(rng.integers(b.n))
        mm = I.m.copy()
        mm[k] += step
        lp = local_loss(I, I.pos, k, mm)
        mm[k] -= 2 * step
        lm = local_loss(I, I.pos, k, mm)
        fd = (lp - lm) / (2 * step)
        errs.append(abs(gm[k] - fd) / (abs(fd) + 1e-3 * sm))
    print(f"adjoint vs FD: max {max(errs):.2e} median {np.median(errs):.2e}")
    assert max(errs) < 1e-3


def test_stale_leaves_are_refused():
    """Positions other than those the leaves were built from raise CRK_ESTATE; equal copies pass."""
    from paper_2310_16122_gb300 import api, autograd as AG, native as N

    b = W.clustered_box(12, 1, 52)
    ctx = api.Context(0)
    db = api.DeviceBox(b)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    m = db.m.clone().requires_grad_(True)
    same = torch.stack([db.x, db.y, db.z]).requires_grad_(True)  # another tensor, equal values
    a = AG.gravity(same, m, ctx, lv, db.gp)
    (a * a).sum().backward()
    assert same.grad is not None and bool(torch.isfinite(same.grad).all())
    moved = torch.stack([db.x, db.y, db.z]).clone()
    moved[0, 7] += 0.01
    for f in (lambda p: AG.gravity(p, m, ctx, lv, db.gp), lambda p: AG.geometry(p, m, ctx, lv)):
        with pytest.raises(N.CrkError) as e:
            f(moved.requires_grad_(True))
        assert e.value.status == N.CRK_ESTATE
    with pytest.raises(N.CrkError) as e:
        AG.gravity(moved[:, :-1], m, ctx, lv, db.gp)
    assert e.value.status == N.CRK_ESTATE
