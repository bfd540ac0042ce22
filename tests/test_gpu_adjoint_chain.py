"""Reverse modes of Corrections and hydro on GB300 against the FP64 oracle.

The single adjoint kernels are fed the oracle's own upstream values (rounded to
FP32), so each comparison tests one kernel; the chain test runs both sides end
to end (each its own geometry, corrections and hydro) through the autograd
functions.  Gate: E <= 1e-4 for every gradient (the adjoint gate; measured
~1e-6: the per-particle reverse of the 3x3 step runs in FP64 and the pair sums
in FP32).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2310_16122_gb300 import workloads as W
from tests._errors import check

pytestmark = pytest.mark.gpu

HP = (W.GAMMA, W.AV_ALPHA, W.AV_BETA, W.AV_ETA2)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(np.sum((a - b) ** 2) / max(np.sum(b * b), 1e-300)))


@pytest.fixture(scope="module")
def api():
    from paper_2310_16122_gb300 import api as A
    from paper_2310_16122_gb300.build import build_library

    build_library()
    return A


def _box(name):
    if name == "clustered12":
        b = W.clustered_box(12, 1, 81)
    elif name == "clustered24":
        b = W.clustered_box(24, 11, 82)
    else:
        b = W.random_box(777, 13.0, 0.4, 83, h=2.0, leaf_mode=0, cells=3)
    rng = np.random.default_rng(5)
    gas = b.species == 0
    b.u = np.where(gas, rng.uniform(0.6, 1.6, b.n), 0.0).astype(np.float32)
    for c in ("vx", "vy", "vz"):
        setattr(b, c, np.where(gas, rng.normal(0.0, 0.3, b.n), 0.0).astype(np.float32))
    return b


def _t(a, dev="cuda"):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)


BOXES = ["clustered12", "clustered24", "random777_mesh3"]


@pytest.mark.parametrize("name", BOXES)
@pytest.mark.parametrize("variant", [0, 1])
def test_corrections_adjoint_matches_oracle(api, name, variant):
    b = _box(name)
    I = O.from_box(b)
    gas = b.species == 0
    V = np.asarray(O.geometry(I)[0], np.float32).astype(np.float64)  # the FP32 volumes the GPU sees
    rng = np.random.default_rng(11)
    cb = [np.where(gas, rng.normal(size=b.n), 0.0), np.where(gas[:, None], rng.normal(size=(b.n, 3)), 0.0),
          np.where(gas[:, None], rng.normal(size=(b.n, 3)), 0.0), np.where(gas[:, None], rng.normal(size=(b.n, 9)), 0.0)]
    ox, oV, ns = O.corrections_adjoint(I, V, *cb)
    assert ns == 0
    ctx = api.Context(0)
    ctx.set_variant("corrections", variant)
    db = api.DeviceBox(b)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    gx, gV, gns = api.corrections_adjoint(ctx, lv, _t(V), _t(cb[0]), _t(cb[1].T), _t(cb[2].T), _t(cb[3].T))
    torch.cuda.synchronize()
    assert int(gns.cpu()) == 0
    check(f"corrections_adjoint/{name}/v{variant}", "xbar", gx.cpu().numpy().T[gas], ox[gas], "adj")
    check(f"corrections_adjoint/{name}/v{variant}", "Vbar", gV.cpu().numpy()[gas], oV[gas], "adj")
    assert np.all(gx.cpu().numpy()[:, ~gas] == 0) and np.all(gV.cpu().numpy()[~gas] == 0)


@pytest.mark.parametrize("name", BOXES)
@pytest.mark.parametrize("variant", [0, 1])
def test_hydro_adjoint_matches_oracle(api, name, variant):
    b = _box(name)
    I = O.from_box(b)
    gas = b.species == 0
    V, rho, _ = O.geometry(I)
    A, B, gA, gB, _ = O.corrections(I, V)
    # the oracle works on the FP32-rounded inputs the GPU sees
    ins = [np.asarray(x, np.float32).astype(np.float64) for x in (V, rho, A, B, gA, gB)]
    rng = np.random.default_rng(12)
    dvbar = np.where(gas[:, None], rng.normal(size=(b.n, 3)), 0.0)
    dubar = np.where(gas, rng.normal(size=b.n), 0.0)
    og = O.hydro_adjoint(I, *ins, *HP, dvbar, dubar)
    ctx = api.Context(0)
    ctx.set_variant("hydro", variant)
    db = api.DeviceBox(b)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    t = [_t(ins[0]), _t(ins[1]), _t(ins[2]), _t(ins[3].T), _t(ins[4].T), _t(ins[5].T)]
    gg = api.hydro_adjoint(ctx, lv, db.hp, db.m, db.v3, db.u, *t, _t(dvbar.T), _t(dubar))
    torch.cuda.synchronize()
    for k, v in gg.items():
        g = v.cpu().numpy()
        g = g.T if g.ndim == 2 else g
        check(f"hydro_adjoint/{name}/v{variant}", k + "bar", g[gas], og[k][gas], "adj")
        assert np.all(g[~gas] == 0), k


@pytest.mark.parametrize("name", ["clustered12", "clustered24"])
def test_chain_gradient_through_autograd(api, name):
    from paper_2310_16122_gb300 import autograd as AG

    b = _box(name)
    I = O.from_box(b)
    gas = b.species == 0
    rng = np.random.default_rng(13)
    dvbar = np.where(gas[:, None], rng.normal(size=(b.n, 3)), 0.0)
    dubar = np.where(gas, rng.normal(size=b.n), 0.0)
    # oracle: hydro adjoint -> corrections adjoint -> geometry adjoint
    V, rho, _ = O.geometry(I)
    A, B, gA, gB, _ = O.corrections(I, V)
    gh = O.hydro_adjoint(I, V, rho, A, B, gA, gB, *HP, dvbar, dubar)
    xc, Vc, _ = O.corrections_adjoint(I, V, gh["A"], gh["B"], gh["gA"], gh["gB"])
    gx, gm = O.geometry_adjoint(I, gh["rho"], gh["V"] + Vc)
    want = dict(x=gh["x"] + xc + gx, m=gh["m"] + gm, v=gh["v"], u=gh["u"])
    # GPU: the autograd chain
    ctx = api.Context(0)
    db = api.DeviceBox(b)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    pos = torch.stack([db.x, db.y, db.z]).requires_grad_(True)
    m = db.m.clone().requires_grad_(True)
    v = db.v3.clone().requires_grad_(True)
    u = db.u.clone().requires_grad_(True)
    Vg, rhog = AG.geometry(pos, m, ctx, lv)
    Ag, Bg, gAg, gBg = AG.corrections(pos, Vg, ctx, lv)
    dv, du = AG.hydro(pos, m, v, u, Vg, rhog, Ag, Bg, gAg, gBg, ctx, lv, db.hp)
    loss = (dv * _t(dvbar.T)).sum() + (du * _t(dubar)).sum()
    loss.backward()
    torch.cuda.synchronize()
    got = dict(x=pos.grad.cpu().numpy().T, m=m.grad.cpu().numpy(), v=v.grad.cpu().numpy().T,
               u=u.grad.cpu().numpy())
    for k in want:
        check(f"chain_autograd/{name}", k + "bar", got[k][gas], want[k][gas], "adj")


def test_fused_chain_equals_autograd_chain(api):
    """crk_hydro_chain_adjoint (kernel order throughout) against the single calls chained by autograd."""
    from paper_2310_16122_gb300 import autograd as AG

    b = _box("clustered24")
    gas = b.species == 0
    rng = np.random.default_rng(14)
    dvbar = _t(np.where(gas[:, None], rng.normal(size=(b.n, 3)), 0.0).T)
    dubar = _t(np.where(gas, rng.normal(size=b.n), 0.0))
    ctx = api.Context(0)
    db = api.DeviceBox(b)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    fused = api.hydro_chain_adjoint(ctx, lv, db, dvbar, dubar)
    pos = torch.stack([db.x, db.y, db.z]).requires_grad_(True)
    m = db.m.clone().requires_grad_(True)
    v = db.v3.clone().requires_grad_(True)
    u = db.u.clone().requires_grad_(True)
    Vg, rhog = AG.geometry(pos, m, ctx, lv)
    Ag, Bg, gAg, gBg = AG.corrections(pos, Vg, ctx, lv)
    dv, du = AG.hydro(pos, m, v, u, Vg, rhog, Ag, Bg, gAg, gBg, ctx, lv, db.hp)
    ((dv * dvbar).sum() + (du * dubar).sum()).backward()
    torch.cuda.synchronize()
    assert int(fused["n_singular"].cpu()) == 0
    # forward outputs: the same kernels on the same pairs in the same order
    assert torch.equal(fused["dv"], dv.detach()) and torch.equal(fused["du"], du.detach())
    for k, ref in (("x", pos.grad), ("m", m.grad), ("v", v.grad), ("u", u.grad)):
        e = rel_l2(fused[k].cpu().numpy(), ref.cpu().numpy())
        print(k, f"{e:.1e}")
        assert e <= 1e-6, (k, e)


def test_adjoint_edge_cases(api):
    """No particles, dark matter only, and a lone gas particle (singular moments, counted)."""
    ctx = api.Context(0)
    # no particles: every call succeeds and returns empty outputs
    db = api.DeviceBox(W.random_box(0, 10.0, 0.5, 91))
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    e = torch.zeros(0, device="cuda")
    gx, gV, ns = api.corrections_adjoint(ctx, lv, e, e, e.view(3, 0), e.view(3, 0), e.view(9, 0))
    out = api.hydro_chain_adjoint(ctx, lv, db, e.view(3, 0), e)
    torch.cuda.synchronize()
    assert gx.numel() == 0 and int(ns.cpu()) == 0 and out["x"].numel() == 0
    # dark matter only: the gas chain has nothing to differentiate
    b = W.random_box(300, 12.0, 0.0, 92)
    db = api.DeviceBox(b)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    rng = np.random.default_rng(3)
    dvbar, dubar = _t(rng.normal(size=(3, b.n))), _t(rng.normal(size=b.n))
    out = api.hydro_chain_adjoint(ctx, lv, db, dvbar, dubar)
    torch.cuda.synchronize()
    for k in ("x", "m", "v", "u", "dv", "du"):
        assert torch.count_nonzero(out[k]).item() == 0, k
    # a lone gas particle: its moment matrix is singular; counted, and the adjoint of the
    # corrections leaves it out (no NaN in the gradient)
    b = W.random_box(1, 12.0, 1.0, 93, h=0.5)
    db = api.DeviceBox(b)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    V, _, _ = api.geometry(ctx, lv, db.m)
    one = torch.ones(1, device="cuda")
    gx, gV, ns = api.corrections_adjoint(ctx, lv, V, one, torch.ones(3, 1, device="cuda"),
                                         torch.ones(3, 1, device="cuda"), torch.ones(9, 1, device="cuda"))
    torch.cuda.synchronize()
    assert int(ns.cpu()) == 1
    assert torch.isfinite(gx).all() and torch.isfinite(gV).all()
