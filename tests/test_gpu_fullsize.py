"""Parity at full size, in the launch configuration bench.py times.

* The clustered 2x64^3 box (524,288 particles, 200 halos): every output of the
  forward path and of both adjoints against the full FP64 oracle; leaves and
  leaf-pair lists bit-exact.
* The large 2x256^3 box (33,554,432 particles, 5000 halos) that bench.py
  times: the oracle's own RCB of the whole box against the GPU leaves
  (bit-exact), the oracle's leaf-pair lists of 64 sampled leaves, and 384
  sampled particles through the oracle's sampled chain (every upstream value
  the oracle needs is computed by the oracle itself), plus the FP64
  conservation sums of the whole box.
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


def gpu_forward_and_adjoint(b):
    from paper_2310_16122_gb300 import api
    from paper_2310_16122_gb300.build import build_library

    build_library()
    ctx = api.Context(0)
    db = api.DeviceBox(b)
    out = api.forward(ctx, db, count=True)
    lv = out["leaves"]
    gx, gm = api.grav_short_adjoint(ctx, lv, db.gp, db.m, 2.0 * out["acc"])
    gas_t = (db.species == 0).float()
    gx2, gm2 = api.geometry_adjoint(ctx, lv, db.m, out["V"], gas_t)
    torch.cuda.synchronize()
    host = {k: v.cpu().numpy() for k, v in out.items() if isinstance(v, torch.Tensor)}
    host.update(gx=gx.cpu().numpy().T, gm=gm.cpu().numpy(), gx2=gx2.cpu().numpy().T, gm2=gm2.cpu().numpy())
    for k in ("acc", "dv", "B", "gA", "gB"):
        host[k] = host[k].T
    host["export"] = lv.export()
    return host


def test_clustered_2x64_full(tmp_path):
    b = W.clustered()
    g = gpu_forward_and_adjoint(b)
    I = O.from_box(b)
    perm, start = O.leaves_rcb(I, b.max_leaf)
    assert np.array_equal(g["export"]["perm"], perm)
    assert np.array_equal(g["export"]["leaf_start"], start)
    for hyd, key in ((False, "grav"), (True, "hydro")):
        ptr, lst = O.leaf_pairs(I, perm, start, hydro=hyd)
        assert np.array_equal(g["export"][key + "_ptr"], ptr)
        assert np.array_equal(g["export"][key + "_list"], lst)
    ref = O.forward(I, W.GAMMA, W.AV_ALPHA, W.AV_BETA, W.AV_ETA2)
    gas = b.species == 0
    where = "clustered_2x64^3"
    check(where, "acc", g["acc"], ref["acc"])
    for k in ("dv", "du", "V", "rho", "A", "B", "gA", "gB"):
        check(where, k, g[k][gas], ref[k][gas])
    ogx, ogm = O.gravity_adjoint(I, 2.0 * ref["acc"])
    ogx2, ogm2 = O.geometry_adjoint(I, gas.astype(np.float64))
    check(where, "grav_gx", g["gx"], ogx, "gx", exclude=cut_boundary_particles(I.pos, b.L, b.r_cut))
    check(where, "grav_gm", g["gm"], ogm, "gm")
    check(where, "geom_gx", g["gx2"], ogx2, "gx")
    check(where, "geom_gm", g["gm2"], ogm2, "gm")


def test_large_2x256_sampled():
    b = W.large()
    g = gpu_forward_and_adjoint(b)
    I = O.from_box(b)
    # leaves of the whole box by the oracle's own RCB
    perm, start = O.leaves_rcb(I, b.max_leaf)
    assert np.array_equal(g["export"]["perm"], perm)
    assert np.array_equal(g["export"]["leaf_start"], start)
    rng = np.random.default_rng(W.SEEDS["large"] + 1)
    asub = np.sort(rng.choice(start.size - 1, 64, replace=False)).astype(np.int32)
    for hyd, key in ((False, "grav"), (True, "hydro")):
        ptr, lst = O.leaf_pairs(I, perm, start, hydro=hyd, asub=asub)
        gptr, glist = g["export"][key + "_ptr"], g["export"][key + "_list"]
        for q, a in enumerate(asub):
            assert np.array_equal(glist[gptr[a]:gptr[a + 1]], lst[ptr[q]:ptr[q + 1]]), (key, a)
    # sampled outputs through the oracle's own chain
    sample = rng.choice(b.n, 384, replace=False)
    r = O.sampled_chain(I, sample, W.GAMMA, W.AV_ALPHA, W.AV_BETA, W.AV_ETA2)
    gas_s = sample[b.species[sample] == 0]
    where = "large_2x256^3/sample384"
    for k in ("acc", "gm"):
        check(where, k, g[k][sample], r[k][sample])
    check(where, "gx", g["gx"][sample], r["gx"][sample],
          exclude=cut_boundary_particles(I.pos, b.L, b.r_cut, subset=sample))
    for k in ("dv", "du", "V", "A", "B"):
        check(where, k, g[k][gas_s], r[k][gas_s])
    # FP64 conservation sums of the whole box: momentum and energy rates vanish up to FP32 rounding
    cons = g["cons"]
    gas = b.species == 0
    scale_p = float(np.sum(np.abs(b.m[gas, None] * g["dv"][gas])))
    assert np.max(np.abs(cons[:3])) < 1e-5 * scale_p
    assert int(g["n_singular"][0]) == 0
