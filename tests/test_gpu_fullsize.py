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
    e = {"acc": rel_l2(g["acc"], ref["acc"]), "dv": rel_l2(g["dv"][gas], ref["dv"][gas]),
         "du": rel_l2(g["du"][gas], ref["du"][gas]), "V": rel_l2(g["V"][gas], ref["V"][gas]),
         "A": rel_l2(g["A"][gas], ref["A"][gas]), "B": rel_l2(g["B"][gas], ref["B"][gas]),
         "gA": rel_l2(g["gA"][gas], ref["gA"][gas]), "gB": rel_l2(g["gB"][gas], ref["gB"][gas])}
    ogx, ogm = O.gravity_adjoint(I, 2.0 * ref["acc"])
    ogx2, ogm2 = O.geometry_adjoint(I, gas.astype(np.float64))
    e.update(grav_gx=rel_l2(g["gx"], ogx), grav_gm=rel_l2(g["gm"], ogm), geom_gx=rel_l2(g["gx2"], ogx2),
             geom_gm=rel_l2(g["gm2"], ogm2))
    print("clustered 2x64^3:", {k: f"{v:.2e}" for k, v in e.items()})
    assert e["acc"] <= 2e-5 and e["dv"] <= 2e-5 and e["du"] <= 5e-5
    assert e["V"] < 1e-5 and e["A"] < 1e-5 and max(e["B"], e["gA"], e["gB"]) < 1e-3
    assert max(e["grav_gx"], e["grav_gm"], e["geom_gx"], e["geom_gm"]) < 1e-4


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
    e = {"acc": rel_l2(g["acc"][sample], r["acc"][sample]),
         "gx": rel_l2(g["gx"][sample], r["gx"][sample]), "gm": rel_l2(g["gm"][sample], r["gm"][sample]),
         "dv": rel_l2(g["dv"][gas_s], r["dv"][gas_s]), "du": rel_l2(g["du"][gas_s], r["du"][gas_s]),
         "V": rel_l2(g["V"][gas_s], r["V"][gas_s]), "A": rel_l2(g["A"][gas_s], r["A"][gas_s]),
         "B": rel_l2(g["B"][gas_s], r["B"][gas_s])}
    print("large 2x256^3 sample:", {k: f"{v:.2e}" for k, v in e.items()})
    assert e["acc"] <= 2e-5 and e["dv"] <= 2e-5 and e["du"] <= 5e-5
    assert e["V"] < 1e-5 and e["A"] < 1e-5 and e["B"] < 1e-3 and max(e["gx"], e["gm"]) < 1e-4
    # FP64 conservation sums of the whole box: momentum and energy rates vanish up to FP32 rounding
    cons = g["cons"]
    gas = b.species == 0
    scale_p = float(np.sum(np.abs(b.m[gas, None] * g["dv"][gas])))
    assert np.max(np.abs(cons[:3])) < 1e-5 * scale_p
    assert int(g["n_singular"][0]) == 0
