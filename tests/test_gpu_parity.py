"""GPU parity: libcrk (through its C ABI) against the FP64 oracle on the same seeded inputs.

Integer results (leaf permutation, leaf starts, leaf-pair lists) must be
bit-exact.  Floating point is gated on the global relative L2 error
E = sqrt(sum |dx|^2 / sum |x_ref|^2) (gravity and hydro accelerations
E <= 2e-5, du/dt E <= 5e-5) and on the largest per-particle relative error
e_i = |dx_i| / (|x_ref,i| + 0.01 rms|x_ref|); the gates of the other outputs
are in tests/_errors.py.
Pair counts come from FP32 range tests on the GPU and FP64 tests in the
oracle; they may differ only for pairs within rounding of the cut.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2310_16122_gb300 import workloads as W
from tests._errors import check, cut_boundary_particles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2310_16122_gb300 import api as A
    from paper_2310_16122_gb300.build import build_library

    build_library()
    return A


@pytest.fixture(scope="module")
def ctx(api):
    return api.Context(0)


BOXES = {
    "tiny_mesh": lambda: W.tiny(),
    "clustered12": lambda: W.clustered_box(12, 1, 31),
    "clustered24": lambda: W.clustered_box(24, 11, 32),
    "random1000_leaf7": lambda: W.random_box(1000, 12.0, 0.5, 33, max_leaf=7, h=0.9),
    "random777_mesh3": lambda: W.random_box(777, 13.0, 0.4, 34, h=2.0, leaf_mode=0, cells=3),
    "random2_leaf1": lambda: W.random_box(2, 12.0, 1.0, 35, max_leaf=1, h=0.5),
    "random1": lambda: W.random_box(1, 12.0, 1.0, 36, h=0.5),
}
_cache = {}


def boundary_pairs(b, hydro):
    """Ordered pairs whose r^2 lies within FP32 rounding (4e-7 relative) of cut^2.

    The GPU decides r^2 < cut^2 in FP32 and the oracle in FP64, so only these
    pairs may be counted differently.  Adaptive h puts each gas particle's
    58th neighbour at r = 2h by construction, so such pairs do occur.
    """
    from scipy.spatial import cKDTree

    pos = np.stack([b.x, b.y, b.z], 1).astype(np.float64)
    h = b.h.astype(np.float64)
    idx = np.nonzero(b.species == 0)[0] if hydro else np.arange(b.n)
    if idx.size < 2:
        return 0
    rmax = (2.0 * h[idx].max() if hydro else float(np.float32(b.r_cut))) * (1 + 1e-6)
    pts = np.where(pos[idx] >= b.L, pos[idx] - b.L, pos[idx])
    pr = cKDTree(pts, boxsize=b.L).query_pairs(rmax, output_type="ndarray")
    i, j = idx[pr[:, 0]], idx[pr[:, 1]]
    d = pos[i] - pos[j]
    d -= b.L * np.rint(d / b.L)
    r2 = np.sum(d * d, axis=1)
    c2 = (h[i] + h[j]) ** 2 if hydro else np.full(i.shape, float(np.float32(b.r_cut)) ** 2)
    return 2 * int(np.count_nonzero(np.abs(r2 - c2) <= 4e-7 * c2))  # ordered pairs


def box_of(name):
    if name not in _cache:
        _cache[name] = BOXES[name]()
    return _cache[name]


def oracle_leaves(I, b):
    if b.leaf_mode == 0:
        return O.leaves_mesh(I, b.cells_per_side)
    return O.leaves_rcb(I, b.max_leaf)


@pytest.mark.parametrize("name", list(BOXES))
def test_leaves_bit_exact(api, ctx, name):
    b = box_of(name)
    db = api.DeviceBox(b)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    ex = lv.export()
    I = O.from_box(b)
    perm, start = oracle_leaves(I, b)
    assert np.array_equal(ex["perm"], perm)
    assert np.array_equal(ex["leaf_start"], start)
    for hyd, key in ((False, "grav"), (True, "hydro")):
        ptr, lst = O.leaf_pairs(I, perm, start, hydro=hyd)
        assert np.array_equal(ex[key + "_ptr"], ptr), key
        assert np.array_equal(ex[key + "_list"], lst), key


def test_empty_input(api, ctx):
    z = torch.zeros(0, device="cuda")
    lv = api.build_leaves(ctx, z, z, z, torch.zeros(0, dtype=torch.uint8, device="cuda"), z, 16.0,
                          api.LeafParams(1, 0, 128, 3.0))
    assert lv.n == 0 and lv.n_leaves == 0
    a, c = api.grav_short(ctx, lv, api.GravParams(0.1, 3.0, tuple(W.gravity_poly())), z, count=True)
    V, rho, _ = api.geometry(ctx, lv, z)
    assert a.numel() == 0 and V.numel() == 0


def test_variant_switch(api, ctx):
    from paper_2310_16122_gb300 import native as N

    assert ctx.get_variant("hydro") == 0 and ctx.get_variant("gravity") == 1
    with pytest.raises(N.CrkError):
        ctx.set_variant("gravity", N.N_VARIANTS)
    ctx.set_variant("hydro", 1)
    assert ctx.get_variant("hydro") == 1
    ctx.set_variant("hydro", 0)


def test_error_statuses(api, ctx):
    from paper_2310_16122_gb300 import native as N

    b = W.random_box(100, 10.0, 0.5, 40, h=0.5)
    db = api.DeviceBox(b)
    with pytest.raises(N.CrkError) as e:
        api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, api.LeafParams(1, 0, 128, 5.0))
    assert e.value.status == N.CRK_EBOX
    with pytest.raises(N.CrkError) as e:
        api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, 5.0, api.LeafParams(1, 0, 128, 2.0))
    assert e.value.status == N.CRK_EBOX  # positions outside [0, 5)
    with pytest.raises(N.CrkError) as e:
        api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, api.LeafParams(7, 0, 128, 2.0))
    assert e.value.status == N.CRK_EINVAL
    hbig = db.h * 0 + 3.0
    with pytest.raises(N.CrkError) as e:
        api.build_leaves(ctx, db.x, db.y, db.z, db.species, hbig, db.L, api.LeafParams(1, 0, 128, 2.0))
    assert e.value.status == N.CRK_EBOX  # 2 h_max >= box/2


VARIANTS = [0, 1, 2, 3, 4]
VARIANT_IDS = ["lists", "tiles", "tiles16", "tiles8", "ring16"]
# the gravity kernels also have the half-warp leaf-pair arms (shuffle, shared memory, second load)
# and the split sweep over 8-particle sub-cells
GRAV_VARIANTS = VARIANTS + [5, 6, 7, 8]
GRAV_VARIANT_IDS = VARIANT_IDS + ["halfwarp_shfl", "halfwarp_smem", "halfwarp_load", "split8"]


@pytest.mark.parametrize("variant", GRAV_VARIANTS, ids=GRAV_VARIANT_IDS)
@pytest.mark.parametrize("name", ["tiny_mesh", "clustered24", "random1000_leaf7", "random777_mesh3"])
def test_gravity_parity(api, ctx, name, variant):
    b = box_of(name)
    db = api.DeviceBox(b)
    ctx.set_variant("gravity", variant)
    try:
        lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
        a, cnt = api.grav_short(ctx, lv, db.gp, db.m, count=True)
    finally:
        ctx.set_variant("gravity", 1)
    I = O.from_box(b)
    ref, npairs = O.gravity(I)
    check(f"gravity/{name}/v{variant}", "acc", a.cpu().numpy().T, ref)
    assert abs(int(cnt.item()) - npairs) <= boundary_pairs(b, False)


@pytest.mark.parametrize("shape", [(False, 64, 2), (True, 96, 2), (True, 32, 4)], ids=["d64w2", "pers_d96w2", "pers_d32w4"])
@pytest.mark.parametrize("name", ["clustered24", "random1000_leaf7"])
def test_gravity_launch_shapes(api, ctx, name, shape):
    """The packed gravity tiles and their adjoint in other launch shapes (persistent, j-tile depth,
    warps per leaf) against the oracle."""
    b = box_of(name)
    db = api.DeviceBox(b)
    for k in ("gravity", "gravity_adjoint"):
        ctx.set_launch(k, *shape)
    try:
        lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
        a, cnt = api.grav_short(ctx, lv, db.gp, db.m, count=True)
        gx, gm = api.grav_short_adjoint(ctx, lv, db.gp, db.m, 2.0 * a)
        torch.cuda.synchronize()
    finally:
        for k in ("gravity", "gravity_adjoint"):
            ctx.set_launch(k, False, 32, 4)
    I = O.from_box(b)
    ref, npairs = O.gravity(I)
    where = f"gravity_shape/{name}/{shape}"
    check(where, "acc", a.cpu().numpy().T, ref)
    assert abs(int(cnt.item()) - npairs) <= boundary_pairs(b, False)
    ogx, ogm = O.gravity_adjoint(I, 2.0 * ref)
    check(where, "grav_gx", gx.cpu().numpy().T, ogx, "gx", exclude=cut_boundary_particles(I.pos, b.L, b.r_cut))
    check(where, "grav_gm", gm.cpu().numpy(), ogm, "gm")


GAS_KERNELS = ("geometry", "corrections", "hydro", "geometry_adjoint", "gravity", "gravity_adjoint")


def set_gas_variant(ctx, variant):
    """variant for every pair kernel; None restores the defaults (lists for gas, tiles for gravity)"""
    for k in GAS_KERNELS:
        ctx.set_variant(k, (1 if k.startswith("gravity") else 0) if variant is None else variant)


# the hydro pass also has the half-warp arms (the other gas kernels then run tiles)
@pytest.mark.parametrize("variant", GRAV_VARIANTS, ids=GRAV_VARIANT_IDS)
@pytest.mark.parametrize("name", ["tiny_mesh", "clustered12", "clustered24", "random777_mesh3"])
def test_hydro_chain_parity(api, ctx, name, variant):
    b = box_of(name)
    db = api.DeviceBox(b)
    set_gas_variant(ctx, variant)
    try:
        out = api.forward(ctx, db, count=True)
        torch.cuda.synchronize()
    finally:
        set_gas_variant(ctx, None)
    I = O.from_box(b)
    ref = O.forward(I, W.GAMMA, W.AV_ALPHA, W.AV_BETA, W.AV_ETA2)
    gas = b.species == 0
    got = {"V": out["V"].cpu().numpy(), "rho": out["rho"].cpu().numpy(), "A": out["A"].cpu().numpy(),
           "B": out["B"].cpu().numpy().T, "gA": out["gA"].cpu().numpy().T, "gB": out["gB"].cpu().numpy().T,
           "dv": out["dv"].cpu().numpy().T, "du": out["du"].cpu().numpy()}
    assert int(out["n_singular"].item()) == ref["singular"] == 0
    for k, g in got.items():
        check(f"hydro_chain/{name}/v{variant}", k, g[gas], ref[k][gas])
    # DM entries of gas-only outputs are zero
    assert float(out["V"][torch.as_tensor(~gas, device="cuda")].abs().max()) == 0.0 if (~gas).any() else True
    # conservation sums accumulated in FP64 on the GPU
    cons = out["cons"].cpu().numpy()
    scale = np.abs(I.m[gas, None] * ref["dv"][gas]).sum()
    assert np.max(np.abs(cons[:3])) < 1e-5 * scale
    assert abs(int(out["count_hydro"].item()) - ref["pairs_hydro"]) <= boundary_pairs(b, True)
    if variant < 5:
        assert int(out["count_geom"].item()) == int(out["count_hydro"].item())
    else:  # the half-warp arm decides boundary pairs in the frame of the lower leaf, geometry in i's
        assert abs(int(out["count_geom"].item()) - int(out["count_hydro"].item())) <= boundary_pairs(b, True)


@pytest.mark.parametrize("variant", GRAV_VARIANTS, ids=GRAV_VARIANT_IDS)
@pytest.mark.parametrize("name", ["clustered12", "clustered24"])
def test_adjoint_parity(api, ctx, name, variant):
    b = box_of(name)
    db = api.DeviceBox(b)
    set_gas_variant(ctx, variant)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    a, _ = api.grav_short(ctx, lv, db.gp, db.m)
    gx, gm = api.grav_short_adjoint(ctx, lv, db.gp, db.m, 2.0 * a)
    V, rho, _ = api.geometry(ctx, lv, db.m)
    gas_t = (db.species == 0).float()
    gx2, gm2 = api.geometry_adjoint(ctx, lv, db.m, V, gas_t)
    torch.cuda.synchronize()
    set_gas_variant(ctx, None)
    I = O.from_box(b)
    ref_a, _ = O.gravity(I)
    ogx, ogm = O.gravity_adjoint(I, 2.0 * ref_a)
    ogx2, ogm2 = O.geometry_adjoint(I, (b.species == 0).astype(np.float64))
    where = f"adjoint/{name}/v{variant}"
    bnd = cut_boundary_particles(I.pos, b.L, b.r_cut)
    check(where, "grav_gx", gx.cpu().numpy().T, ogx, "gx", exclude=bnd)
    check(where, "grav_gm", gm.cpu().numpy(), ogm, "gm")
    check(where, "geom_gx", gx2.cpu().numpy().T, ogx2, "gx")
    check(where, "geom_gm", gm2.cpu().numpy(), ogm2, "gm")
