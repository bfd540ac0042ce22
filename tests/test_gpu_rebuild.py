"""Capture-safe leaf rebuild and the batched driver's graph (leaf rebuild + whole step).

crk_leaves_rebuild recomputes leaves in place for moved particles with no host
synchronisation; it must give exactly the leaves a fresh build of the moved
particles gives (bit for bit: permutation, leaf starts, leaf-pair lists) and
exactly the same step outputs.  The graph of rebuild + step, replayed after the
positions change in place, must equal an eager fresh build + step, also with
persistent kernels.  What a build checks on the host becomes a status bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2310_16122_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2310_16122_gb300 import api as A
    from paper_2310_16122_gb300.build import build_library

    build_library()
    return A


def moved(b, seed, sigma=0.05):
    """A copy of box b with every particle displaced by N(0, sigma^2) per axis, wrapped into [0, L)."""
    import copy

    c = copy.copy(b)
    rng = np.random.default_rng(seed)
    for k in ("x", "y", "z"):
        v = getattr(b, k).astype(np.float64) + rng.normal(0.0, sigma, b.n)
        v = np.mod(v, b.L).astype(np.float32)
        v = np.where(v >= np.float32(b.L), np.float32(0.0), v)  # rounding up to L wraps to 0
        setattr(c, k, v)
    return c



BOXES = [W.clustered_box(12, 1, 71), W.clustered_box(14, 2, 72), W.random_box(900, 11.0, 0.5, 73, h=0.8)]


def set_positions(dst, boxes):
    for k in ("x", "y", "z"):
        getattr(dst, k).copy_(torch.as_tensor(np.concatenate([getattr(b, k) for b in boxes])))


def exports_equal(a, b):
    for k in ("perm", "leaf_start", "grav_ptr", "grav_list", "hydro_ptr", "hydro_list"):
        assert np.array_equal(a[k], b[k]), k


OUTS = ("acc", "dv", "du", "V", "rho", "A", "B", "gA", "gB", "gx_grav", "gm_grav", "gx_geom", "gm_geom")


def assert_outputs_equal(io_a, io_b, step):
    """Every step output bit for bit; on a mismatch, report every output that differs and by how much."""
    bad = {}
    for k in OUTS:
        a, b = getattr(io_a, k), getattr(io_b, k)
        if a is None:
            continue
        same = (a == b) | (torch.isnan(a) & torch.isnan(b))  # singular particles are NaN in both
        if not bool(same.all()):
            d = torch.where(same, torch.zeros_like(a), (a - b).abs())
            bad[k] = (int((~same).sum()), float(torch.nan_to_num(d, nan=float("inf")).max()))
    assert not bad, (step, bad)


def test_rebuild_equals_fresh_build(api):
    ctx = api.Context(0)
    boxes = BOXES
    dbt = api.DeviceBatch(boxes)
    lv = api.build_leaves_batch(ctx, dbt)
    assert lv.status() == 0
    io_r = api.StepIO(ctx, dbt)
    for step in range(3):  # three successive moves of the same particles
        now = [moved(b, 10 * step + k) for k, b in enumerate(boxes)]
        set_positions(dbt, now)
        api.rebuild_leaves(ctx, lv, dbt)
        api.step(ctx, lv, dbt, io_r)
        assert lv.status() == 0
        fresh = api.build_leaves_batch(ctx, dbt)
        io_f = api.StepIO(ctx, dbt)
        api.step(ctx, fresh, dbt, io_f)
        torch.cuda.synchronize()
        exports_equal(lv.export(), fresh.export())
        assert (lv.n_grav_pairs, lv.n_hydro_pairs) == (fresh.n_grav_pairs, fresh.n_hydro_pairs)
        assert_outputs_equal(io_r, io_f, step)
        fresh.free()
        boxes = now


def test_single_box_rebuild(api):
    from paper_2310_16122_gb300 import native as N

    ctx = api.Context(0)
    b = W.clustered_box(16, 3, 74)
    db = api.DeviceBox(b)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    b2 = moved(b, 5)
    for k in ("x", "y", "z"):
        getattr(db, k).copy_(torch.as_tensor(getattr(b2, k)))
    api.rebuild_leaves(ctx, lv, db)
    assert lv.status() == 0
    fresh = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    exports_equal(lv.export(), fresh.export())
    # the chaining mesh rebuilds too
    t = W.tiny()
    dt = api.DeviceBox(t)
    lm = api.build_leaves(ctx, dt.x, dt.y, dt.z, dt.species, dt.h, dt.L, dt.lp)
    t2 = moved(t, 6)
    for k in ("x", "y", "z"):
        getattr(dt, k).copy_(torch.as_tensor(getattr(t2, k)))
    api.rebuild_leaves(ctx, lm, dt)
    assert lm.status() == 0
    exports_equal(lm.export(), api.build_leaves(ctx, dt.x, dt.y, dt.z, dt.species, dt.h, dt.L, dt.lp).export())
    # inputs that do not belong to the leaves are refused before anything runs
    other = api.DeviceBox(W.clustered_box(12, 1, 75))
    with pytest.raises(N.CrkError) as e:
        api.rebuild_leaves(ctx, lv, other)
    assert e.value.status == N.CRK_ESTATE


@pytest.mark.parametrize("persistent", [False, True])
def test_rebuild_step_graph(api, persistent):
    st = torch.cuda.Stream()  # capture needs a stream other than the legacy default stream
    with torch.cuda.stream(st):
        rebuild_step_graph(api, persistent, st)


def rebuild_step_graph(api, persistent, st):
    ctx = api.Context(0, stream=st)
    ctx.set_persistent(persistent)
    boxes = BOXES
    dbt = api.DeviceBatch(boxes)
    lv = api.build_leaves_batch(ctx, dbt)
    io = api.StepIO(ctx, dbt)
    g = api.RebuildStepGraph(ctx, lv, dbt, io)
    for step in range(2):
        now = [moved(b, 50 + 10 * step + k) for k, b in enumerate(boxes)]
        set_positions(dbt, now)
        g.launch()
        assert lv.status() == 0
        fresh = api.build_leaves_batch(ctx, dbt)
        io_f = api.StepIO(ctx, dbt)
        api.step(ctx, fresh, dbt, io_f)
        torch.cuda.synchronize()
        assert_outputs_equal(io, io_f, step)
        # FP64 conservation sums: per-block partials (the persistent queue deals leaves to blocks in any order)
        assert torch.allclose(io.cons, io_f.cons, rtol=1e-9, atol=0.0, equal_nan=True)  # NaN: singular particles
        fresh.free()
        boxes = now
    g.close()


def test_rebuild_status_reports_a_changed_gas_count(api):
    from paper_2310_16122_gb300 import native as N

    ctx = api.Context(0)
    b = W.clustered_box(12, 1, 76)
    db = api.DeviceBox(b)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    gas = np.nonzero(b.species == 0)[0]
    db.species[int(gas[3])] = 1  # one gas particle becomes dark matter
    api.rebuild_leaves(ctx, lv, db)
    s = lv.status()
    assert s & 4, N.LEAVES_STATUS
    db.species[int(gas[3])] = 0
    api.rebuild_leaves(ctx, lv, db)
    assert lv.status() == 0
