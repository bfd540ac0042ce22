"""The allocation-free gravity entry point, grav_short_noalloc, against grav_short.

Some callers cannot let a library allocate device memory: an application
whose own memory pool already owns the GPU, or a step loop that must never
pay the synchronisation cudaMalloc/cudaFree can imply.  They call
grav_short_noalloc, which keeps its scratch in a fixed device array inside
libcrk.  These tests call it through the C ABI and check that it returns
what grav_short returns, on two calls in a row with different masses (the
shared array keeps the previous call's contents), and that it refuses a box
larger than its fixed limit without touching the output.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    a = a.double()
    b = b.double()
    return float(torch.sqrt(((a - b) ** 2).sum() / (b * b).sum().clamp_min(1e-300)))


@pytest.fixture(scope="module")
def setup():
    from paper_2310_16122_gb300 import api, native
    from paper_2310_16122_gb300.build import build_library

    build_library()
    return api, native, api.Context(0)


@pytest.mark.parametrize("variant", ["tiles", "lists"])
def test_noalloc_matches_grav_short_on_two_calls(setup, variant):
    """Both branches of the entry point (the tiles kernel, and the lists kernel when the
    gravity variant is lists and the leaves were built with gravity lists) against
    grav_short in the same variant: within the gravity tolerance, and bit for bit."""
    api, N, ctx = setup
    from paper_2310_16122_gb300 import workloads as W

    b = W.clustered_box(16, 2, 4242)
    db = api.DeviceBox(b)
    ctx.set_variant("gravity", 0 if variant == "lists" else 1)
    try:
        lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
        gp = db.gp.c()
        for m in (db.m, db.m * 1.7 + 0.05):
            ref, _ = api.grav_short(ctx, lv, db.gp, m)
            out = torch.full((3, b.n), float("nan"), device="cuda")
            st = N.lib().grav_short_noalloc(ctx.handle, lv.handle, ctypes.byref(gp), ctypes.c_void_p(m.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()))
            assert st == N.CRK_OK
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert _rel_l2(out, ref) <= 2e-5
            assert torch.equal(out, ref)
    finally:
        ctx.set_variant("gravity", 1)


def test_noalloc_rejects_boxes_above_its_limit(setup):
    api, N, ctx = setup
    from paper_2310_16122_gb300 import workloads as W

    n = N.NOALLOC_MAX_PARTICLES + 1
    b = W.random_box(n, 100.0, 0.5, 4243, h=0.6)
    db = api.DeviceBox(b)
    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    gp = db.gp.c()
    out = torch.full((3, n), float("nan"), device="cuda")
    st = N.lib().grav_short_noalloc(ctx.handle, lv.handle, ctypes.byref(gp), ctypes.c_void_p(db.m.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()))
    torch.cuda.synchronize()
    assert st == N.CRK_ETOOLARGE
    assert torch.isnan(out).all()
