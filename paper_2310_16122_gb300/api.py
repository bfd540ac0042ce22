"""PyTorch-facing wrappers of libcrk (device memory and streams from torch; compute in CUDA).

Tensors are CUDA, contiguous, float32 (species uint8), in the caller's
original particle order; vectors are component-major (3, n).  Every call is
asynchronous on the context's stream (the torch stream given at creation).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import native as N


def _f32(t: torch.Tensor, name: str, numel: int | None = None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


class Context:
    """Owns a crk_ctx bound to one device and one torch stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        L = N.lib()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        st = L.crk_create(ctypes.byref(h), int(device), ctypes.c_void_p(self.stream.cuda_stream))
        if st != N.CRK_OK:
            raise N.CrkError(st, "crk_create failed")
        self.handle = h

    def check(self, status: int) -> None:
        N.check(status, self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            N.lib().crk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_variant(self, kernel: str, variant: int) -> None:
        self.check(N.lib().crk_set_variant(self.handle, N.KERNELS[kernel], int(variant)))

    def set_persistent(self, on: bool) -> None:
        self.check(N.lib().crk_set_persistent(self.handle, int(bool(on))))

    def set_launch(self, kernel: str, persistent: bool, depth: int = 32, warps: int = 4) -> None:
        self.check(N.lib().crk_set_launch(self.handle, N.KERNELS[kernel], int(bool(persistent)), int(depth),
                                          int(warps)))

    def get_launch(self, kernel: str) -> tuple:
        """(persistent, depth, warps per leaf) of one pair kernel."""
        p, d, w = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        self.check(N.lib().crk_get_launch(self.handle, N.KERNELS[kernel], ctypes.byref(p), ctypes.byref(d),
                                          ctypes.byref(w)))
        return bool(p.value), int(d.value), int(w.value)

    def get_variant(self, kernel: str) -> int:
        v = ctypes.c_int(0)
        self.check(N.lib().crk_get_variant(self.handle, N.KERNELS[kernel], ctypes.byref(v)))
        return int(v.value)

    def empty(self, *shape, dtype=torch.float32):
        return torch.empty(*shape, dtype=dtype, device=self.device)


@dataclass
class LeafParams:
    mode: int = 1            # 0 chaining mesh, 1 RCB
    cells_per_side: int = 0
    max_leaf: int = 128
    r_cut_grav: float = 3.0


@dataclass
class GravParams:
    eps: float
    r_cut: float
    poly: tuple

    def c(self) -> N.crk_grav_params:
        g = N.crk_grav_params()
        g.eps = self.eps
        g.r_cut = self.r_cut
        for k in range(6):
            g.poly[k] = float(self.poly[k])
        return g


@dataclass
class HydroParams:
    gamma: float = 5.0 / 3.0
    alpha: float = 1.0
    beta: float = 2.0
    eta2: float = 0.01

    def c(self) -> N.crk_hydro_params:
        return N.crk_hydro_params(self.gamma, self.alpha, self.beta, self.eta2)


class Leaves:
    """A leaf build (library-owned device buffers)."""

    def __init__(self, ctx: Context, handle: ctypes.c_void_p, keep: tuple):
        self.ctx = ctx
        self.handle = handle
        self._keep = keep  # input tensors must outlive nothing after the build, kept for safety
        info = (ctypes.c_int64 * 6)()
        ctx.check(N.lib().crk_leaves_info(handle, info))
        self.n, self.n_leaves, self.n_grav_pairs, self.n_hydro_pairs, self.n_grav_images, self.n_hydro_images = \
            (int(v) for v in info)

    def export(self) -> dict:
        nl = self.n_leaves
        out = dict(perm=np.zeros(max(self.n, 1), np.int32), leaf_start=np.zeros(nl + 1, np.int32),
                   grav_ptr=np.zeros(nl + 1, np.int32), grav_list=np.zeros(max(self.n_grav_pairs, 1), np.int32),
                   hydro_ptr=np.zeros(nl + 1, np.int32), hydro_list=np.zeros(max(self.n_hydro_pairs, 1), np.int32))
        p = {k: v.ctypes.data_as(ctypes.c_void_p) for k, v in out.items()}
        self.ctx.check(N.lib().crk_leaves_export(self.ctx.handle, self.handle, p["perm"], p["leaf_start"],
                                                 p["grav_ptr"], p["grav_list"], p["hydro_ptr"], p["hydro_list"]))
        out["perm"] = out["perm"][:self.n]
        out["grav_list"] = out["grav_list"][:self.n_grav_pairs]
        out["hydro_list"] = out["hydro_list"][:self.n_hydro_pairs]
        return out

    def status(self) -> int:
        """Status word of the last build or rebuild (synchronises; 0 = valid), and fresh counts."""
        s = ctypes.c_int(0)
        self.ctx.check(N.lib().crk_leaves_status(self.ctx.handle, self.handle, ctypes.byref(s)))
        info = (ctypes.c_int64 * 6)()
        self.ctx.check(N.lib().crk_leaves_info(self.handle, info))
        self.n, self.n_leaves, self.n_grav_pairs, self.n_hydro_pairs, self.n_grav_images, self.n_hydro_images = \
            (int(v) for v in info)
        return int(s.value)

    def free(self) -> None:
        if self.handle:
            # a closed context cannot take the buffers back: free them directly
            N.lib().crk_leaves_free(self.ctx.handle if self.ctx.handle else None, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_leaves(ctx: Context, x, y, z, species, h, box: float, lp: LeafParams) -> Leaves:
    n = x.numel()
    p = N.crk_particles(_f32(x, "x", n) if n else 0, _f32(y, "y", n) if n else 0, _f32(z, "z", n) if n else 0,
                        species.data_ptr() if n else 0, n, float(box))
    if n and (species.dtype != torch.uint8 or not species.is_cuda or species.numel() != n):
        raise TypeError("species must be a CUDA uint8 tensor of length n")
    c = N.crk_leaf_params(int(lp.mode), int(lp.cells_per_side), int(lp.max_leaf), float(lp.r_cut_grav))
    out = ctypes.c_void_p()
    ctx.check(N.lib().crk_build_leaves(ctx.handle, ctypes.byref(p), _f32(h, "h", n) if n else None,
                                       ctypes.byref(c), ctypes.byref(out)))
    return Leaves(ctx, out, (x, y, z, species, h))


def _count(ctx, want):
    return torch.zeros(1, dtype=torch.int64, device=ctx.device) if want else None


def geometry(ctx: Context, lv: Leaves, m, count=False):
    n = lv.n
    V, rho = ctx.empty(n), ctx.empty(n)
    c = _count(ctx, count)
    ctx.check(N.lib().crk_geometry(ctx.handle, lv.handle, _f32(m, "m", n), V.data_ptr(), rho.data_ptr(),
                                   c.data_ptr() if c is not None else None))
    return V, rho, c


def corrections(ctx: Context, lv: Leaves, V):
    n = lv.n
    A, B, gA, gB = ctx.empty(n), ctx.empty(3, n), ctx.empty(3, n), ctx.empty(9, n)
    ns = torch.zeros(1, dtype=torch.int32, device=ctx.device)
    ctx.check(N.lib().crk_corrections(ctx.handle, lv.handle, _f32(V, "V", n), A.data_ptr(), B.data_ptr(),
                                      gA.data_ptr(), gB.data_ptr(), ns.data_ptr()))
    return A, B, gA, gB, ns


def hydro(ctx: Context, lv: Leaves, hp: HydroParams, m, v3, u, V, rho, A, B, gA, gB, count=False):
    n = lv.n
    dv, du = ctx.empty(3, n), ctx.empty(n)
    cons = torch.zeros(4, dtype=torch.float64, device=ctx.device)
    c = _count(ctx, count)
    hpc = hp.c()
    ctx.check(N.lib().crk_hydro(ctx.handle, lv.handle, ctypes.byref(hpc), _f32(m, "m", n), _f32(v3, "v3", 3 * n),
                                _f32(u, "u", n), _f32(V, "V", n), _f32(rho, "rho", n), _f32(A, "A", n),
                                _f32(B, "B", 3 * n), _f32(gA, "gradA", 3 * n), _f32(gB, "gradB", 9 * n),
                                dv.data_ptr(), du.data_ptr(), cons.data_ptr(),
                                c.data_ptr() if c is not None else None))
    return dv, du, cons, c


def extras(ctx: Context, lv: Leaves, m, v3, V, A, B, gA, gB, count=False):
    """Corrected-kernel density rho_r [n] and velocity gradient dvdx [9, n] (dvdx[3a+b] = dv^a/dx^b)."""
    n = lv.n
    rho_r, dvdx = ctx.empty(n), ctx.empty(9, n)
    c = _count(ctx, count)
    ctx.check(N.lib().crk_extras(ctx.handle, lv.handle, _f32(m, "m", n), _f32(v3, "v3", 3 * n), _f32(V, "V", n),
                                 _f32(A, "A", n), _f32(B, "B", 3 * n), _f32(gA, "gradA", 3 * n),
                                 _f32(gB, "gradB", 9 * n), rho_r.data_ptr(), dvdx.data_ptr(),
                                 c.data_ptr() if c is not None else None))
    return rho_r, dvdx, c


def hydro_limited(ctx: Context, lv: Leaves, hp: HydroParams, m, v3, u, V, rho, A, B, gA, gB, dvdx, count=False):
    """crk_hydro with the limited viscosity fed by the Extras velocity gradient."""
    n = lv.n
    dv, du = ctx.empty(3, n), ctx.empty(n)
    cons = torch.zeros(4, dtype=torch.float64, device=ctx.device)
    c = _count(ctx, count)
    hpc = hp.c()
    ctx.check(N.lib().crk_hydro_limited(ctx.handle, lv.handle, ctypes.byref(hpc), _f32(m, "m", n),
                                        _f32(v3, "v3", 3 * n), _f32(u, "u", n), _f32(V, "V", n),
                                        _f32(rho, "rho", n), _f32(A, "A", n), _f32(B, "B", 3 * n),
                                        _f32(gA, "gradA", 3 * n), _f32(gB, "gradB", 9 * n),
                                        _f32(dvdx, "dvdx", 9 * n), dv.data_ptr(), du.data_ptr(), cons.data_ptr(),
                                        c.data_ptr() if c is not None else None))
    return dv, du, cons, c


def hydro_accel(ctx: Context, lv: Leaves, hp: HydroParams, m, v3, u, V, rho, A, B, gA, gB, dvdx=None,
                sig_beta: float = 3.0, vsig_h=None, count=False):
    """Acceleration pass: dv/dt and the signal-velocity max (vsig_h: int32[1] holding FP32 bits of
    max_i vsig_i / h_i, raised in place; a zeroed one is made when None)."""
    n = lv.n
    dv = ctx.empty(3, n)
    if vsig_h is None:
        vsig_h = torch.zeros(1, dtype=torch.int32, device=ctx.device)
    cons = torch.zeros(4, dtype=torch.float64, device=ctx.device)
    c = _count(ctx, count)
    hpc = hp.c()
    ctx.check(N.lib().crk_hydro_accel(ctx.handle, lv.handle, ctypes.byref(hpc), _f32(m, "m", n),
                                      _f32(v3, "v3", 3 * n), _f32(u, "u", n), _f32(V, "V", n), _f32(rho, "rho", n),
                                      _f32(A, "A", n), _f32(B, "B", 3 * n), _f32(gA, "gradA", 3 * n),
                                      _f32(gB, "gradB", 9 * n), _f32(dvdx, "dvdx", 9 * n) if dvdx is not None else None,
                                      float(sig_beta), dv.data_ptr(), vsig_h.data_ptr(), cons.data_ptr(),
                                      c.data_ptr() if c is not None else None))
    return dv, vsig_h, cons, c


def hydro_energy(ctx: Context, lv: Leaves, hp: HydroParams, m, v3, u, V, rho, A, B, gA, gB, vstar3, dvdx=None,
                 count=False):
    """Energy pass with the compatible split of the pair work on the time-centred velocities vstar3."""
    n = lv.n
    du = ctx.empty(n)
    cons = torch.zeros(4, dtype=torch.float64, device=ctx.device)
    c = _count(ctx, count)
    hpc = hp.c()
    ctx.check(N.lib().crk_hydro_energy(ctx.handle, lv.handle, ctypes.byref(hpc), _f32(m, "m", n),
                                       _f32(v3, "v3", 3 * n), _f32(u, "u", n), _f32(V, "V", n), _f32(rho, "rho", n),
                                       _f32(A, "A", n), _f32(B, "B", 3 * n), _f32(gA, "gradA", 3 * n),
                                       _f32(gB, "gradB", 9 * n),
                                       _f32(dvdx, "dvdx", 9 * n) if dvdx is not None else None,
                                       _f32(vstar3, "vstar3", 3 * n), du.data_ptr(), cons.data_ptr(),
                                       c.data_ptr() if c is not None else None))
    return du, cons, c


def timestep(ctx: Context, vsig_h, cfl: float, dt_max: float):
    """Courant step dt = min(dt_max, cfl / max_i vsig_i/h_i) as a device float[1]."""
    dt = ctx.empty(1)
    if vsig_h.dtype != torch.int32 or not vsig_h.is_cuda:
        raise TypeError("vsig_h must be the CUDA int32 tensor of hydro_accel")
    ctx.check(N.lib().crk_timestep(ctx.handle, vsig_h.data_ptr(), float(cfl), float(dt_max), dt.data_ptr()))
    return dt


@dataclass
class AdvanceParams:
    cfl: float = 0.25
    dt_max: float = 1.0
    dt_fixed: float = 0.0
    sig_beta: float = 3.0
    limited: bool = False
    gravity: bool = False

    def c(self) -> N.crk_advance_params:
        return N.crk_advance_params(self.cfl, self.dt_max, self.dt_fixed, self.sig_beta, int(self.limited),
                                    int(self.gravity))


def advance(ctx: Context, db: "DeviceBox", ap: AdvanceParams, conservation=None, n_singular=None):
    """One two-stage kick-drift step of db in place (x, y, z, v3, u); returns dt as a device float[1]."""
    n = db.n
    dt = ctx.empty(1)
    if conservation is not None and (conservation.dtype != torch.float64 or conservation.numel() < 4):
        raise TypeError("conservation must be a CUDA float64 tensor of 4")
    if n_singular is not None and n_singular.dtype != torch.int32:
        raise TypeError("n_singular must be a CUDA int32 tensor")
    lpc = N.crk_leaf_params(int(db.lp.mode), int(db.lp.cells_per_side), int(db.lp.max_leaf), float(db.lp.r_cut_grav))
    hpc, gpc, apc = db.hp.c(), db.gp.c(), ap.c()
    if n and (db.species.dtype != torch.uint8 or not db.species.is_cuda or db.species.numel() != n):
        raise TypeError("species must be a CUDA uint8 tensor of length n")
    arrs = [(db.x, "x", n), (db.y, "y", n), (db.z, "z", n)]
    ptrs = [_f32(t, nm, k) if n else None for t, nm, k in arrs]
    ctx.check(N.lib().crk_advance(ctx.handle, n, float(db.L), *ptrs, db.species.data_ptr() if n else None,
                                  _f32(db.h, "h", n) if n else None, _f32(db.m, "m", n) if n else None,
                                  _f32(db.v3, "v3", 3 * n) if n else None, _f32(db.u, "u", n) if n else None,
                                  ctypes.byref(lpc), ctypes.byref(hpc), ctypes.byref(gpc), ctypes.byref(apc),
                                  dt.data_ptr(), conservation.data_ptr() if conservation is not None else None,
                                  n_singular.data_ptr() if n_singular is not None else None))
    return dt


def corrections_adjoint(ctx: Context, lv: Leaves, V, Abar, Bbar, gAbar, gBbar):
    """Gradient of sum Abar A + Bbar.B + gAbar.gradA + gBbar:gradB in the positions (3, n) and
    volumes (n); also the singular count (device int32)."""
    n = lv.n
    gx, gV = ctx.empty(3, n), ctx.empty(n)
    ns = torch.zeros(1, dtype=torch.int32, device=ctx.device)
    ctx.check(N.lib().crk_corrections_adjoint(ctx.handle, lv.handle, _f32(V, "V", n), _f32(Abar, "Abar", n),
                                              _f32(Bbar, "Bbar", 3 * n), _f32(gAbar, "gradAbar", 3 * n),
                                              _f32(gBbar, "gradBbar", 9 * n), gx.data_ptr(), gV.data_ptr(),
                                              ns.data_ptr()))
    return gx, gV, ns


def hydro_adjoint(ctx: Context, lv: Leaves, hp: HydroParams, m, v3, u, V, rho, A, B, gA, gB, dvbar, dubar):
    """Reverse mode of hydro for the cotangents dvbar (3, n), dubar (n): a dict of the gradients in
    x, v (3, n), u, m, V, rho, A (n), B, gA (3, n) and gB (9, n), every input held independent."""
    n = lv.n
    out = dict(x=ctx.empty(3, n), v=ctx.empty(3, n), u=ctx.empty(n), m=ctx.empty(n), V=ctx.empty(n),
               rho=ctx.empty(n), A=ctx.empty(n), B=ctx.empty(3, n), gA=ctx.empty(3, n), gB=ctx.empty(9, n))
    hpc = hp.c()
    ctx.check(N.lib().crk_hydro_adjoint(ctx.handle, lv.handle, ctypes.byref(hpc), _f32(m, "m", n),
                                        _f32(v3, "v3", 3 * n), _f32(u, "u", n), _f32(V, "V", n), _f32(rho, "rho", n),
                                        _f32(A, "A", n), _f32(B, "B", 3 * n), _f32(gA, "gradA", 3 * n),
                                        _f32(gB, "gradB", 9 * n), _f32(dvbar, "dvbar", 3 * n),
                                        _f32(dubar, "dubar", n),
                                        *[out[k].data_ptr() for k in ("x", "v", "u", "m", "V", "rho", "A", "B", "gA",
                                                                      "gB")]))
    return out


def hydro_chain_adjoint(ctx: Context, lv: Leaves, db: "DeviceBox", dvbar, dubar, forward: bool = True):
    """Forward and reverse pass of geometry -> corrections -> hydro in the library's kernel order:
    the gradients of sum dvbar.dv + dubar.du in x (3, n), m, v (3, n) and u, plus dv, du when
    `forward`; also the singular count."""
    n = lv.n
    out = dict(x=ctx.empty(3, n), m=ctx.empty(n), v=ctx.empty(3, n), u=ctx.empty(n),
               n_singular=torch.zeros(1, dtype=torch.int32, device=ctx.device))
    if forward:
        out["dv"], out["du"] = ctx.empty(3, n), ctx.empty(n)
    io = N.crk_chain_adjoint_io(_f32(db.m, "m", n), _f32(db.v3, "v3", 3 * n), _f32(db.u, "u", n),
                                _f32(dvbar, "dvbar", 3 * n), _f32(dubar, "dubar", n),
                                out["dv"].data_ptr() if forward else None,
                                out["du"].data_ptr() if forward else None, out["x"].data_ptr(), out["m"].data_ptr(),
                                out["v"].data_ptr(), out["u"].data_ptr(), out["n_singular"].data_ptr())
    hpc = db.hp.c()
    ctx.check(N.lib().crk_hydro_chain_adjoint(ctx.handle, lv.handle, ctypes.byref(hpc), ctypes.byref(io)))
    return out


def grav_short(ctx: Context, lv: Leaves, gp: GravParams, m, count=False):
    n = lv.n
    a = ctx.empty(3, n)
    c = _count(ctx, count)
    g = gp.c()
    ctx.check(N.lib().grav_short(ctx.handle, lv.handle, ctypes.byref(g), _f32(m, "m", n), a.data_ptr(),
                                 c.data_ptr() if c is not None else None))
    return a, c


def grav_short_adjoint(ctx: Context, lv: Leaves, gp: GravParams, m, abar3):
    n = lv.n
    gx, gm = ctx.empty(3, n), ctx.empty(n)
    g = gp.c()
    ctx.check(N.lib().grav_short_adjoint(ctx.handle, lv.handle, ctypes.byref(g), _f32(m, "m", n),
                                         _f32(abar3, "abar3", 3 * n), gx.data_ptr(), gm.data_ptr()))
    return gx, gm


def geometry_adjoint(ctx: Context, lv: Leaves, m, V, rhobar, Vbar=None):
    n = lv.n
    gx, gm = ctx.empty(3, n), ctx.empty(n)
    ctx.check(N.lib().crk_geometry_adjoint(ctx.handle, lv.handle, _f32(m, "m", n), _f32(V, "V", n),
                                           _f32(rhobar, "rhobar", n),
                                           _f32(Vbar, "Vbar", n) if Vbar is not None else None,
                                           gx.data_ptr(), gm.data_ptr()))
    return gx, gm


# ----------------------------------------------------------------- box helpers

class DeviceBox:
    """A workload box uploaded to the device (original order, SoA)."""

    def __init__(self, box, device="cuda"):
        t = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        self.L = float(box.L)
        self.n = box.n
        self.x, self.y, self.z = t(box.x), t(box.y), t(box.z)
        self.species = t(box.species, torch.uint8)
        self.m, self.h, self.u = t(box.m), t(box.h), t(box.u)
        self.v3 = t(np.stack([box.vx, box.vy, box.vz]))
        self.lp = LeafParams(box.leaf_mode, box.cells_per_side, box.max_leaf, float(box.r_cut))
        self.gp = GravParams(float(box.eps), float(box.r_cut), tuple(float(c) for c in box.poly))
        self.hp = HydroParams()


class DeviceBatch:
    """Several independent boxes uploaded as one concatenated particle set (box b = one range)."""

    def __init__(self, boxes, device="cuda"):
        cat = lambda f, dt=np.float32: torch.as_tensor(np.ascontiguousarray(np.concatenate([f(b) for b in boxes]))
                                                       ).to(device=device, dtype=torch.float32 if dt is np.float32
                                                            else dt)
        self.boxes = boxes
        self.n = int(sum(b.n for b in boxes))
        self.box_start = np.concatenate([[0], np.cumsum([b.n for b in boxes])]).astype(np.int64)
        self.box_side = np.array([b.L for b in boxes], np.float32)
        self.x, self.y, self.z = cat(lambda b: b.x), cat(lambda b: b.y), cat(lambda b: b.z)
        self.species = torch.as_tensor(np.concatenate([b.species for b in boxes])).to(device=device,
                                                                                       dtype=torch.uint8)
        self.m, self.h, self.u = cat(lambda b: b.m), cat(lambda b: b.h), cat(lambda b: b.u)
        self.v3 = torch.stack([cat(lambda b: b.vx), cat(lambda b: b.vy), cat(lambda b: b.vz)]).contiguous()
        b0 = boxes[0]
        self.lp = LeafParams(1, 0, b0.max_leaf, float(b0.r_cut))
        self.gp = GravParams(float(b0.eps), float(b0.r_cut), tuple(float(c) for c in b0.poly))
        self.hp = HydroParams()


def _batch_c(dbt):
    """crk_batch of a DeviceBatch (or a DeviceBox as a batch of one); the host arrays it points to
    are returned with it and must stay alive while it is used."""
    n = dbt.n
    if hasattr(dbt, "box_start"):
        bs = np.ascontiguousarray(dbt.box_start, np.int64)
        side = np.ascontiguousarray(dbt.box_side, np.float32)
    else:
        bs = np.array([0, n], np.int64)
        side = np.array([dbt.L], np.float32)
    c = N.crk_batch(_f32(dbt.x, "x", n), _f32(dbt.y, "y", n), _f32(dbt.z, "z", n), dbt.species.data_ptr(), n,
                    len(side), bs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                    side.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return c, (bs, side)


def rebuild_leaves(ctx: Context, lv: Leaves, dbt) -> None:
    """crk_leaves_rebuild_batch: lv recomputed in place for the current positions and h of dbt (a
    DeviceBatch or DeviceBox with the particles lv was built from); no synchronisation (see
    Leaves.status)."""
    c, keep = _batch_c(dbt)
    ctx.check(N.lib().crk_leaves_rebuild_batch(ctx.handle, lv.handle, ctypes.byref(c), _f32(dbt.h, "h", dbt.n)))


def build_leaves_batch(ctx: Context, dbt: DeviceBatch) -> Leaves:
    n = dbt.n
    c, keep = _batch_c(dbt)
    lp = N.crk_leaf_params(int(dbt.lp.mode), 0, int(dbt.lp.max_leaf), float(dbt.lp.r_cut_grav))
    out = ctypes.c_void_p()
    ctx.check(N.lib().crk_build_leaves_batch(ctx.handle, ctypes.byref(c), _f32(dbt.h, "h", n), ctypes.byref(lp),
                                             ctypes.byref(out)))
    return Leaves(ctx, out, (dbt.x, dbt.y, dbt.z, dbt.species, dbt.h))


def forward(ctx: Context, db: DeviceBox, count=False):
    """Leaves, then geometry -> corrections -> hydro, then gravity; returns a dict of device tensors."""
    lv = build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    V, rho, cg = geometry(ctx, lv, db.m, count)
    A, B, gA, gB, ns = corrections(ctx, lv, V)
    dv, du, cons, ch = hydro(ctx, lv, db.hp, db.m, db.v3, db.u, V, rho, A, B, gA, gB, count)
    a, ca = grav_short(ctx, lv, db.gp, db.m, count)
    return dict(leaves=lv, V=V, rho=rho, A=A, B=B, gA=gA, gB=gB, n_singular=ns, dv=dv, du=du, cons=cons, acc=a,
                count_geom=cg, count_hydro=ch, count_grav=ca)


# ------------------------------------------------------------------- whole step

class StepIO:
    """Device arrays of one whole step (crk_step): inputs from a DeviceBox, outputs allocated here.

    outputs=False allocates only what a step must return to a caller that wants the
    accelerations, energy rates and gradients (dv, du, a, both adjoints); the
    intermediates (V, rho, A, B, dA, dB) then stay inside the library.
    """

    def __init__(self, ctx: Context, db, outputs: bool = True, extras: bool = False):
        n = db.n
        e = ctx.empty
        self.db = db
        self.full = outputs
        self.extras = extras
        self.rho_r, self.dvdx = (e(n), e(9, n)) if (extras and outputs) else (None, None)
        if outputs:
            self.V, self.rho, self.A, self.B, self.gA, self.gB = e(n), e(n), e(n), e(3, n), e(3, n), e(9, n)
        else:
            self.V = self.rho = self.A = self.B = self.gA = self.gB = None
        self.dv, self.du = e(3, n), e(n)
        self.cons = torch.zeros(4, dtype=torch.float64, device=ctx.device)
        self.acc = e(3, n)
        self.gx_grav, self.gm_grav, self.gx_geom, self.gm_geom = e(3, n), e(n), e(3, n), e(n)
        self.n_singular = torch.zeros(1, dtype=torch.int32, device=ctx.device)
        self.pair_count = torch.zeros(3, dtype=torch.int64, device=ctx.device)
        self.swept_count = torch.zeros(3, dtype=torch.int64, device=ctx.device)

    def c(self, count: bool = False) -> N.crk_step_io:
        d, P = self.db, lambda t: t.data_ptr() if t is not None else None
        return N.crk_step_io(P(d.m), P(d.v3), P(d.u), P(self.V), P(self.rho), P(self.A), P(self.B), P(self.gA),
                             P(self.gB), P(self.dv), P(self.du), P(self.cons), P(self.acc), None, P(self.gx_grav),
                             P(self.gm_grav), None, None, P(self.gx_geom), P(self.gm_geom), P(self.n_singular),
                             P(self.pair_count) if count else None, 1 if self.extras else 0, P(self.rho_r),
                             P(self.dvdx), P(self.swept_count) if count else None)


def step(ctx: Context, lv: Leaves, db: "DeviceBox", io: StepIO, count: bool = False) -> None:
    """geometry -> corrections -> hydro -> gravity -> gravity adjoint -> geometry adjoint (one C call)."""
    gp, hp, c = db.gp.c(), db.hp.c(), io.c(count)
    ctx.check(N.lib().crk_step(ctx.handle, lv.handle, ctypes.byref(gp), ctypes.byref(hp), ctypes.byref(c)))


class StepGraph:
    """A captured CUDA graph of one crk_step on fixed leaves and arrays."""

    def __init__(self, ctx: Context, lv: Leaves, db: "DeviceBox", io: StepIO):
        self.ctx, self.keep = ctx, (lv, db, io)
        gp, hp, c = db.gp.c(), db.hp.c(), io.c(False)
        h = ctypes.c_void_p()
        ctx.check(N.lib().crk_step_graph_create(ctx.handle, lv.handle, ctypes.byref(gp), ctypes.byref(hp),
                                                ctypes.byref(c), ctypes.byref(h)))
        self.handle = h

    def launch(self) -> None:
        self.ctx.check(N.lib().crk_graph_launch(self.handle))

    def close(self) -> None:
        if getattr(self, "handle", None):
            N.lib().crk_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RebuildStepGraph(StepGraph):
    """The batched driver as one CUDA graph: leaf rebuild (crk_leaves_rebuild_batch) and crk_step."""

    def __init__(self, ctx: Context, lv: Leaves, dbt, io: StepIO):
        self.ctx, self.keep = ctx, (lv, dbt, io)
        c, self._host = _batch_c(dbt)
        self._c = c
        gp, hp, ci = dbt.gp.c(), dbt.hp.c(), io.c(False)
        h = ctypes.c_void_p()
        ctx.check(N.lib().crk_rebuild_step_graph_create(ctx.handle, lv.handle, ctypes.byref(c),
                                                        _f32(dbt.h, "h", dbt.n), ctypes.byref(gp),
                                                        ctypes.byref(hp), ctypes.byref(ci), ctypes.byref(h)))
        self.handle = h


def tune(ctx: Context, lv: Leaves, db: "DeviceBox", io: StepIO, reps: int = 3) -> dict:
    """Autotune every pair kernel on these leaves (crk_tune): the sweep variant, then the launch
    mode, then (gravity tiles) the j-tile depth and the warps per leaf.  Returns {kernel:
    {"variant", "persistent", "depth", "warps", "ms": {"variant": [ms per variant], "launch":
    [off, on], "depth": [32, 64, 96], "warps": [4, 2]}}} (-1 = not timed; extras only when io
    has the Extras outputs)."""
    gp, hp, c = db.gp.c(), db.hp.c(), io.c(False)
    ms = (ctypes.c_float * (N.N_KERNELS * N.TUNE_COLS))()
    best = (ctypes.c_int * (4 * N.N_KERNELS))()
    ctx.check(N.lib().crk_tune(ctx.handle, lv.handle, ctypes.byref(gp), ctypes.byref(hp), ctypes.byref(c),
                               int(reps), ms, best))
    out = {}
    for k, i in N.KERNELS.items():
        row = [round(float(ms[N.TUNE_COLS * i + q]), 4) for q in range(N.TUNE_COLS)]
        out[k] = {"variant": int(best[4 * i]), "persistent": bool(best[4 * i + 1]), "depth": int(best[4 * i + 2]),
                  "warps": int(best[4 * i + 3]),
                  "ms": {"variant": row[:N.N_VARIANTS], "launch": row[N.N_VARIANTS:N.N_VARIANTS + 2],
                         "depth": row[N.N_VARIANTS + 2:N.N_VARIANTS + 5], "warps": row[N.N_VARIANTS + 5:]}}
    return out


def autotune(ctx: Context, lv: Leaves, db, io: StepIO, cache_path: str | None = None, reps: int = 3) -> dict:
    """Pick every kernel's variant with crk_tune, remembering choices in a JSON cache.

    The cache key is the GPU name and the shape of the leaf structure (particles, leaves,
    image entries); a hit applies the stored variants without timing anything.
    """
    import json
    import os

    key = (f"{torch.cuda.get_device_name(ctx.device)}|n={lv.n}|leaves={lv.n_leaves}|"
           f"gimg={lv.n_grav_images}|himg={lv.n_hydro_images}")
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if key in cache and "launch" in cache[key] and all(len(v) == 3 for v in cache[key]["launch"].values()):
        for k, v in cache[key]["variants"].items():
            ctx.set_variant(k, int(v))
        for k, (pm, d, w) in cache[key]["launch"].items():
            ctx.set_launch(k, bool(pm), int(d), int(w))
        return dict(cache[key], cached=True)
    res = tune(ctx, lv, db, io, reps)
    entry = {"variants": {k: r["variant"] for k, r in res.items()},
             "launch": {k: [int(r["persistent"]), r["depth"], r["warps"]] for k, r in res.items()},
             "ms": {k: r["ms"] for k, r in res.items()}}
    if cache_path:
        cache[key] = entry
        tmp = cache_path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(entry, cached=False)
