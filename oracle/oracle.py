"""Python front end of the FP64 CPU oracle (oracle/crk_oracle.c).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's CPU
baseline import this module; the product library never does.  It shares no
code with the CUDA path: it compiles and loads its own C file with gcc and
passes FP64 numpy arrays through ctypes.

Every function takes plain arrays (positions as f64[n, 3], vectors as
f64[n, 3], tensors as f64[n, 9]) so that finite-difference checks can perturb
positions in FP64.  ``from_box`` promotes a workload's FP32 arrays exactly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "crk_oracle.c")
LIB = os.path.join(HERE, "liborc.so")

_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_u8 = ctypes.POINTER(ctypes.c_uint8)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


def compile_c(src: str, out: str) -> str:
    """gcc a copy of the oracle's C file into a shared library (FP64, OpenMP, no FP contraction)."""
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP, no FP contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        compile_c(SRC, LIB)
    return LIB


def bind(L):
    """Declare the argument and result types of the oracle's exported functions on a loaded CDLL."""
    L.orc_num_threads.restype = ctypes.c_int
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_wendland.argtypes = [ctypes.c_int64, _d, _d, _d, _d]
    L.orc_grav_g.argtypes = [ctypes.c_int64, _d, ctypes.c_double, _d, _d, _d]
    L.orc_gravity.argtypes = [ctypes.c_int64, _d, _d, ctypes.c_double, ctypes.c_double, ctypes.c_double, _d,
                              _i64, ctypes.c_int64, ctypes.c_int, _d, _i64]
    L.orc_gravity_adjoint.argtypes = [ctypes.c_int64, _d, _d, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, _d, _d, _i64, ctypes.c_int64, ctypes.c_int, _d, _d,
                                      _i64]
    L.orc_geometry.argtypes = [ctypes.c_int64, _d, _u8, _d, _d, ctypes.c_double, _i64, ctypes.c_int64,
                               ctypes.c_int, _d, _d, _i64]
    L.orc_corrections.argtypes = [ctypes.c_int64, _d, _u8, _d, _d, ctypes.c_double, _i64, ctypes.c_int64,
                                  ctypes.c_int, _d, _d, _d, _d, _i64, _i64]
    L.orc_hydro.argtypes = [ctypes.c_int64, _d, _u8, _d, _d, _d, _d, _d, _d, _d, _d, _d, _d, _d,
                            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, _i64, ctypes.c_int64, ctypes.c_int, _d, _d, _i64]
    L.orc_hydro_compatible.argtypes = [ctypes.c_int64, _d, _u8, _d, _d, _d, _d, _d, _d, _d, _d, _d, _d,
                                       _d, _d, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, _i64,
                                       ctypes.c_int64, ctypes.c_int, _d, _d, _d, _i64]
    L.orc_wendland2.argtypes = [ctypes.c_int64, _d, _d, _d, _d, _d]
    L.orc_corrections_adjoint.argtypes = [ctypes.c_int64, _d, _u8, _d, _d, ctypes.c_double, _d, _d, _d,
                                          _d, _d, _d, _i64]
    L.orc_hydro_adjoint.argtypes = [ctypes.c_int64, _d, _u8, _d, _d, _d, _d, _d, _d, _d, _d, _d, _d,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, _d, _d] + [_d] * 10
    L.orc_energy_share.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.orc_energy_share.restype = ctypes.c_double
    L.orc_extras.argtypes = [ctypes.c_int64, _d, _u8, _d, _d, _d, _d, _d, _d, _d, _d, ctypes.c_double,
                             _i64, ctypes.c_int64, ctypes.c_int, _d, _d, _i64]
    L.orc_geometry_adjoint.argtypes = [ctypes.c_int64, _d, _u8, _d, _d, _d, _d, ctypes.c_double, _i64,
                                       ctypes.c_int64, ctypes.c_int, _d, _d]
    L.orc_leaves_mesh.argtypes = [ctypes.c_int64, _d, _u8, ctypes.c_double, ctypes.c_int, _i32, _i32]
    L.orc_leaves_rcb.argtypes = [ctypes.c_int64, _d, _u8, ctypes.c_int, _i32, _i32, ctypes.c_int64, _i64]
    L.orc_leaf_pairs.argtypes = [ctypes.c_int64, _i32, _i32, _d, _u8, _d, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_double, _i32, ctypes.c_int64, _i32, _i32, ctypes.c_int64, _i64]
    L.orc_mark_neighbours.argtypes = [ctypes.c_int64, _d, _u8, _d, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, _u8, _u8]
    for name in ("orc_mark_neighbours", "orc_gravity", "orc_gravity_adjoint", "orc_geometry", "orc_corrections",
                 "orc_hydro", "orc_extras",
                 "orc_geometry_adjoint", "orc_leaves_mesh", "orc_leaves_rcb", "orc_leaf_pairs"):
        getattr(L, name).restype = ctypes.c_int
    return L


def load(path: str):
    """Load and bind an oracle library built from a (possibly modified) copy of crk_oracle.c."""
    return bind(ctypes.CDLL(path))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load(LIB)
    return _lib


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


class Inputs:
    """FP64 copy of one box: the oracle's view of the workload."""

    def __init__(self, pos, species, m, h, u, v, L, r_cut, eps, poly):
        self.pos = _f64(pos).reshape(-1, 3)
        self.species = np.ascontiguousarray(species, dtype=np.uint8)
        self.m = _f64(m)
        self.h = _f64(h)
        self.u = _f64(u)
        self.v = _f64(v).reshape(-1, 3)
        self.L = float(L)
        self.r_cut = float(r_cut)
        self.eps = float(eps)
        self.poly = _f64(poly)
        self.n = self.pos.shape[0]

    def with_pos(self, pos):
        c = Inputs(pos, self.species, self.m, self.h, self.u, self.v, self.L, self.r_cut, self.eps, self.poly)
        return c

    def with_m(self, m):
        return Inputs(self.pos, self.species, m, self.h, self.u, self.v, self.L, self.r_cut, self.eps, self.poly)


def from_box(box) -> Inputs:
    pos = np.stack([box.x, box.y, box.z], axis=1).astype(np.float64)
    v = np.stack([box.vx, box.vy, box.vz], axis=1).astype(np.float64)
    return Inputs(pos, box.species, box.m, box.h, box.u, v, box.L, box.r_cut, box.eps,
                  np.asarray(box.poly, dtype=np.float32).astype(np.float64))


def _sub(sub):
    if sub is None:
        return None, 0
    s = np.ascontiguousarray(sub, dtype=np.int64)
    return s, s.size


# ------------------------------------------------------------------ kernels

def wendland(r, h):
    r = _f64(r)
    h = _f64(np.broadcast_to(h, r.shape))
    W = np.empty_like(r)
    dWr = np.empty_like(r)
    lib().orc_wendland(r.size, _p(r, _d), _p(h, _d), _p(W, _d), _p(dWr, _d))
    return W, dWr


def grav_g(s, eps, poly):
    s = _f64(s)
    c = _f64(poly)
    g = np.empty_like(s)
    dg = np.empty_like(s)
    lib().orc_grav_g(s.size, _p(s, _d), float(eps), _p(c, _d), _p(g, _d), _p(dg, _d))
    return g, dg


def gravity(I: Inputs, sub=None, brute=False):
    """Short-range gravity accelerations f64[n, 3] and the ordered in-range pair count."""
    acc = np.zeros((I.n, 3))
    npairs = ctypes.c_int64(0)
    s, ns = _sub(sub)
    _check(lib().orc_gravity(I.n, _p(I.pos, _d), _p(I.m, _d), I.L, I.r_cut, I.eps, _p(I.poly, _d), _p(s, _i64), ns,
                             int(brute), _p(acc, _d), ctypes.byref(npairs)), "gravity")
    return acc, int(npairs.value)


def gravity_adjoint(I: Inputs, abar, sub=None, brute=False, with_pairs=False):
    abar = _f64(abar).reshape(-1, 3)
    gx = np.zeros((I.n, 3))
    gm = np.zeros(I.n)
    npairs = ctypes.c_int64(0)
    s, ns = _sub(sub)
    _check(lib().orc_gravity_adjoint(I.n, _p(I.pos, _d), _p(I.m, _d), I.L, I.r_cut, I.eps, _p(I.poly, _d),
                                     _p(abar, _d), _p(s, _i64), ns, int(brute), _p(gx, _d), _p(gm, _d),
                                     ctypes.byref(npairs)), "gravity_adjoint")
    if with_pairs:
        return gx, gm, int(npairs.value)
    return gx, gm


def geometry(I: Inputs, sub=None, brute=False):
    """Gas volumes V and densities rho (dark-matter entries 0) and the hydro pair count."""
    V = np.zeros(I.n)
    rho = np.zeros(I.n)
    npairs = ctypes.c_int64(0)
    s, ns = _sub(sub)
    _check(lib().orc_geometry(I.n, _p(I.pos, _d), _p(I.species, _u8), _p(I.h, _d), _p(I.m, _d), I.L, _p(s, _i64),
                              ns, int(brute), _p(V, _d), _p(rho, _d), ctypes.byref(npairs)), "geometry")
    return V, rho, int(npairs.value)


def corrections(I: Inputs, V, sub=None, brute=False, with_pairs=False):
    """A f64[n], B f64[n,3], gradA f64[n,3], gradB f64[n,9] (gradB[i, 3g+a] = d_g B^a) and #singular."""
    V = _f64(V)
    A = np.zeros(I.n)
    B = np.zeros((I.n, 3))
    gA = np.zeros((I.n, 3))
    gB = np.zeros((I.n, 9))
    ns_ = ctypes.c_int64(0)
    np_ = ctypes.c_int64(0)
    s, ns = _sub(sub)
    _check(lib().orc_corrections(I.n, _p(I.pos, _d), _p(I.species, _u8), _p(I.h, _d), _p(V, _d), I.L, _p(s, _i64),
                                 ns, int(brute), _p(A, _d), _p(B, _d), _p(gA, _d), _p(gB, _d), ctypes.byref(ns_),
                                 ctypes.byref(np_)),
           "corrections")
    if with_pairs:
        return A, B, gA, gB, int(ns_.value), int(np_.value)
    return A, B, gA, gB, int(ns_.value)


def hydro(I: Inputs, V, rho, A, B, gA, gB, gamma, alpha, beta, eta2, sub=None, brute=False, dvg=None):
    """dv/dt f64[n,3], du/dt f64[n] (gas only) and the hydro pair count.

    dvg (f64[n,9], dvg[i, 3a+b] = dv^a/dx^b, e.g. from extras) switches on the
    limited viscosity: velocities reconstructed to the pair midpoint."""
    args = [_f64(a) for a in (V, rho, A, B, gA, gB)]
    g = _f64(dvg).reshape(I.n, 9) if dvg is not None else None
    dv = np.zeros((I.n, 3))
    du = np.zeros(I.n)
    npairs = ctypes.c_int64(0)
    s, ns = _sub(sub)
    _check(lib().orc_hydro(I.n, _p(I.pos, _d), _p(I.species, _u8), _p(I.h, _d), _p(I.m, _d), _p(I.v, _d),
                           _p(I.u, _d), *[_p(a, _d) for a in args], _p(g, _d), I.L, float(gamma), float(alpha),
                           float(beta), float(eta2), _p(s, _i64), ns, int(brute), _p(dv, _d), _p(du, _d),
                           ctypes.byref(npairs)),
           "hydro")
    return dv, du, int(npairs.value)


def hydro_compatible(I: Inputs, V, rho, A, B, gA, gB, gamma, alpha, beta, eta2, vstar=None, sig_beta=3.0,
                     dvg=None, sub=None, brute=False):
    """The hydro pair force with the compatible energy split and the signal velocity.

    vstar (f64[n,3]): time-centred velocities the pair work is taken on; the
    work -f_ij.(v*_i - v*_j) is shared by the weights of energy_share (None:
    the equal split on v).  Returns dv/dt f64[n,3], du/dt f64[n] and vsig
    f64[n] = max_j (c_i + c_j - sig_beta min(0, v_ij.x_ij/r)) (gas only)."""
    args = [_f64(a) for a in (V, rho, A, B, gA, gB)]
    g = _f64(dvg).reshape(I.n, 9) if dvg is not None else None
    w = _f64(vstar).reshape(I.n, 3) if vstar is not None else None
    dv = np.zeros((I.n, 3))
    du = np.zeros(I.n)
    vsig = np.zeros(I.n)
    npairs = ctypes.c_int64(0)
    s, ns = _sub(sub)
    _check(lib().orc_hydro_compatible(I.n, _p(I.pos, _d), _p(I.species, _u8), _p(I.h, _d), _p(I.m, _d),
                                      _p(I.v, _d), _p(I.u, _d), *[_p(a, _d) for a in args], _p(g, _d), _p(w, _d),
                                      float(sig_beta), I.L, float(gamma), float(alpha), float(beta), float(eta2),
                                      _p(s, _i64), ns, int(brute), _p(dv, _d), _p(du, _d), _p(vsig, _d),
                                      ctypes.byref(npairs)),
           "hydro_compatible")
    return dv, du, vsig


def wendland2(r, h):
    """W, (dW/dr)/r and (d[(dW/dr)/r]/dr)/r of the Wendland C4 kernel (support 2h)."""
    r = _f64(np.atleast_1d(r))
    h = _f64(np.broadcast_to(h, r.shape))
    W, dWr, ddWr = np.zeros_like(r), np.zeros_like(r), np.zeros_like(r)
    lib().orc_wendland2(r.size, _p(r, _d), _p(h, _d), _p(W, _d), _p(dWr, _d), _p(ddWr, _d))
    return W, dWr, ddWr


def corrections_adjoint(I: Inputs, V, Abar, Bbar, gAbar, gBbar):
    """Gradient of sum Abar A + Bbar.B + gAbar.gA + gBbar:gB (the outputs of corrections, same
    layouts: B f64[n,3], gA f64[n,3], gB f64[n,9]) in the positions f64[n,3] and volumes f64[n];
    also the count of singular particles (they contribute nothing)."""
    a = [_f64(x) for x in (V, Abar, Bbar, gAbar, gBbar)]
    xbar = np.zeros((I.n, 3))
    Vbar = np.zeros(I.n)
    nsing = ctypes.c_int64(0)
    _check(lib().orc_corrections_adjoint(I.n, _p(I.pos, _d), _p(I.species, _u8), _p(I.h, _d), _p(a[0], _d), I.L,
                                         *[_p(x, _d) for x in a[1:]], _p(xbar, _d), _p(Vbar, _d),
                                         ctypes.byref(nsing)),
           "corrections_adjoint")
    return xbar, Vbar, int(nsing.value)


def hydro_adjoint(I: Inputs, V, rho, A, B, gA, gB, gamma, alpha, beta, eta2, dvbar, dubar):
    """Reverse mode of hydro (Monaghan viscosity, equal split) for the cotangents dvbar f64[n,3],
    dubar f64[n], with every input of the pair force independent.  Returns a dict of the
    gradients in x, v (f64[n,3]), u, m, V, rho (f64[n]), A (f64[n]), B, gA (f64[n,3]), gB (f64[n,9])."""
    a = [_f64(x) for x in (V, rho, A, B, gA, gB, dvbar, dubar)]
    out = dict(x=np.zeros((I.n, 3)), v=np.zeros((I.n, 3)), u=np.zeros(I.n), m=np.zeros(I.n), V=np.zeros(I.n),
               rho=np.zeros(I.n), A=np.zeros(I.n), B=np.zeros((I.n, 3)), gA=np.zeros((I.n, 3)),
               gB=np.zeros((I.n, 9)))
    _check(lib().orc_hydro_adjoint(I.n, _p(I.pos, _d), _p(I.species, _u8), _p(I.h, _d), _p(I.m, _d), _p(I.v, _d),
                                   _p(I.u, _d), *[_p(x, _d) for x in a[:6]], I.L, float(gamma), float(alpha),
                                   float(beta), float(eta2), _p(a[6], _d), _p(a[7], _d),
                                   *[_p(out[k], _d) for k in ("x", "v", "u", "m", "V", "rho", "A", "B", "gA", "gB")]),
           "hydro_adjoint")
    return out


def energy_share(ui, uj, dE):
    """The share w_ij of a pair's heat dE that particle i receives (compatible split)."""
    return float(lib().orc_energy_share(float(ui), float(uj), float(dE)))


def timestep(I: Inputs, vsig, cfl, dt_max):
    """Courant step: dt = min(dt_max, cfl min_i h_i / vsig_i) over gas particles."""
    gas = (I.species == 0) & (vsig > 0)
    if not np.any(gas):
        return float(dt_max)
    return float(min(dt_max, cfl * np.min(I.h[gas] / vsig[gas])))


def _wrap(x, L):
    y = x - L * np.floor(x / L)
    return np.where(y >= L, 0.0, y)


def _chain(I: Inputs, limited):
    """Geometry, corrections and (limited) Extras: the inputs of the hydro pair force."""
    V, rho, _ = geometry(I)
    A, B, gA, gB, _ = corrections(I, V)
    dvg = None
    if limited:
        rho, dvg = extras(I, V, A, B, gA, gB)
    return V, rho, A, B, gA, gB, dvg


def advance(I: Inputs, gamma, alpha, beta, eta2, cfl, dt_max, sig_beta=3.0, limited=False, gravity_on=False,
            dt=None, fp32_state=False):
    """One two-stage kick-drift step with the compatible energy update.

    Stage 1 at t^n: geometry, corrections (Extras when limited), Acceleration
    and Energy (v* = v^n) and the Courant step dt (unless given).  Predictor:
    v_p = v + dt/2 a, u_p = u + dt/2 du, x_p = x + dt/2 v_p.  Stage 2 at the
    predicted state: the same chain, Acceleration a_p; kick v1 = v + dt a_p;
    Energy on v* = (v + v1)/2 with the predicted state's forces; u1 = u + dt du;
    drift x1 = x + dt v*.  Gas feels hydro (+ gravity), dark matter gravity
    only; h and m stay fixed.  Returns (Inputs at t^n+1, dt).

    fp32_state: round the states a single-precision code stores (the predicted
    v_p, u_p, x_p, then v1, v*, u1, x1) to FP32 where it stores them, so that a
    comparison with such a code sees its pair arithmetic, not its storage
    precision; the arithmetic between the stores stays FP64."""
    r32 = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if fp32_state else (lambda a: a)

    def wrap32(x):
        y = r32(_wrap(x, I.L))
        return np.where(y >= I.L, 0.0, y)
    hp = (gamma, alpha, beta, eta2)
    V, rho, A, B, gA, gB, dvg = _chain(I, limited)
    dv0, du0, vsig = hydro_compatible(I, V, rho, A, B, gA, gB, *hp, vstar=I.v, sig_beta=sig_beta, dvg=dvg)
    a0 = dv0 + (gravity(I)[0] if gravity_on else 0.0)
    if dt is None:
        dt = timestep(I, vsig, cfl, dt_max)
    vp = r32(I.v + 0.5 * dt * a0)
    up = r32(I.u + 0.5 * dt * du0)
    xp = wrap32(I.pos + 0.5 * dt * vp)
    Ip = Inputs(xp, I.species, I.m, I.h, up, vp, I.L, I.r_cut, I.eps, I.poly)
    V, rho, A, B, gA, gB, dvg = _chain(Ip, limited)
    dvp, _, _ = hydro_compatible(Ip, V, rho, A, B, gA, gB, *hp, sig_beta=sig_beta, dvg=dvg)
    ap = dvp + (gravity(Ip)[0] if gravity_on else 0.0)
    v1 = r32(I.v + dt * ap)
    vstar = r32(0.5 * (I.v + v1))
    _, du, _ = hydro_compatible(Ip, V, rho, A, B, gA, gB, *hp, vstar=vstar, sig_beta=sig_beta, dvg=dvg)
    u1 = r32(I.u + dt * du)
    x1 = wrap32(I.pos + dt * vstar)
    return Inputs(x1, I.species, I.m, I.h, u1, v1, I.L, I.r_cut, I.eps, I.poly), float(dt)


def extras(I: Inputs, V, A, B, gA, gB, sub=None, brute=False, with_pairs=False):
    """Corrected-kernel density rhoR f64[n] and velocity gradient f64[n,9] (dv[i, 3a+b] = dv^a/dx^b), gas only."""
    args = [_f64(a) for a in (V, A, B, gA, gB)]
    rhoR = np.zeros(I.n)
    dvg = np.zeros((I.n, 9))
    npairs = ctypes.c_int64(0)
    s, ns = _sub(sub)
    _check(lib().orc_extras(I.n, _p(I.pos, _d), _p(I.species, _u8), _p(I.h, _d), _p(I.m, _d), _p(I.v, _d),
                            *[_p(a, _d) for a in args], I.L, _p(s, _i64), ns, int(brute), _p(rhoR, _d), _p(dvg, _d),
                            ctypes.byref(npairs)),
           "extras")
    if with_pairs:
        return rhoR, dvg, int(npairs.value)
    return rhoR, dvg


def geometry_adjoint(I: Inputs, rhobar, Vbar=None, sub=None, brute=False):
    rb = _f64(rhobar)
    vb = _f64(Vbar) if Vbar is not None else None
    gx = np.zeros((I.n, 3))
    gm = np.zeros(I.n)
    s, ns = _sub(sub)
    _check(lib().orc_geometry_adjoint(I.n, _p(I.pos, _d), _p(I.species, _u8), _p(I.h, _d), _p(I.m, _d), _p(rb, _d),
                                      _p(vb, _d), I.L, _p(s, _i64), ns, int(brute), _p(gx, _d), _p(gm, _d)),
           "geometry_adjoint")
    return gx, gm


def conservation(I: Inputs, dv, du):
    """FP64 global sums: total momentum rate (3) and total energy rate."""
    gas = I.species == 0
    mom = (I.m[gas, None] * dv[gas]).sum(axis=0)
    ene = float((I.m[gas] * (np.sum(I.v[gas] * dv[gas], axis=1) + du[gas])).sum())
    return np.array([mom[0], mom[1], mom[2], ene])


def forward(I: Inputs, gamma, alpha, beta, eta2, brute=False):
    """The whole forward chain geometry -> corrections -> hydro, plus gravity."""
    V, rho, nh = geometry(I, brute=brute)
    A, B, gA, gB, nsing = corrections(I, V, brute=brute)
    dv, du, _ = hydro(I, V, rho, A, B, gA, gB, gamma, alpha, beta, eta2, brute=brute)
    acc, ng = gravity(I, brute=brute)
    return dict(V=V, rho=rho, A=A, B=B, gA=gA, gB=gB, dv=dv, du=du, acc=acc, pairs_hydro=nh, pairs_grav=ng,
                singular=nsing)


def neighbour_closure(I: Inputs, sub, hydro: bool):
    """Indices of sub together with every particle in range of one of them."""
    mi = np.zeros(I.n, np.uint8)
    mi[np.asarray(sub, np.int64)] = 1
    mo = np.zeros(I.n, np.uint8)
    _check(lib().orc_mark_neighbours(I.n, _p(I.pos, _d), _p(I.species, _u8), _p(I.h, _d), I.L, I.r_cut,
                                     int(hydro), _p(mi, _u8), _p(mo, _u8)), "mark_neighbours")
    return np.nonzero(mo)[0]


def sampled_chain(I: Inputs, sample, gamma, alpha, beta, eta2):
    """The forward chain plus the gravity adjoint for a sample of i-particles, every upstream
    value computed by the oracle itself: geometry on the two-hop gas closure, corrections on
    the one-hop closure, hydro and gravity on the sample.  Returns outputs and pair counts."""
    gas = I.species == 0
    s0 = np.asarray(sample, np.int64)
    s1 = neighbour_closure(I, s0[gas[s0]], True) if np.any(gas[s0]) else s0[:0]
    s2 = neighbour_closure(I, s1, True) if s1.size else s1
    g1 = neighbour_closure(I, s0, False)
    V, rho, n_geo = geometry(I, sub=s2)
    A, B, gA, gB, _, n_corr = corrections(I, V, sub=s1, with_pairs=True)
    dv, du, n_hyd = hydro(I, V, rho, A, B, gA, gB, gamma, alpha, beta, eta2, sub=s0)
    acc, n_grav = gravity(I, sub=g1)
    gx, gm, n_adj = gravity_adjoint(I, 2.0 * acc, sub=s0, with_pairs=True)
    pairs = n_geo + n_corr + n_hyd + n_grav + n_adj
    return dict(V=V, rho=rho, A=A, B=B, gA=gA, gB=gB, dv=dv, du=du, acc=acc, gx=gx, gm=gm, s1=s1, s2=s2,
                g1=g1, pairs=pairs, n_grav=n_grav, n_hydro=n_hyd)


# ------------------------------------------------------------------- leaves

def leaves_mesh(I: Inputs, nc: int):
    perm = np.zeros(I.n, np.int32)
    start = np.zeros(nc ** 3 + 1, np.int32)
    _check(lib().orc_leaves_mesh(I.n, _p(I.pos, _d), _p(I.species, _u8), I.L, int(nc), _p(perm, _i32),
                                 _p(start, _i32)), "leaves_mesh")
    return perm, start


def leaves_rcb(I: Inputs, max_leaf: int):
    perm = np.zeros(max(I.n, 1), np.int32)
    cap = max(1, 2 * (I.n // max(1, max_leaf // 2) + 2))
    start = np.zeros(cap + 1, np.int32)
    nl = ctypes.c_int64(0)
    _check(lib().orc_leaves_rcb(I.n, _p(I.pos, _d), _p(I.species, _u8), int(max_leaf), _p(perm, _i32),
                                _p(start, _i32), cap, ctypes.byref(nl)), "leaves_rcb")
    return perm[:I.n], start[:nl.value + 1]


def leaf_pairs(I: Inputs, perm, leaf_start, hydro: bool, asub=None):
    """Canonical leaf-pair CSR (ptr, list) over all leaves or the subset asub."""
    perm = np.ascontiguousarray(perm, np.int32)
    start = np.ascontiguousarray(leaf_start, np.int32)
    nl = start.size - 1
    a = np.ascontiguousarray(asub, np.int32) if asub is not None else None
    na = a.size if a is not None else nl
    ptr = np.zeros(na + 1, np.int32)
    cap = 64
    while True:
        lst = np.zeros(cap, np.int32)
        tot = ctypes.c_int64(0)
        rc = lib().orc_leaf_pairs(nl, _p(start, _i32), _p(perm, _i32), _p(I.pos, _d), _p(I.species, _u8),
                                  _p(I.h, _d), I.L, int(hydro), I.r_cut, _p(a, _i32), na if a is not None else 0,
                                  _p(ptr, _i32), _p(lst, _i32), cap, ctypes.byref(tot))
        if rc == 0:
            return ptr, lst[:tot.value]
        if tot.value <= cap:
            _check(rc, "leaf_pairs")
        cap = int(tot.value)
