"""Seeded synthetic particle boxes shaped like the paper's adiabatic workloads.

This module only *generates inputs*.  It holds none of the arithmetic of the
pair kernels (no smoothing kernel, no corrections, no forces): both the CUDA
library and the CPU oracle receive exactly the arrays made here.

The paper's own initial conditions (a 2x512^3, 177 Mpc/h box started at z=200,
split over 8 ranks as 2x256^3 particles per device; Sec. 3.4 "Problem Size" and
"Physics") are not available, so seeded stand-ins with the same species mix
(equal dark-matter and gas counts, Sec. 3.1) are generated:

* two interleaved unit lattices (dark matter on integer points, gas offset by
  half a cell), displaced either by Gaussian noise (the tiny box) or by a
  Zel'dovich field with P(k) ~ k^-2 (the clustered boxes),
* dense Plummer spheres that replace randomly chosen lattice particles,
* adaptive gas smoothing lengths h = half the distance to the 58th nearest
  other gas particle (about 58 neighbours inside the support 2h),
* gas internal energy U(0.9, 1.1) and velocities N(0, 0.05^2).

The short-range gravity polynomial (order 5, the build constant of the paper's
appendix) is also an *input* here: the paper does not print HACC's
coefficients, so a least-squares fit of a Gaussian-split long-range force is
made once in FP64 and rounded to FP32 (see ``gravity_poly``).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAS = 0
DM = 1

# Runtime physics parameters shared by every configuration.
R_CUT = 3.0          # short-range gravity cutoff r_c
EPS = 0.1            # Plummer softening
GAMMA = 5.0 / 3.0    # ideal-gas adiabatic index
AV_ALPHA = 1.0
AV_BETA = 2.0
AV_ETA2 = 0.01
MASS_DM = 1.0
MASS_GAS = 0.2

SEEDS = {"tiny": 1001, "clustered": 1002, "adjoint": 1003, "batched": 1004, "large": 1005}


@dataclasses.dataclass
class Box:
    """One periodic box of particles, all arrays in the caller's original order."""

    L: float
    x: np.ndarray        # f32[n]   positions in [0, L)
    y: np.ndarray
    z: np.ndarray
    species: np.ndarray  # u8[n]    0 = gas, 1 = dark matter
    m: np.ndarray        # f32[n]
    h: np.ndarray        # f32[n]   smoothing length (0 for dark matter)
    u: np.ndarray        # f32[n]   specific internal energy (0 for dark matter)
    vx: np.ndarray       # f32[n]   velocity (0 for dark matter)
    vy: np.ndarray
    vz: np.ndarray
    leaf_mode: int = 1           # 0 = fixed chaining mesh, 1 = recursive coordinate bisection
    cells_per_side: int = 0      # chaining-mesh cells per side (mode 0)
    max_leaf: int = 128          # RCB leaf capacity (mode 1)
    r_cut: float = R_CUT
    eps: float = EPS
    poly: np.ndarray = None      # f32[6] polynomial coefficients c_0..c_5 in s = r^2
    seed: int = 0
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_gas(self) -> int:
        return int(np.count_nonzero(self.species == GAS))

    def pos64(self) -> np.ndarray:
        return np.stack([self.x, self.y, self.z], axis=1).astype(np.float64)

    def v3(self) -> np.ndarray:
        """Velocities packed component-major, f32[3, n]."""
        return np.stack([self.vx, self.vy, self.vz]).astype(np.float32)


# --------------------------------------------------------------------------
# gravity polynomial (an input of the short-range kernel)
# --------------------------------------------------------------------------

def long_range_force_over_r(r: np.ndarray, r_s: float) -> np.ndarray:
    """|F_LR(r)| / r for a unit point mass under a Gaussian force split of scale r_s.

    F_LR is the part of 1/r^2 that a mesh solver with a Gaussian filter
    exp(-k^2 r_s^2) carries: [erf(r/2r_s) - r/(sqrt(pi) r_s) exp(-r^2/4r_s^2)] / r^2.
    Near r = 0 a series is used (the limit is 1/(6 sqrt(pi) r_s^3)).
    """
    from scipy.special import erf

    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    small = r < 1e-3 * r_s
    rs = r[~small]
    x = rs / (2.0 * r_s)
    out[~small] = (erf(x) - rs / (math.sqrt(math.pi) * r_s) * np.exp(-x * x)) / rs**3
    xs = r[small] / (2.0 * r_s)
    # erf(x) - 2x/sqrt(pi) e^{-x^2} = (4/(3 sqrt(pi))) x^3 (1 - 3x^2/5 + ...)
    out[small] = (4.0 / (3.0 * math.sqrt(math.pi))) * (1.0 - 0.6 * xs * xs) / (8.0 * r_s**3)
    return out


def gravity_poly(r_cut: float = R_CUT, eps: float = EPS, order: int = 5) -> np.ndarray:
    """FP64 equality-constrained least-squares fit of F_LR(r)/r by a polynomial in s = r^2.

    The fit runs on 4001 points of [0, r_cut] with the Gaussian split scale
    r_s = r_cut / 4.  The one constraint P(r_cut^2) = (r_cut^2 + eps^2)^-3/2 makes
    the short-range term (s + eps^2)^-3/2 - P(s) vanish at the cutoff, so the
    pair force is continuous there.  The result is rounded to FP32 once.
    """
    r_s = r_cut / 4.0
    r = np.linspace(0.0, r_cut, 4001)
    s = r * r
    target = long_range_force_over_r(r, r_s)
    V = np.vander(s, order + 1, increasing=True)
    # scale columns for conditioning
    scale = np.array([r_cut ** (-2 * k) for k in range(order + 1)])
    Vs = V * scale
    c_row = (np.array([r_cut ** (2 * k) for k in range(order + 1)]) * scale)[None, :]
    c_val = (r_cut * r_cut + eps * eps) ** -1.5
    n = order + 1
    kkt = np.zeros((n + 1, n + 1))
    kkt[:n, :n] = Vs.T @ Vs
    kkt[:n, n] = c_row[0]
    kkt[n, :n] = c_row[0]
    rhs = np.concatenate([Vs.T @ target, [c_val]])
    sol = np.linalg.solve(kkt, rhs)
    coef = sol[:n] * scale
    return coef.astype(np.float32)


# --------------------------------------------------------------------------
# particle layouts
# --------------------------------------------------------------------------

def _wrap32(a: np.ndarray, L: float) -> np.ndarray:
    """Wrap FP64 coordinates into [0, L) and round to FP32 (L itself maps to 0)."""
    w = np.mod(a, L).astype(np.float32)
    w[w >= np.float32(L)] = np.float32(0.0)
    w[w < 0] = np.float32(0.0)
    return w


def _lattices(side: int, L: float):
    g = np.arange(side, dtype=np.float64) * (L / side)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    dm = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    gas = dm + 0.5 * (L / side)
    return dm, gas


def zeldovich_displacement(side: int, L: float, rms: float, rng: np.random.Generator) -> np.ndarray:
    """Displacement field psi = IFFT[i k / k^2 delta_k] on a side^3 grid, P(k) ~ k^-2.

    delta is seeded Gaussian white noise filtered by k^-1 in amplitude.  The
    field is scaled so that the rms of |psi| over grid points is ``rms``.
    Returns f64[side^3, 3] in the (i, j, k) ravel order of ``_lattices``.
    """
    noise = rng.standard_normal((side, side, side))
    nk = np.fft.rfftn(noise)
    kf = 2.0 * np.pi * np.fft.fftfreq(side, d=L / side)
    kr = 2.0 * np.pi * np.fft.rfftfreq(side, d=L / side)
    KX, KY, KZ = np.meshgrid(kf, kf, kr, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    k2[0, 0, 0] = 1.0
    dk = nk / np.sqrt(k2)
    dk[0, 0, 0] = 0.0
    psi = np.empty((side, side, side, 3))
    for a, K in enumerate((KX, KY, KZ)):
        psi[..., a] = np.fft.irfftn(1j * K / k2 * dk, s=(side, side, side), axes=(0, 1, 2))
    psi = psi.reshape(-1, 3)
    cur = math.sqrt(float(np.mean(np.sum(psi * psi, axis=1))))
    return psi * (rms / cur)


def plummer_offsets(count: int, a: float, rng: np.random.Generator) -> np.ndarray:
    """Isotropic Plummer-sphere radii r = a / sqrt(U^(-2/3) - 1), truncated at 10a."""
    r = np.empty(count)
    filled = 0
    while filled < count:
        u = rng.random(count - filled)
        u = np.clip(u, 1e-12, 1.0 - 1e-12)
        rr = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        rr = rr[rr <= 10.0 * a]
        r[filled:filled + rr.size] = rr
        filled += rr.size
    v = rng.standard_normal((count, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * r[:, None]


def adaptive_h(pos_gas: np.ndarray, L: float, n_nbr: int = 58) -> np.ndarray:
    """Half the periodic distance to the n_nbr-th nearest *other* gas particle (FP64 kd-tree)."""
    from scipy.spatial import cKDTree

    if pos_gas.shape[0] <= n_nbr:
        raise ValueError("too few gas particles for adaptive h")
    pts = np.ascontiguousarray(pos_gas, dtype=np.float64)
    pts = np.where(pts >= L, pts - L, pts)
    tree = cKDTree(pts, boxsize=L)
    out = np.empty(pts.shape[0])
    chunk = 1 << 20
    for s in range(0, pts.shape[0], chunk):
        d, _ = tree.query(pts[s:s + chunk], k=[n_nbr + 1], workers=-1)
        out[s:s + chunk] = d[:, 0]
    return (0.5 * out).astype(np.float32)


def _finish(L, pos, species, rng, h_gas, name, seed, leaf_mode, cells, max_leaf, shuffle=True) -> Box:
    n = pos.shape[0]
    if shuffle:
        order = rng.permutation(n)
        pos = pos[order]
        species = species[order]
        if h_gas is not None and not np.isscalar(h_gas):
            raise ValueError("array h must be computed after shuffling")
    x = _wrap32(pos[:, 0], L)
    y = _wrap32(pos[:, 1], L)
    z = _wrap32(pos[:, 2], L)
    gas = species == GAS
    m = np.where(gas, MASS_GAS, MASS_DM).astype(np.float32)
    u = np.where(gas, rng.uniform(0.9, 1.1, n), 0.0).astype(np.float32)
    v = rng.normal(0.0, 0.05, (3, n))
    v[:, ~gas] = 0.0
    v = v.astype(np.float32)
    h = np.zeros(n, np.float32)
    ng = int(np.count_nonzero(gas))
    if h_gas is None:
        if ng > 0:
            pg = np.stack([x[gas], y[gas], z[gas]], axis=1).astype(np.float64)
            h[gas] = adaptive_h(pg, L)
    else:
        h[gas] = np.float32(h_gas)
    return Box(L=float(L), x=x, y=y, z=z, species=species.astype(np.uint8), m=m, h=h, u=u,
               vx=v[0].copy(), vy=v[1].copy(), vz=v[2].copy(), leaf_mode=leaf_mode,
               cells_per_side=cells, max_leaf=max_leaf, r_cut=R_CUT, eps=EPS,
               poly=gravity_poly(R_CUT, EPS), seed=seed, name=name)


def lattice_box(side: int, sigma: float, seed: int, h: float | None = 1.0, leaf_mode: int = 0,
                cells: int = 4, max_leaf: int = 128, name: str = "lattice") -> Box:
    """Two interleaved unit lattices (L = side) displaced by N(0, sigma^2) per axis."""
    rng = np.random.default_rng(seed)
    L = float(side)
    dm, gas = _lattices(side, L)
    pos = np.concatenate([dm, gas])
    if sigma > 0:
        pos = pos + rng.normal(0.0, sigma, pos.shape)
    species = np.concatenate([np.full(len(dm), DM, np.uint8), np.full(len(gas), GAS, np.uint8)])
    return _finish(L, pos, species, rng, h, name, seed, leaf_mode, cells, max_leaf)


def clustered_box(side: int, n_halos: int, seed: int, zel_rms: float = 0.5, halo_a: float = 0.5,
                  halo_n: int = 500, max_leaf: int = 128, name: str = "clustered") -> Box:
    """Zel'dovich-displaced lattices plus Plummer halos (the clustered recipe).

    The halos *replace* randomly chosen lattice particles, half dark matter and
    half gas, so the total stays 2 side^3.  Smoothing lengths are adaptive.
    """
    rng = np.random.default_rng(seed)
    L = float(side)
    dm, gas = _lattices(side, L)
    psi = zeldovich_displacement(side, L, zel_rms, rng)
    dm = dm + psi
    gas = gas + psi
    n_lat = side ** 3
    per_species = halo_n // 2
    need = n_halos * per_species
    if need > n_lat:
        raise ValueError("too many halo particles for this box")
    if n_halos > 0:
        centres = rng.random((n_halos, 3)) * L
        for arr in (dm, gas):
            pick = rng.choice(n_lat, size=need, replace=False)
            offs = plummer_offsets(need, halo_a, rng)
            arr[pick] = np.repeat(centres, per_species, axis=0) + offs
    pos = np.concatenate([dm, gas])
    species = np.concatenate([np.full(n_lat, DM, np.uint8), np.full(n_lat, GAS, np.uint8)])
    return _finish(L, pos, species, rng, None, name, seed, 1, 0, max_leaf)


def random_box(n: int, L: float, gas_frac: float, seed: int, max_leaf: int = 128, h: float | None = None,
               leaf_mode: int = 1, cells: int = 0, name: str = "random") -> Box:
    """Uniform random particles (any count, for ragged and edge cases)."""
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * L
    species = np.where(rng.random(n) < gas_frac, GAS, DM).astype(np.uint8)
    return _finish(L, pos, species, rng, h, name, seed, leaf_mode, cells, max_leaf, shuffle=False)


# --------------------------------------------------------------------------
# the five named workloads
# --------------------------------------------------------------------------

def tiny() -> Box:
    """L = 16, 2x16^3 (8192) lattice + sigma 0.2, h = 1, chaining mesh 4^3."""
    return lattice_box(16, 0.2, SEEDS["tiny"], h=1.0, leaf_mode=0, cells=4, name="tiny_2x16^3")


def clustered(side: int = 64, n_halos: int = 200) -> Box:
    """L = 64, 2x64^3 (524,288): Zel'dovich rms 0.5 + 200 Plummer halos, RCB <= 128."""
    return clustered_box(side, n_halos, SEEDS["clustered"], name=f"clustered_2x{side}^3")


def adjoint_box() -> Box:
    """L = 32, 2x32^3 (65,536), 25 halos: the adjoint workload."""
    return clustered_box(32, 25, SEEDS["adjoint"], name="adjoint_2x32^3")


def batched_sides(count: int = 96, seed: int = SEEDS["batched"]) -> list[int]:
    rng = np.random.default_rng(seed)
    return [int(round(math.exp(rng.uniform(math.log(12.0), math.log(48.0))))) for _ in range(count)]


def batched(count: int = 96) -> list[Box]:
    """96 boxes, integer sides log-uniform in [12, 48], 2 s^3 particles, round(200 (s/64)^3) halos."""
    out = []
    for b, s in enumerate(batched_sides(count)):
        nh = int(round(200.0 * (s / 64.0) ** 3))
        out.append(clustered_box(s, nh, SEEDS["batched"] * 1000 + b, name=f"batched[{b}]_2x{s}^3"))
    return out


def large() -> Box:
    """L = 256, 2x256^3 (33,554,432) with 5000 Plummer halos, RCB <= 128."""
    return clustered_box(256, 5000, SEEDS["large"], name="large_2x256^3")


WORKLOADS = {"tiny": tiny, "clustered": clustered, "adjoint": adjoint_box, "large": large}
