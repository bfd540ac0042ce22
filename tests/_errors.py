"""Error statistics of a GPU output against the FP64 oracle, and the parity gates.

Two measures per output, over the particles it is defined for:

* E = sqrt(sum_i |d_i|^2 / sum_i |ref_i|^2), the global relative L2 error;
* e_i = |d_i| / (|ref_i| + 0.01 rms|ref|), the per-particle relative error,
  reported as its median, 99th percentile and maximum (the 0.01 rms floor
  keeps e_i defined where |ref_i| vanishes, e.g. on a lattice).

|.| is the Euclidean norm of a particle's row (3 components for vectors, 9
for tensors).  The benchmark spec fixes E <= 2e-5 for accelerations and dv/dt and
5e-5 for du/dt; every other gate here is about ten times the largest error
measured on GB300 for that output (the table of measured errors is kept with
the design notes).  Every comparison is recorded; with CRK_ERRORS_OUT set, the
test session writes the records to that JSON file.
"""
import numpy as np

RECORDS = []

# output -> (gate on E, gate on max_i e_i), about ten times the largest value measured on GB300
# over every box and variant of the GPU tests (E <= 2e-5 / 5e-5 for acc, dv, du is the benchmark spec's)
GATES = {
    "acc": (2e-5, 1e-4),
    "dv": (2e-5, 3e-4),
    "du": (5e-5, 3e-3),
    "V": (1e-5, 2e-5),
    "rho": (1e-5, 3e-5),
    "A": (1e-6, 2e-5),
    "B": (1e-5, 2e-4),
    "gA": (1e-5, 3e-4),
    "gB": (1e-5, 1e-4),
    "rhoR": (1e-5, 2e-5),
    "dvdx": (1e-5, 3e-5),
    # gravity adjoint: particles with a pair within FP32 rounding of r_c are left out of the
    # per-particle maximum (the force is continuous at r_c, its derivative g' is not, so FP32 and
    # FP64 deciding such a pair differently changes that particle's gradient at O(1))
    "gx": (3e-5, 5e-4),
    "gm": (1e-5, 2e-4),
    # adjoints of corrections and hydro, and the autograd chain
    "adj": (2e-5, 3e-3),
}


def rows(a, n):
    a = np.asarray(a, np.float64)
    return a.reshape(n, -1)


def stats(got, ref, exclude=None):
    """E and the per-particle e_i distribution of got against ref (rows = particles).

    exclude (bool per row, optional): rows left out of the e_i distribution (they still
    count in E); max_all is then the maximum over every row."""
    r = np.asarray(ref, np.float64)
    n = r.shape[0]
    r = rows(r, n)
    g = rows(got, n)
    if n == 0:
        return {"n": 0, "E": 0.0, "median": 0.0, "p99": 0.0, "max": 0.0, "max_all": 0.0, "excluded": 0}
    d = np.linalg.norm(g - r, axis=1)
    a = np.linalg.norm(r, axis=1)
    rms = float(np.sqrt(np.mean(a * a)))
    e = d / (a + 0.01 * rms + 1e-300)
    E = float(np.sqrt(np.sum(d * d) / max(np.sum(a * a), 1e-300)))
    keep = np.ones(n, bool) if exclude is None else ~np.asarray(exclude, bool)
    ek = e[keep] if keep.any() else np.zeros(1)
    return {"n": int(n), "E": E, "median": float(np.median(ek)), "p99": float(np.percentile(ek, 99)),
            "max": float(ek.max()), "max_all": float(e.max()), "excluded": int(n - keep.sum())}


def check(where, output, got, ref, gate=None, exclude=None):
    """Record the statistics of one output and assert its gates; returns the statistics.

    gate names the GATES entry (default: output); exclude as in stats."""
    s = stats(got, ref, exclude)
    key = gate or output
    gE, gmax = GATES[key]
    RECORDS.append({"where": where, "output": output, "gate": key, **s})
    assert s["E"] <= gE, (where, output, s)
    assert s["max"] <= gmax, (where, output, s)
    return s


def cut_boundary_particles(pos, L, r_cut, rel=4e-7, subset=None):
    """Particles with a partner whose squared distance lies within rel of r_cut^2 (FP32 rounding
    of the range decision, with r_cut rounded to FP32 as the kernels see it).  With subset
    (indices), the mask covers those rows only."""
    from scipy.spatial import cKDTree

    pos = np.asarray(pos, np.float64)
    n = pos.shape[0]
    rc = float(np.float32(r_cut))
    pts = np.where(pos >= L, pos - L, pos)
    tree = cKDTree(pts, boxsize=L)
    if subset is None:
        mask = np.zeros(n, bool)
        if n < 2:
            return mask
        pr = tree.query_pairs(rc * (1 + 1e-6), output_type="ndarray")
        if pr.size == 0:
            return mask
        d = pos[pr[:, 0]] - pos[pr[:, 1]]
        d -= L * np.rint(d / L)
        r2 = np.sum(d * d, axis=1)
        near = np.abs(r2 - rc * rc) <= rel * rc * rc
        mask[pr[near, 0]] = True
        mask[pr[near, 1]] = True
        return mask
    subset = np.asarray(subset, np.int64)
    mask = np.zeros(subset.size, bool)
    for q, i in enumerate(subset):
        js = np.asarray(tree.query_ball_point(pts[i], rc * (1 + 1e-6)), np.int64)
        d = pos[js] - pos[i]
        d -= L * np.rint(d / L)
        r2 = np.sum(d * d, axis=1)
        mask[q] = bool(np.any(np.abs(r2 - rc * rc) <= rel * rc * rc))
    return mask
