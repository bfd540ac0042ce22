"""Test-side brute-force pair enumeration in numpy (independent of the oracle's C search).

Used to check invariants that are sums over neighbours: it re-derives the
neighbour sets from the minimum-image convention directly, in vectorised
numpy, for small boxes only.
"""
import numpy as np


def min_image(d, L):
    return d - L * np.rint(d / L)


def all_pairs(pos, L, cut_ij, species_mask=None, include_self=True, chunk=512):
    """Return (i, j, x_ij) for every ordered pair with |x_ij| < cut_ij(i, j).

    cut_ij is a callable taking index arrays (I, J) and returning the cut for
    each pair.  species_mask restricts both i and j.
    """
    n = pos.shape[0]
    idx = np.arange(n) if species_mask is None else np.nonzero(species_mask)[0]
    out_i, out_j, out_x = [], [], []
    for s in range(0, idx.size, chunk):
        I = idx[s:s + chunk]
        d = min_image(pos[I][:, None, :] - pos[idx][None, :, :], L)
        r2 = np.sum(d * d, axis=2)
        II = np.broadcast_to(I[:, None], r2.shape)
        JJ = np.broadcast_to(idx[None, :], r2.shape)
        c = cut_ij(II, JJ)
        ok = r2 < c * c
        if not include_self:
            ok &= II != JJ
        out_i.append(II[ok])
        out_j.append(JJ[ok])
        out_x.append(d[ok])
    return np.concatenate(out_i), np.concatenate(out_j), np.concatenate(out_x)


def segment_sum(values, index, n):
    """sum values over groups given by index (values may be (k,) or (k, m))."""
    if values.ndim == 1:
        return np.bincount(index, weights=values, minlength=n)
    return np.stack([np.bincount(index, weights=values[:, c], minlength=n) for c in range(values.shape[1])], axis=1)
