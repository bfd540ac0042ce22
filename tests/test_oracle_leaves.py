"""Pins of the oracle's leaves and leaf-pair lists (integer results, bit-exact).

The paper names the RCB tree (Sec. 3.1) and leaf-pair work (Sec. 5.3) but
fixes no tie rule; the oracle header states the rules.  The pins are hand-
worked examples (tests/golden/leaves_hand_worked.json), properties that
characterise recursive coordinate bisection completely, and brute-force
coverage of every in-range particle pair by the listed leaf pairs.
"""
import json
import os

import numpy as np
import pytest

from paper_2310_16122_gb300 import workloads as W
from tests._pairs import all_pairs, min_image

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "leaves_hand_worked.json")))


def _inputs(orc, pos, species, L=10.0, h=None):
    n = len(pos)
    h = np.zeros(n) if h is None else np.asarray(h, float)
    return orc.Inputs(np.asarray(pos, float), species, np.ones(n), h, np.zeros(n), np.zeros((n, 3)), L, 1.5, 0.1,
                      np.zeros(6))


@pytest.mark.parametrize("case", GOLD["rcb"], ids=lambda c: c["name"])
def test_rcb_hand_worked(orc, case):
    I = _inputs(orc, case["pos"], case["species"])
    perm, start = orc.leaves_rcb(I, case["max_leaf"])
    assert perm.tolist() == case["perm"]
    assert start.tolist() == case["leaf_start"]


def test_mesh_hand_worked(orc):
    case = GOLD["mesh"][0]
    I = _inputs(orc, case["pos"], case["species"], L=case["L"], h=case["h"])
    I.r_cut = case["grav_rc"]
    perm, start = orc.leaves_mesh(I, case["nc"])
    leaf_of = np.empty(I.n, int)
    for a in range(start.size - 1):
        leaf_of[perm[start[a]:start[a + 1]]] = a
    assert leaf_of.tolist() == case["leaf_of"]
    assert perm[start[0]:start[1]].tolist() == case["leaf0_order"]
    ptr, lst = orc.leaf_pairs(I, perm, start, hydro=False)
    assert lst[ptr[0]:ptr[1]].tolist() == case["grav_pairs_of_leaf0"]
    ptr, lst = orc.leaf_pairs(I, perm, start, hydro=True)
    assert lst[ptr[0]:ptr[1]].tolist() == case["hydro_pairs_of_leaf0"]


def _leaf_sizes(n, max_leaf):
    """Leaf ranges of the bisection tree, which depend on n alone (left child floor(n/2))."""
    out = []

    def rec(lo, hi, depth):
        if hi - lo <= max_leaf:
            out.append((lo, hi))
            return
        mid = lo + (hi - lo) // 2
        nodes.append((lo, mid, hi))
        rec(lo, mid, depth + 1)
        rec(mid, hi, depth + 1)

    nodes = []
    if n > 0:
        rec(0, n, 0)
    return out, nodes


@pytest.mark.parametrize("n,max_leaf,seed", [(3456, 128, 1), (1000, 7, 2), (129, 128, 3), (1, 128, 4), (0, 128, 5)])
def test_rcb_characterisation(orc, n, max_leaf, seed):
    """Every internal node splits its longest extent at floor(n/2) in (coordinate, index) order."""
    if n >= 3456:
        b = W.clustered_box(12, 1, seed)
    else:
        b = W.random_box(n, 10.0, 0.5, seed, h=0.3)
    I = orc.from_box(b)
    perm, start = orc.leaves_rcb(I, max_leaf)
    assert sorted(perm.tolist()) == list(range(I.n))
    leaves, nodes = _leaf_sizes(I.n, max_leaf)
    assert start.tolist() == ([lo for lo, _ in leaves] + [I.n] if I.n else [0])
    for lo, mid, hi in nodes:
        mem = perm[lo:hi]
        p = I.pos[mem]
        ext = p.max(axis=0) - p.min(axis=0)
        axis = int(np.argmax(ext))  # argmax returns the first maximum: ties prefer x, then y
        key = lambda k: (I.pos[k, axis], k)
        left = max(map(key, perm[lo:mid]))
        right = min(map(key, perm[mid:hi]))
        assert left < right
    for lo, hi in leaves:
        mem = perm[lo:hi]
        sp = I.species[mem]
        assert np.all(np.diff(sp.astype(int)) >= 0)  # gas first
        for s in (0, 1):
            ids = mem[sp == s]
            assert np.all(np.diff(ids) > 0)


def test_mesh_membership_tiny(orc):
    b = W.tiny()
    I = orc.from_box(b)
    perm, start = orc.leaves_mesh(I, 4)
    c = np.minimum(3, np.floor(I.pos * 4 / I.L).astype(int))
    lid = (c[:, 0] * 4 + c[:, 1]) * 4 + c[:, 2]
    for a in range(64):
        mem = perm[start[a]:start[a + 1]]
        assert np.all(lid[mem] == a)
        assert np.all(np.diff(I.species[mem].astype(int)) >= 0)
    assert start[-1] == I.n


def _gap2(I, perm, start):
    nl = start.size - 1
    lo = np.full((nl, 3), np.inf)
    hi = np.full((nl, 3), -np.inf)
    for a in range(nl):
        mem = perm[start[a]:start[a + 1]]
        if mem.size:
            lo[a] = I.pos[mem].min(axis=0)
            hi[a] = I.pos[mem].max(axis=0)
    L = I.L
    g = np.full((nl, nl, 3), np.inf)
    for s in (-L, 0.0, L):
        t1 = (lo[None, :, :] + s) - hi[:, None, :]
        t2 = (lo[:, None, :] - hi[None, :, :]) - s
        g = np.minimum(g, np.maximum(0.0, np.maximum(t1, t2)))
    return (g[..., 0] ** 2 + g[..., 1] ** 2) + g[..., 2] ** 2


@pytest.mark.parametrize("which", ["tiny", "clustered12"])
def test_leaf_pairs_exact_and_covering(orc, which):
    """The list equals the box-gap rule (numpy restatement) and covers every in-range particle pair."""
    if which == "tiny":
        b = W.tiny()
        I = orc.from_box(b)
        perm, start = orc.leaves_mesh(I, 4)
    else:
        b = W.clustered_box(12, 1, 21)
        I = orc.from_box(b)
        perm, start = orc.leaves_rcb(I, 128)
    nl = start.size - 1
    leaf_of = np.empty(I.n, int)
    for a in range(nl):
        leaf_of[perm[start[a]:start[a + 1]]] = a
    d2 = _gap2(I, perm, start)
    cnt = np.diff(start)
    ngas = np.array([np.sum(I.species[perm[start[a]:start[a + 1]]] == 0) for a in range(nl)])
    hmax = np.array([I.h[perm[start[a]:start[a + 1]]].max(initial=0.0) for a in range(nl)])
    for hydro in (False, True):
        ptr, lst = orc.leaf_pairs(I, perm, start, hydro=hydro)
        listed = np.zeros((nl, nl), bool)
        for a in range(nl):
            listed[a, lst[ptr[a]:ptr[a + 1]]] = True
            assert np.all(np.diff(lst[ptr[a]:ptr[a + 1]]) > 0)
        if hydro:
            cut = 2.0 * np.maximum(hmax[:, None], hmax[None, :])
            ok = (ngas[:, None] > 0) & (ngas[None, :] > 0)
            i, j, _ = all_pairs(I.pos, I.L, lambda a, c: I.h[a] + I.h[c], species_mask=I.species == 0)
        else:
            cut = np.full((nl, nl), I.r_cut)
            ok = (cnt[:, None] > 0) & (cnt[None, :] > 0)
            i, j, _ = all_pairs(I.pos, I.L, lambda a, c: np.full(a.shape, I.r_cut))
        expect = ok & (d2 < cut * cut)
        assert np.array_equal(listed, expect)
        assert np.all(listed[leaf_of[i], leaf_of[j]])
        assert np.array_equal(listed, listed.T)
