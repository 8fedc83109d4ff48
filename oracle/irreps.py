"""Form factors of the irreducible representations of C4v (Sec. 2) -- TEST INFRASTRUCTURE ONLY.

Sec. 2 allows any orthonormal set of form factors and names linear combinations of the plane waves
f_R(k) = e^{-ik.R} that transform under an irreducible representation of the point group.  For a bond set closed
under the eight point operations of the square lattice, this module builds them shell by shell (a shell = one
orbit of bonds): the permutation representation D(g) of the shell is projected with the characters of each
irreducible representation (A1, A2, B1, B2, E), P = (d / |G|) sum_g chi(g) D(g), and the projected space is given an
orthonormal real basis.  The combinations are f_i(k) = sum_R W[i, R] f_R(k), and the exchange propagators in that
basis are (W x 1) X (W x 1)^T per transfer momentum (W real orthogonal, 1 on the orbital pairs).

Written from the group's definition, independently of the library's construction; the two are compared through
quantities that do not depend on the choice of basis inside an irreducible subspace (its projector, block norms).
"""
from __future__ import annotations

import numpy as np

IRREPS = ("A1", "A2", "B1", "B2", "E")

# the eight operations as integer matrices acting on (x, y), with their class: identity, the two quarter turns,
# the half turn, the two axis mirrors, the two diagonal mirrors
_OPS = [(((1, 0), (0, 1)), "E"), (((0, -1), (1, 0)), "C4"), (((0, 1), (-1, 0)), "C4"), (((-1, 0), (0, -1)), "C2"),
        (((1, 0), (0, -1)), "sv"), (((-1, 0), (0, 1)), "sv"), (((0, 1), (1, 0)), "sd"), (((0, -1), (-1, 0)), "sd")]
# characters per class
_CHI = {"A1": {"E": 1, "C4": 1, "C2": 1, "sv": 1, "sd": 1},
        "A2": {"E": 1, "C4": 1, "C2": 1, "sv": -1, "sd": -1},
        "B1": {"E": 1, "C4": -1, "C2": 1, "sv": 1, "sd": -1},
        "B2": {"E": 1, "C4": -1, "C2": 1, "sv": -1, "sd": 1},
        "E": {"E": 2, "C4": 0, "C2": -2, "sv": 0, "sd": 0}}
_DIM = {"A1": 1, "A2": 1, "B1": 1, "B2": 1, "E": 2}


def operations():
    return [(np.array(m, dtype=int), c) for m, c in _OPS]


def perm_rep(ff_R: np.ndarray, g: np.ndarray) -> np.ndarray:
    """D(g)[i, j] = 1 when g R_j = R_i (the bonds as integer vectors)."""
    idx = {tuple(r): i for i, r in enumerate(np.asarray(ff_R).tolist())}
    n = len(idx)
    D = np.zeros((n, n))
    for j, r in enumerate(np.asarray(ff_R)):
        i = idx.get(tuple(g @ r))
        if i is None:
            raise ValueError("the bond set is not closed under the point group")
        D[i, j] = 1.0
    return D


def basis(ff_R: np.ndarray):
    """(W, labels): W [n][n] real orthogonal (row i = form factor i over the bonds), labels[i] = (shell, irrep index,
    partner); shells in order of first appearance in ff_R, irreps in the order A1, A2, B1, B2, E."""
    ff = np.asarray(ff_R, dtype=int)
    n = ff.shape[0]
    ops = operations()
    # shells: orbits of the bonds
    shell_of = -np.ones(n, dtype=int)
    shells = []
    for i in range(n):
        if shell_of[i] >= 0:
            continue
        members = sorted({tuple(g @ ff[i]) for g, _ in ops})
        ids = [int(np.where((ff == m).all(axis=1))[0][0]) for m in members]
        for j in ids:
            shell_of[j] = len(shells)
        shells.append(ids)
    D = {c: [perm_rep(ff, g) for g, cc in ops if cc == c] for c in ("E", "C4", "C2", "sv", "sd")}
    rows, labels = [], []
    for s, ids in enumerate(shells):
        sel = np.zeros((n, len(ids)))
        sel[ids, np.arange(len(ids))] = 1.0
        for gi, name in enumerate(IRREPS):
            P = sum(_CHI[name][c] * Dg for c in D for Dg in D[c]) * _DIM[name] / 8.0
            Ps = P @ sel                                  # the projector applied to the shell's bonds
            u, sv, _ = np.linalg.svd(Ps, full_matrices=False)
            vecs = u[:, sv > 1e-9]
            for p in range(vecs.shape[1]):
                v = vecs[:, p]
                v = v / np.linalg.norm(v)
                k = np.argmax(np.abs(v) > 1e-12)           # a fixed sign: first non-zero entry positive
                rows.append(v * np.sign(v[k]))
                labels.append((s, gi, p))
    W = np.array(rows)
    return W, labels


def transform(W: np.ndarray, X: np.ndarray, ns2: int) -> np.ndarray:
    """(W x 1) X (W x 1)^T for states X [2][Nq][M][M] (M = n_ff ns2)."""
    T = np.kron(W, np.eye(ns2))
    return np.einsum("ij,cqjk,lk->cqil", T, X, T)
