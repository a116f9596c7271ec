"""CPU oracle of the automatic subdomain-levelset construction -- TEST
INFRASTRUCTURE ONLY (only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` may import it).

Section 3.2.2 and the physics-based deflation of Section 4 build one
deflation vector per region of nearly constant permeability inside each
subdomain: levelset classes split by thresholds, and, in the paper's manual
vectors, one vector per layer.  Automatically: every (subdomain, levelset
class) region is split into its face-connected components (6-neighbour
connectivity, inside the subdomain), and each component gets its own label.

Canonical numbering (so that results compare bit for bit): components are
ordered by (subdomain, class, smallest cell index of the component), i.e. by
(plain SLD label, smallest cell index), and numbered 0, 1, ... in that order.

Written as a plain union-find over the cells in index order (union by the
smaller root, so each component's root is its smallest cell index).
"""
from __future__ import annotations

import numpy as np

from . import labels as sld_labels


def cc_labels(K, S, tau, L):
    """(labels, d): labels int32 (flattened, x fastest), d components."""
    K = np.asarray(K, dtype=np.float64)
    nz, ny, nx = K.shape
    base = sld_labels(K, S, tau, L)
    n = K.size
    parent = list(range(n))

    def find(i):
        r = i
        while parent[r] != r:
            r = parent[r]
        while parent[i] != r:  # path compression
            parent[i], i = r, parent[i]
        return r

    def union(i, j):
        a, b = find(i), find(j)
        if a == b:
            return
        if a < b:
            parent[b] = a
        else:
            parent[a] = b

    b3 = base.reshape(nz, ny, nx)
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                i = (iz * ny + iy) * nx + ix
                lb = b3[iz, iy, ix]
                if ix + 1 < nx and b3[iz, iy, ix + 1] == lb:
                    union(i, i + 1)
                if iy + 1 < ny and b3[iz, iy + 1, ix] == lb:
                    union(i, i + nx)
                if iz + 1 < nz and b3[iz + 1, iy, ix] == lb:
                    union(i, i + nx * ny)
    root = np.array([find(i) for i in range(n)], dtype=np.int64)
    heads = np.flatnonzero(root == np.arange(n))          # ascending cell index
    order = np.lexsort((heads, base[heads]))               # by (SLD label, smallest index)
    newlab = np.empty(n, dtype=np.int64)
    newlab[heads[order]] = np.arange(heads.size)
    return newlab[root].astype(np.int32), int(heads.size)
