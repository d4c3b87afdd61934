"""Zincblende sites and nearest-neighbour bonds by brute-force search (oracle; test infrastructure).

The paper (Section II-A) describes each subdomain as a list of atoms plus their neighbour
atoms; the structures are zincblende (Si, SiGe, Section I).  Here every atom position is
generated and bonds are found by a k-d tree distance search (minimum image along periodic
directions), independently of any implicit indexing rule.

Positions are integers in units of a/4.  Sites per conventional cell:
A: (0,0,0) (0,2,2) (2,0,2) (2,2,0);  B = A + (1,1,1).
atom = b*ncells + cell, cell = (iz*ny + iy)*nx + ix.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.spatial import cKDTree

A_SITES = np.array([[0, 0, 0], [0, 2, 2], [2, 0, 2], [2, 2, 0]])
SITES = np.concatenate([A_SITES, A_SITES + 1])
BOND_DIRS = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]])


def positions(nx: int, ny: int, nz: int) -> np.ndarray:
    """Integer positions (a/4 units) of all 8*nx*ny*nz atoms, atom = b*ncells + cell."""
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1) * 4      # cell-major
    return (SITES[:, None, :] + cells[None, :, :]).reshape(-1, 3)


@dataclass
class Bonds:
    a: np.ndarray       # A-atom index per bond
    b: np.ndarray       # B-atom index per bond
    k: np.ndarray       # direction 0..3 of (B - A)
    T: np.ndarray       # image translation of the B atom (a/4 units), (nbonds, 3)
    slot: np.ndarray    # strain slot (k*4 + s)*ncells + cell of the A atom


def find_bonds(nx: int, ny: int, nz: int, periodic) -> Bonds:
    """All nearest-neighbour A-B pairs; a bond crossing a hard wall is absent."""
    pos = positions(nx, ny, nz)
    ncells = nx * ny * nz
    L = np.array([4 * nx, 4 * ny, 4 * nz])
    per = np.array([p != 0 for p in periodic])
    box = np.where(per, L, L + 64).astype(float)
    tree = cKDTree(pos.astype(float), boxsize=box)
    pairs = tree.query_pairs(r=1.9, output_type="ndarray")     # bond length sqrt(3) ~ 1.732
    i, j = pairs[:, 0], pairs[:, 1]
    isA = (i // ncells) < 4
    a = np.where(isA, i, j)
    b = np.where(isA, j, i)
    if np.any((a // ncells) >= 4) or np.any((b // ncells) < 4):
        raise AssertionError("a nearest-neighbour pair is not an A-B pair")
    d = pos[b] - pos[a]
    dmin = d.copy()
    for ax in range(3):
        if per[ax]:
            dmin[:, ax] = (d[:, ax] + 1) % L[ax] - 1
    T = dmin - d
    if not np.all(np.abs(dmin) == 1):
        raise AssertionError("bond vector is not of the form (+-1,+-1,+-1)")
    match = (dmin[:, None, :] == BOND_DIRS[None, :, :]).all(axis=2)
    if not np.all(match.sum(axis=1) == 1):
        raise AssertionError("bond vector is not one of the four zincblende directions")
    k = match.argmax(axis=1)
    s = a // ncells
    cell = a % ncells
    slot = (k * 4 + s) * ncells + cell
    order = np.argsort(slot, kind="stable")
    return Bonds(a[order], b[order], k[order], T[order], slot[order])
