"""Pins for the oracle's Slater–Koster blocks.

The oracle builds each bond block by rotating the bond-frame (sigma/pi/delta) block.  These
tests compare it with the closed-form entries of Slater & Koster, Phys. Rev. 94, 1498 (1954),
Table I, typed here independently (with the cyclic permutations the table prescribes), for
random directions and random parameters, and check the reversal rule and Harrison scaling.
"""
import numpy as np
import pytest

from oracle.sk import sk_block, harrison_factor

S3 = np.sqrt(3.0)
ORB = ["s", "x", "y", "z", "yz", "zx", "xy", "x2", "z2", "S"]
L_OF = {"s": 0, "S": 0, "x": 1, "y": 1, "z": 1, "yz": 2, "zx": 2, "xy": 2, "x2": 2, "z2": 2}
P = dict(ss=0, SS=1, sS=2, sp=3, Sp=4, sd=5, Sd=6, pps=7, ppp=8, pds=9, pdp=10, dds=11, ddp=12, ddd=13)


def table(a, b, c, V):
    """SK Table I entry E_{a,b}(l,m,n) with L_a <= L_b (s* treated as s)."""
    l, m, n = c
    sl = {"s": "s", "S": "S"}
    if a in sl and b in sl:
        key = {"ss": "ss", "SS": "SS", "sS": "sS"}[a + b]
        return V[P[key]]
    if a in sl and b in ("x", "y", "z"):
        return {"x": l, "y": m, "z": n}[b] * V[P["sp" if a == "s" else "Sp"]]
    if a in sl:
        Vs = V[P["sd" if a == "s" else "Sd"]]
        return {"xy": S3 * l * m, "yz": S3 * m * n, "zx": S3 * n * l,
                "x2": S3 / 2 * (l * l - m * m), "z2": n * n - (l * l + m * m) / 2}[b] * Vs
    if a in ("x", "y", "z") and b in ("x", "y", "z"):
        ci = {"x": l, "y": m, "z": n}
        if a == b:
            return ci[a] ** 2 * V[P["pps"]] + (1 - ci[a] ** 2) * V[P["ppp"]]
        return ci[a] * ci[b] * (V[P["pps"]] - V[P["ppp"]])
    if a in ("x", "y", "z"):
        ps, pp = V[P["pds"]], V[P["pdp"]]
        if b in ("xy", "yz", "zx"):
            # table rows E_x,xy  E_x,yz  E_x,zx ; others by cyclic permutation
            k = {"x": 0, "y": 1, "z": 2}[a]
            base = {0: {"xy": "xy", "yz": "yz", "zx": "zx"},
                    1: {"yz": "xy", "zx": "yz", "xy": "zx"},
                    2: {"zx": "xy", "xy": "yz", "yz": "zx"}}[k][b]
            # with x->y->z->x applied k times, E_{a,b}(l,m,n) = E_{x,base}(cosines rotated back)
            L, M, N = {0: (l, m, n), 1: (m, n, l), 2: (n, l, m)}[k]
            if base == "xy":
                return S3 * L * L * M * ps + M * (1 - 2 * L * L) * pp
            if base == "yz":
                return S3 * L * M * N * ps - 2 * L * M * N * pp
            return S3 * L * L * N * ps + N * (1 - 2 * L * L) * pp
        if b == "x2":
            return {"x": S3 / 2 * l * (l * l - m * m) * ps + l * (1 - l * l + m * m) * pp,
                    "y": S3 / 2 * m * (l * l - m * m) * ps - m * (1 + l * l - m * m) * pp,
                    "z": S3 / 2 * n * (l * l - m * m) * ps - n * (l * l - m * m) * pp}[a]
        if b == "z2":
            q = n * n - (l * l + m * m) / 2
            return {"x": l * q * ps - S3 * l * n * n * pp,
                    "y": m * q * ps - S3 * m * n * n * pp,
                    "z": n * q * ps + S3 * n * (l * l + m * m) * pp}[a]
    # d - d
    s_, p_, d_ = V[P["dds"]], V[P["ddp"]], V[P["ddd"]]
    t2g = ("xy", "yz", "zx")
    if a in t2g and b in t2g:
        # table rows E_xy,xy and E_xy,yz, E_xy,zx; others by cyclic permutation
        k = {"xy": 0, "yz": 1, "zx": 2}[a]
        L, M, N = {0: (l, m, n), 1: (m, n, l), 2: (n, l, m)}[k]
        rel = {0: {"xy": "xy", "yz": "yz", "zx": "zx"},
               1: {"yz": "xy", "zx": "yz", "xy": "zx"},
               2: {"zx": "xy", "xy": "yz", "yz": "zx"}}[k][b]
        if rel == "xy":
            return 3 * L * L * M * M * s_ + (L * L + M * M - 4 * L * L * M * M) * p_ + (N * N + L * L * M * M) * d_
        if rel == "yz":
            return 3 * L * M * M * N * s_ + L * N * (1 - 4 * M * M) * p_ + L * N * (M * M - 1) * d_
        return 3 * L * L * M * N * s_ + M * N * (1 - 4 * L * L) * p_ + M * N * (L * L - 1) * d_
    if a in t2g and b == "x2":
        q = l * l - m * m
        return {"xy": 1.5 * l * m * q * s_ + 2 * l * m * (m * m - l * l) * p_ + 0.5 * l * m * q * d_,
                "yz": 1.5 * m * n * q * s_ - m * n * (1 + 2 * q) * p_ + m * n * (1 + q / 2) * d_,
                "zx": 1.5 * n * l * q * s_ + n * l * (1 - 2 * q) * p_ - n * l * (1 - q / 2) * d_}[a]
    if a in t2g and b == "z2":
        q = n * n - (l * l + m * m) / 2
        return {"xy": S3 * l * m * q * s_ - 2 * S3 * l * m * n * n * p_ + S3 / 2 * l * m * (1 + n * n) * d_,
                "yz": S3 * m * n * q * s_ + S3 * m * n * (l * l + m * m - n * n) * p_ - S3 / 2 * m * n * (l * l + m * m) * d_,
                "zx": S3 * l * n * q * s_ + S3 * l * n * (l * l + m * m - n * n) * p_ - S3 / 2 * l * n * (l * l + m * m) * d_}[a]
    if a == "x2" and b == "x2":
        q = l * l - m * m
        return 0.75 * q * q * s_ + (l * l + m * m - q * q) * p_ + (n * n + q * q / 4) * d_
    if a == "x2" and b == "z2":
        q = l * l - m * m
        return S3 / 2 * q * (n * n - (l * l + m * m) / 2) * s_ + S3 * n * n * (m * m - l * l) * p_ + S3 / 4 * (1 + n * n) * q * d_
    if a == "z2" and b == "z2":
        q = n * n - (l * l + m * m) / 2
        return q * q * s_ + 3 * n * n * (l * l + m * m) * p_ + 0.75 * (l * l + m * m) ** 2 * d_
    raise KeyError((a, b))


def _canonical(a, b):
    la, lb = L_OF[a], L_OF[b]
    if la != lb:
        return la < lb
    if la == 0:
        return not (a == "S" and b == "s")
    if la == 2:
        rank = ["xy", "yz", "zx", "x2", "z2"]
        return rank.index(a) <= rank.index(b)
    return True


def table_block(c, V12, V21):
    """Full 10x10 block from Table I: <1a|H|2b> = E_ab(c; V12) if (a,b) is a table pair,
    else (-1)^(La+Lb) E_ba(c; V21) (the parity of the two-centre integral)."""
    B = np.zeros((10, 10))
    for i, a in enumerate(ORB):
        for j, b in enumerate(ORB):
            if _canonical(a, b):
                B[i, j] = table(a, b, c, V12)
            else:
                B[i, j] = (-1) ** (L_OF[a] + L_OF[b]) * table(b, a, c, V21)
    return B


@pytest.mark.parametrize("seed", range(6))
def test_rotated_block_matches_sk_table(seed):
    g = np.random.default_rng(seed)
    for _ in range(5):
        u = g.normal(size=3)
        u /= np.linalg.norm(u)
        V12 = g.uniform(-3, 3, 14)
        V21 = g.uniform(-3, 3, 14)
        V21[[P["pps"], P["ppp"], P["dds"], P["ddp"], P["ddd"], P["ss"], P["SS"]]] = \
            V12[[P["pps"], P["ppp"], P["dds"], P["ddp"], P["ddd"], P["ss"], P["SS"]]]
        ref = table_block(tuple(u), V12, V21)
        got = sk_block(u, V12, V21, 10)
        np.testing.assert_allclose(got, ref, atol=1e-12)


def test_sp3s_block_is_the_sp3d5s_block_without_d():
    g = np.random.default_rng(11)
    u = g.normal(size=3)
    V12, V21 = g.uniform(-3, 3, 14), g.uniform(-3, 3, 14)
    full = sk_block(u, V12, V21, 10)
    keep = [0, 1, 2, 3, 9]
    np.testing.assert_allclose(sk_block(u, V12, V21, 5), full[np.ix_(keep, keep)], atol=1e-13)


SAME_L = [P["pps"], P["ppp"], P["dds"], P["ddp"], P["ddd"], P["ss"], P["SS"]]


def test_reversed_bond_gives_transposed_block():
    """Swapping the atoms reverses u and exchanges V12/V21 (same-l integrals are symmetric)."""
    g = np.random.default_rng(3)
    for _ in range(10):
        u = g.normal(size=3)
        V12, V21 = g.uniform(-3, 3, 14), g.uniform(-3, 3, 14)
        V21[SAME_L] = V12[SAME_L]
        np.testing.assert_allclose(sk_block(-u, V21, V12, 10), sk_block(u, V12, V21, 10).T, atol=1e-12)


def test_harrison_scaling():
    assert harrison_factor(1.0) == 1.0
    np.testing.assert_allclose(harrison_factor(1.02), 1.02 ** -2)
    np.testing.assert_allclose(harrison_factor(0.5, eta=3.0), 8.0)
