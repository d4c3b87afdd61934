"""Self-consistent Schrödinger–Poisson loop (oracle; test infrastructure).

Paper Section III-A: eigenstates of the tight-binding Hamiltonian -> charge (Fermi level by
neutrality) -> finite-difference Poisson -> potential back into the Hamiltonian, repeated
until self-consistent.  The paper's outer iteration is Newton–Raphson; this loop uses linear
mixing phi <- phi + mix (phi_out - phi), or Anderson mixing over the last mix_history iterates,
and stops when max |phi_out - phi| < tol_V, the reading the GPU path follows.  Electron potential energy U = -phi (eV per V).  Only states
above e_cut (mid-gap) hold electrons; g_s = 2.

poisson="newton": phi_out is the root of the nonlinear Poisson equation with the frozen
states' predicted charge (oracle/newton.py: Newton–Raphson, Section III-A item 3) instead of
the linear Poisson solution with the states' charge; the loop, the mixing and the stopping rule
are the same, and a self-consistent potential is a fixed point of both maps.
"""
from __future__ import annotations

import numpy as np

from . import charge, eigs, hamiltonian, lattice, newton, poisson

Q_E = poisson.Q_E


def atom_positions_nm(spec):
    return lattice.positions(spec.nx, spec.ny, spec.nz) * (spec.a_nm / 4.0)


def nearest_states(H, sigma, nev, dense_limit=2500):
    """nev eigenpairs nearest sigma: dense eigensolve for small H, else ARPACK shift-invert."""
    if H.shape[0] <= dense_limit:
        w, V = eigs.dense_eigh(H)
        order = np.lexsort((w, np.abs(w - sigma)))[:nev]
        order = order[np.argsort(w[order])]
        return w[order], V[:, order]
    return eigs.nearest_shift_invert(H, sigma, nev)


def anderson_update(phi, F, dX, dF, beta):
    """Anderson mixing (Anderson, J. ACM 12, 547 (1965)): gamma minimises |F - sum_j gamma_j dF_j|,
    phi_next = phi + beta F - sum_j gamma_j (dX_j + beta dF_j)."""
    if not dF:
        return phi + beta * F
    A = np.stack([d.ravel() for d in dF], axis=1)
    G = A.T @ A
    G = G + 1e-12 * np.max(np.diag(G)) * np.eye(len(dF))
    gamma = np.linalg.solve(G, A.T @ F.ravel())
    out = phi + beta * F
    for g, dx, df in zip(gamma, dX, dF):
        out = out - g * (dx + beta * df)
    return out


def scf(spec, params, grid, donor_rho, n_electrons, kT, kpts, kweights, nev, sigma, e_cut,
        mix=0.1, tol_V=1e-6, max_iter=300, phi0=None, gs=2.0, mix_history=0, poisson_mode="linear",
        newton_tol=1e-10):
    pos = atom_positions_nm(spec)
    bonds = lattice.find_bonds(spec.nx, spec.ny, spec.nz, spec.periodic)
    phi = np.zeros(grid.shape) if phi0 is None else np.array(phi0, float).reshape(grid.shape)
    history = []
    EF = None
    dX, dF = [], []
    F_prev = X_prev = None
    for it in range(1, max_iter + 1):
        U = -charge.gather(grid, phi, pos)
        levels, weights, states = [], [], []
        for k, wk in zip(kpts, kweights):
            H = hamiltonian.assemble(spec, params, U_atom=U, kvec=k, bonds=bonds)
            w, V = nearest_states(H, sigma, nev)
            states.append((w, V, wk))
            for e in w:
                if e > e_cut:
                    levels.append(e)
                    weights.append(gs * wk)
        EF = _fermi(np.array(levels), np.array(weights), n_electrons, kT)
        for w, V, wk in states:
            if charge.fermi(w.max(), EF, kT) > 1e-12:
                raise RuntimeError("highest computed state is occupied: raise nev")
        n_atom = np.zeros(spec.natoms)
        for w, V, wk in states:
            occ = np.where(w > e_cut, charge.fermi(w, EF, kT), 0.0)
            n_atom += gs * wk * charge.atom_density(V, occ, spec.natoms)
        if poisson_mode == "newton":
            cols, levels_n = [], []
            for w, V, wk in states:
                m = w > e_cut
                if m.any():
                    cols.append(newton.state_weights(V[:, m], gs * wk, spec.natoms))
                    levels_n.append(w[m])
            prob = newton.Problem(grid, pos, np.hstack(cols), np.concatenate(levels_n), EF, kT, phi, donor_rho)
            phi_out, _ = newton.solve(prob, phi, tol=newton_tol)
        else:
            rho = charge.deposit(grid, pos, -Q_E * n_atom) + donor_rho
            phi_out = poisson.solve_direct(grid, rho)
        dV = np.abs(phi_out - phi).max()
        history.append(dV)
        if dV < tol_V:
            return phi, {"iterations": it, "E_F": EF, "dV_inf": dV, "history": history, "n_atom": n_atom}
        if mix_history <= 0:
            phi = phi + mix * (phi_out - phi)
            continue
        F = phi_out - phi
        if F_prev is not None:
            dF.append(F - F_prev)
            dX.append(phi - X_prev)
            if len(dF) > mix_history:
                dF.pop(0)
                dX.pop(0)
        F_prev, X_prev = F, phi
        phi = anderson_update(phi, F, dX, dF, mix)
    return phi, {"iterations": max_iter, "E_F": EF, "dV_inf": history[-1], "history": history,
                 "converged": False}


def _fermi(levels, weights, n_target, kT):
    """Bisection on sum_i w_i f(E_i) = n_target."""
    lo, hi = levels.min() - 50 * kT, levels.max() + 50 * kT
    if weights.sum() < n_target:
        raise RuntimeError("not enough states for the electron count")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (weights * charge.fermi(levels, mid, kT)).sum() < n_target:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-13:
            break
    return 0.5 * (lo + hi)
