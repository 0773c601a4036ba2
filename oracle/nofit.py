"""Exact (no-fit) multigrid exchange: the quantity ISDF approximates.

TEST INFRASTRUCTURE ONLY.  Two independent routes to the same matrix:

  * ``nofit_exchange`` follows the occ-RI / FFT route of Section II.A (second
    item of the list of remedies): for each occupied orbital i the densities
    rho_{mu i} are Fourier transformed and K_{mu nu} = sum_i (rho_{mu i}|rho_{nu i}).
    With the multigrid split (Section II.B) a pair is represented on the grid
    of its sharper factor, so rho_{mu i} = sum_l rho^l_{mu i} with
    rho^l_{mu i} = phi_mu sum_{lam : min(l(mu), l(lam)) = l} C_{lam i} phi_lam.
  * ``brute_exchange`` forms every pair density on its own level, builds the
    full 4-index tensor (mu lam|sig nu) by FFT and contracts it with D.

``brute_exchange_local`` is the same 4-index construction for the local
grids of Section III: a product with a finest-level (sharp) factor lives on
the finest grid, cut to the sphere of radius r_max (Eq. 5) around its owner
atom -- the sharp factor's atom, the lower index of the two when both are
sharp (reading R11) -- and every other product on its level as above.

All use the Coulomb rule of the oracle (reading R5).  They pin the ISDF
oracle from outside: with N_ip at the pair-space rank ISDF must reproduce them.
"""
from __future__ import annotations

import numpy as np

from .isdf import (basis_on_level, coulomb_pair, expand_functions, fourier_coeffs, level_sets, local_grid,
                   local_radius)


def _coul(Fa, la, Fb, lb, system):
    if la <= lb:
        return coulomb_pair(Fa, system["grids"][la], Fb, system["grids"][lb], system["edges"])
    return coulomb_pair(Fb, system["grids"][lb], Fa, system["grids"][la], system["edges"]).T


def nofit_exchange(system, C):
    """K^nofit (N x N) and E_x = -Tr(D K) by the occ-RI FFT route."""
    funcs = expand_functions(system)
    nfun = funcs["level"].shape[0]
    nlev = len(system["grids"])
    n_occ = C.shape[1]
    K = np.zeros((nfun, nfun))
    # per level: basis values of every function evaluated there (G_l)
    Phi = []
    for lev in range(nlev):
        L, N, G = level_sets(funcs, lev)
        Phi.append((L, N, G, basis_on_level(system, funcs, G, lev)))
    for i in range(n_occ):
        F = []
        for lev in range(nlev):
            L, N, G, PhiG = Phi[lev]
            pos = {int(mu): r for r, mu in enumerate(G)}
            psiG = C[G, i] @ PhiG  # sum over lam in G_l
            psiL = C[L, i] @ PhiG[[pos[int(m)] for m in L]] if L.size else np.zeros(PhiG.shape[1])
            rho = np.zeros((nfun, PhiG.shape[1]))
            for mu in L:
                rho[mu] = PhiG[pos[int(mu)]] * psiG
            for mu in N:
                rho[mu] = PhiG[pos[int(mu)]] * psiL
            F.append(fourier_coeffs(rho.T, system["grids"][lev]))
        for la in range(nlev):
            for lb in range(nlev):
                K += _coul(F[la], la, F[lb], lb, system)
    D = C @ C.T
    return K, -float(np.sum(D * K))


def brute_exchange(system, C):
    """K from the full 4-index tensor (tiny cells only)."""
    funcs = expand_functions(system)
    nfun = funcs["level"].shape[0]
    nlev = len(system["grids"])
    Phi = [basis_on_level(system, funcs, np.arange(nfun), lev) for lev in range(nlev)]
    pairs = [(m, l) for m in range(nfun) for l in range(nfun)]
    lev_of = [min(funcs["level"][m], funcs["level"][l]) for m, l in pairs]
    F = {}
    idx = {}
    for lev in range(nlev):
        sel = [q for q, lv in enumerate(lev_of) if lv == lev]
        idx[lev] = sel
        if not sel:
            continue
        rho = np.stack([Phi[lev][pairs[q][0]] * Phi[lev][pairs[q][1]] for q in sel], axis=0)
        F[lev] = fourier_coeffs(rho.T, system["grids"][lev])
    npair = len(pairs)
    eri = np.zeros((npair, npair))
    for la in F:
        for lb in F:
            eri[np.ix_(idx[la], idx[lb])] = _coul(F[la], la, F[lb], lb, system)
    eri = eri.reshape(nfun, nfun, nfun, nfun)  # (mu lam | sig nu)
    D = C @ C.T
    K = np.einsum("ls,mlsn->mn", D, eri)
    return K, -float(np.sum(D * K)), eri


def brute_exchange_local(system, C, eps_r):
    """K from the 4-index tensor of the local-grid pair partition (tiny cells).
    Built pair by pair from its definition, with no ISDF and no L/N sets."""
    funcs = expand_functions(system)
    nfun = funcs["level"].shape[0]
    nlev = len(system["grids"])
    fl, fa = funcs["level"], funcs["atom"]
    Phi = [basis_on_level(system, funcs, np.arange(nfun), lev) for lev in range(nlev)]
    r_max = local_radius(float(system["level_min_exp"][0]), eps_r)
    ng0 = Phi[0].shape[1]
    sphere = []
    for A in range(system["xyz"].shape[0]):
        _, parent, inside = local_grid(system, A, r_max)
        m = np.zeros(ng0, dtype=bool)
        m[parent[inside]] = True
        sphere.append(m)
    pairs = [(m, l) for m in range(nfun) for l in range(nfun)]
    rho = {lev: [] for lev in range(nlev)}
    idx = {lev: [] for lev in range(nlev)}
    for q, (m, l) in enumerate(pairs):
        lev = min(fl[m], fl[l])
        r = Phi[lev][m] * Phi[lev][l]
        if lev == 0:
            owners = [fa[x] for x in (m, l) if fl[x] == 0]
            r = np.where(sphere[min(owners)], r, 0.0)
        rho[lev].append(r)
        idx[lev].append(q)
    F = {lev: fourier_coeffs(np.stack(rho[lev], axis=0).T, system["grids"][lev]) for lev in range(nlev) if idx[lev]}
    npair = len(pairs)
    eri = np.zeros((npair, npair))
    for la in F:
        for lb in F:
            eri[np.ix_(idx[la], idx[lb])] = _coul(F[la], la, F[lb], lb, system)
    eri = eri.reshape(nfun, nfun, nfun, nfun)
    D = C @ C.T
    K = np.einsum("ls,mlsn->mn", D, eri)
    return K, -float(np.sum(D * K))
