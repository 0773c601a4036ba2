"""Seeded synthetic periodic systems and occupied orbitals.

This module only builds INPUTS: cell geometry, the uncontracted Gaussian basis
(shell list), the real-space grid levels, and seeded occupied-orbital
coefficients.  It holds none of the ISDF / Coulomb / exchange arithmetic, so the
FP64 oracle and the CUDA path can both take their inputs from here.

Stand-in workloads.  The paper benchmarks diamond and LiH supercells with GTH
pseudopotentials and uncontracted GTH-CC-XZVP basis sets (Section IV, first
paragraph).  Those basis files are not available, so the workloads here are the
synthetic diamond cells described in the hot-path scope: a conventional cubic
cell of edge 6.74 bohr with 8 carbon atoms on the diamond sites, per atom
uncontracted Cartesian s exponents {0.1, 0.4, 1.6, 6.4} and p exponents
{0.15, 0.6, 2.4} (13 functions per atom), replicated into supercells and
optionally displaced by seeded Gaussian noise.

Function order convention (shared with the C ABI): shells in the order given;
an s shell contributes one function, a p shell three (x, y, z).
"""
from __future__ import annotations

import math

import numpy as np

A_DIAMOND = 6.74
DIAMOND_SITES = np.array(
    [
        [0.0, 0.0, 0.0],
        [0.0, 0.5, 0.5],
        [0.5, 0.0, 0.5],
        [0.5, 0.5, 0.0],
        [0.25, 0.25, 0.25],
        [0.25, 0.75, 0.75],
        [0.75, 0.25, 0.75],
        [0.75, 0.75, 0.25],
    ]
)
S_EXPS = (0.1, 0.4, 1.6, 6.4)
P_EXPS = (0.15, 0.6, 2.4)
LEVEL_EDGES_3 = (1.6, 0.4)  # >=1.6 fine, [0.4,1.6) mid, <0.4 coarse
SEED_BASE = 20240409


def make_system(
    reps=(1, 1, 1),
    sigma=0.0,
    rng=None,
    grids_per_cell=((48, 48, 48),),
    level_min_exp=(),
    a=A_DIAMOND,
    sites=DIAMOND_SITES,
    s_exps=S_EXPS,
    p_exps=P_EXPS,
    image_tol=1e-10,
):
    """Build a periodic orthorhombic supercell.

    grids_per_cell: per level, the number of grid points per axis for ONE
    conventional cell; the supercell grid is that times ``reps`` per axis.
    Atoms are wrapped into [0, L) after displacement.
    """
    reps = tuple(int(r) for r in reps)
    edges = np.array([a * reps[0], a * reps[1], a * reps[2]], dtype=np.float64)
    xyz = []
    for i in range(reps[0]):
        for j in range(reps[1]):
            for k in range(reps[2]):
                for s in sites:
                    xyz.append([(s[0] + i) * a, (s[1] + j) * a, (s[2] + k) * a])
    xyz = np.array(xyz, dtype=np.float64).reshape(-1, 3)
    if sigma > 0.0:
        if rng is None:
            raise ValueError("sigma > 0 needs an rng")
        xyz = xyz + rng.normal(0.0, sigma, size=xyz.shape)
    xyz = np.mod(xyz, edges)
    shell_atom, shell_l, shell_exp = [], [], []
    for ia in range(xyz.shape[0]):
        for e in s_exps:
            shell_atom.append(ia), shell_l.append(0), shell_exp.append(e)
        for e in p_exps:
            shell_atom.append(ia), shell_l.append(1), shell_exp.append(e)
    grids = np.array(
        [[g[0] * reps[0], g[1] * reps[1], g[2] * reps[2]] for g in grids_per_cell],
        dtype=np.int64,
    )
    return {
        "edges": edges,
        "xyz": xyz,
        "shell_atom": np.array(shell_atom, dtype=np.int32),
        "shell_l": np.array(shell_l, dtype=np.int32),
        "shell_exp": np.array(shell_exp, dtype=np.float64),
        "grids": grids,
        "level_min_exp": np.array(level_min_exp, dtype=np.float64),
        "image_tol": float(image_tol),
    }


def nbasis(system) -> int:
    return int(sum(1 if l == 0 else 3 for l in system["shell_l"]))


# ---------------------------------------------------------------------------
# Seeded occupied orbitals.  The overlap used to orthonormalise them is the
# analytic overlap of periodic Cartesian Gaussians (a property of the basis,
# not part of the ISDF method), so C is S-orthonormal and E_x is physical-ish.
# Parity never depends on it: both sides receive the same FP64 array.
# ---------------------------------------------------------------------------


def _overlap_1d(a, b, alpha, beta, A, B, L):
    """sum_t int (x-A)^a (x-B-tL)^b exp(-alpha(x-A)^2 - beta(x-B-tL)^2) dx."""
    p = alpha + beta
    mu = alpha * beta / p
    tmax = int(math.ceil(math.sqrt(40.0 / mu) / L)) + 1
    tot = 0.0
    for t in range(-tmax, tmax + 1):
        Bt = B + t * L
        d = A - Bt
        E = math.exp(-mu * d * d) * math.sqrt(math.pi / p)
        P = (alpha * A + beta * Bt) / p
        if a == 0 and b == 0:
            v = 1.0
        elif a == 1 and b == 0:
            v = P - A
        elif a == 0 and b == 1:
            v = P - Bt
        else:
            v = (P - A) * (P - Bt) + 0.5 / p
        tot += v * E
    return tot


def _functions(system):
    """List of (atom, alpha, (lx,ly,lz)) in the ABI function order."""
    out = []
    for ia, l, e in zip(system["shell_atom"], system["shell_l"], system["shell_exp"]):
        if l == 0:
            out.append((int(ia), float(e), (0, 0, 0)))
        else:
            for ax in range(3):
                lv = [0, 0, 0]
                lv[ax] = 1
                out.append((int(ia), float(e), tuple(lv)))
    return out


def analytic_overlap(system):
    funcs = _functions(system)
    xyz, edges = system["xyz"], system["edges"]
    n = len(funcs)
    norms = []
    for _, e, lv in funcs:
        nrm = (2.0 * e / math.pi) ** 0.75
        if sum(lv) == 1:
            nrm *= 2.0 * math.sqrt(e)
        norms.append(nrm)
    S = np.zeros((n, n))
    for i in range(n):
        ai, ei, li = funcs[i]
        for j in range(i, n):
            aj, ej, lj = funcs[j]
            v = norms[i] * norms[j]
            for ax in range(3):
                v *= _overlap_1d(li[ax], lj[ax], ei, ej, xyz[ai, ax], xyz[aj, ax], edges[ax])
            S[i, j] = S[j, i] = v
    return S


def make_orbitals(system, n_occ, rng):
    """C = C0 (C0^T S C0)^(-1/2) with C0 ~ N(0,1) of shape (N, n_occ)."""
    N = nbasis(system)
    C0 = rng.standard_normal((N, n_occ))
    S = analytic_overlap(system)
    G = C0.T @ S @ C0
    w, U = np.linalg.eigh(G)
    return np.ascontiguousarray(C0 @ (U * w ** -0.5) @ U.T)


# ---------------------------------------------------------------------------
# Named workloads.
# ---------------------------------------------------------------------------


def config(k: int):
    """Return (system, C, nip) for the named diamond workloads.

    1: 1x1x1 undisplaced, single 48^3 grid, N=104, n=16, N_ip=8N.
    2: 2x2x2, sigma=0.05, 3 levels 96^3/48^3/24^3, N=832, n=128, N_ip=6N.
    Seeds: numpy default_rng(20240409 + k); displacements are drawn first,
    then the N x n Gaussian orbital coefficients.
    """
    rng = np.random.default_rng(SEED_BASE + k)
    if k == 1:
        sysd = make_system((1, 1, 1), 0.0, rng, ((48, 48, 48),), ())
        n_occ, nip_per_n = 16, 8
    elif k == 2:
        sysd = make_system((2, 2, 2), 0.05, rng, ((48, 48, 48), (24, 24, 24), (12, 12, 12)), LEVEL_EDGES_3)
        n_occ, nip_per_n = 128, 6
    else:
        raise ValueError("only workloads 1 and 2 are defined here")
    C = make_orbitals(sysd, n_occ, rng)
    return sysd, C, nip_per_n * nbasis(sysd)


def batch_cells(sigma=0.1, n_each=6, per_cell=(48, 24, 12)):
    """The batched workload: n_each cells each of 1x1x1, 1x1x2, 1x2x2 and 2x2x2
    diamond supercells (24 by default), seeded displacements, three grid
    levels scaled with the cell, N_ip = 6N, n = 2 per atom.  Cell j of the
    batch uses numpy default_rng(20240409 + 3 + 1000 j)."""
    out = []
    j = 0
    for reps in ((1, 1, 1), (1, 1, 2), (1, 2, 2), (2, 2, 2)):
        for _ in range(n_each):
            rng = np.random.default_rng(SEED_BASE + 3 + 1000 * j)
            sysd = make_system(reps, sigma, rng, tuple((p, p, p) for p in per_cell), LEVEL_EDGES_3)
            C = make_orbitals(sysd, 2 * sysd["xyz"].shape[0], rng)
            out.append((sysd, C, 6 * nbasis(sysd)))
            j += 1
    return out


def small_multigrid(reps=(1, 1, 1), sigma=0.05, seed=7, per_cell=(16, 8, 4), n_occ=None, sites=DIAMOND_SITES,
                    a=A_DIAMOND):
    """A small 3-level cell for parity tests (same basis, coarser grids)."""
    rng = np.random.default_rng(seed)
    g = tuple((p, p, p) for p in per_cell)
    sysd = make_system(reps, sigma, rng, g, LEVEL_EDGES_3[: len(per_cell) - 1], a=a, sites=sites)
    if n_occ is None:
        n_occ = 2 * sysd["xyz"].shape[0]
    C = make_orbitals(sysd, n_occ, rng)
    return sysd, C
