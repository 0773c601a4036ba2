"""Plain FP64 NumPy/SciPy multigrid ISDF and THC exchange (test oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Nothing here is tuned;
every step follows the paper's definitions in the paper's order:

  * Section II ("THEORY"): THC form of the ERIs, interpolative decomposition of
    the pair densities (mu nu | R) = sum_xi (mu nu | xi) xi(R), and the
    two-centre Coulomb matrix (xi|xi') of Eq. 1 evaluated with FFTs.
  * Section II.A: Eq. 2 (M(R,R') = sum_{mu nu} (mu nu|R)(mu nu|R')), pivoted
    Cholesky on M for the interpolation points, Eq. 3 (least-squares fit of the
    interpolation vectors xi(R)).
  * Section II.B / III: the basis is split by exponent; a product is only
    represented on the grid of its sharper factor (Eq. 7 with the L / G / N
    function sets).
  * Section III.A: the four-term multigrid THC form of the ERIs, Eq. 8, used to
    build the exchange matrix.

Readings of places where the paper is silent or garbled:
  R1 levels: a function of exponent a lives on level l = #{edges e : a < e};
     level 0 is the finest grid.  Level l holds the pairs whose sharper factor
     is on level l: L_l = {mu: l(mu)=l}, N_l = {mu: l(mu)>l}, G_l = L_l u N_l.
     The pair set of level l is (L_l x G_l) u (N_l x L_l) (ordered pairs), so
     M_l = A_L o A_L + 2 A_L o A_N with A_X(g,g') = sum_{mu in X} phi_mu(g) phi_mu(g').
  R2 selection: one greedy pivoted Cholesky over the block-diagonal matrix
     (+)_l w_l M_l with w_l = dV_l (grid volume element), so a pivot value is a
     quadrature of squared pair density on every level.
  R3 ties: among points with d >= d_max - max(tie_rel*d_max, tie_abs*d_0) the
     smallest (level, g) wins; the chosen point's residual is then set to 0.
  R4 fit regularisation: lambda = reg_rel * tr(CC^T) / k_l (per level).
  R5 Coulomb: every grid function stands for its trigonometric interpolant (a
     coefficient whose mode sits at +-n/2 on an axis is split evenly between
     the two); (f|g) is the exact periodic Coulomb integral of the interpolants
     with the G=0 term dropped.  Cross-level pairs therefore sum over the
     coarser level's (extended) mode set.
  R6 Eq. 8 reading: c_{mu lam}(P) = X^L_{mu P} X^G_{lam P} + X^N_{mu P} X^L_{lam P}
     where X^L_{mu P} = phi_mu(P) for mu in L_{l(P)} (else 0) and X^N likewise
     for N_{l(P)}; (mu lam|sig nu) = sum_PQ c_{mu lam}(P) V_PQ c_{sig nu}(Q).
  R7 images: on an orthorhombic cell the image sum of a Cartesian Gaussian is
     taken over the box of lattice translations t (per axis) whose shifted
     centre A + t L lies within r_cut = sqrt(ln(1/image_tol)/alpha) of [0, L].
  R10 local grids: alpha_min is the finest level's edge; atom A's grid is
     the finest grid's points within r_max (Eq. 5) of A, taken from a box
     around A's nearest grid index (local_grid); a box wider than the cell
     is refused.
  R11 local function sets: L_A = finest-level functions of A, N_A = finest-
     level functions of atoms with a larger index plus all coarser functions
     (a sharp-sharp product of two atoms is represented once, on the grid of
     the lower-index atom; functions vanishing on the sphere are kept).
  R12 local ISDF: per atom its own greedy (Eq. 2) with a cap and a threshold
     relative to the atom's largest initial residual, its own fit (Eq. 3,
     lambda per atom); the coarser levels are selected together as usual.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

PIVOT_SHIFT = 40  # pivot code = (level << 40) | g


# ---------------------------------------------------------------------------
# Basis functions and levels (Section II.B / III, Fig. Grids; reading R1, R7)
# ---------------------------------------------------------------------------


def expand_functions(system):
    """Expand the shell list into functions (atom, alpha, lx, ly, lz, norm, level).

    Normalisation of an uncontracted Cartesian Gaussian x^l exp(-alpha r^2):
    s: (2 alpha/pi)^(3/4); p: (2 alpha/pi)^(3/4) * 2 sqrt(alpha).
    Level of a function (reading R1): the number of level edges above alpha.
    """
    edges = np.asarray(system["level_min_exp"], dtype=np.float64)
    atom, alpha, lvec, norm, level = [], [], [], [], []
    for ia, l, e in zip(system["shell_atom"], system["shell_l"], system["shell_exp"]):
        comps = [(0, 0, 0)] if l == 0 else [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
        for c in comps:
            atom.append(int(ia))
            alpha.append(float(e))
            lvec.append(c)
            nrm = (2.0 * e / math.pi) ** 0.75
            if l == 1:
                nrm *= 2.0 * math.sqrt(e)
            norm.append(nrm)
            level.append(int(np.sum(float(e) < edges)))
    return {
        "atom": np.array(atom, dtype=np.int64),
        "alpha": np.array(alpha),
        "lvec": np.array(lvec, dtype=np.int64),
        "norm": np.array(norm),
        "level": np.array(level, dtype=np.int64),
    }


def level_sets(funcs, lev):
    """(L, N, G) index arrays for level ``lev`` (reading R1, Eq. 7 notation)."""
    fl = funcs["level"]
    L = np.flatnonzero(fl == lev)
    N = np.flatnonzero(fl > lev)
    G = np.flatnonzero(fl >= lev)
    return L, N, G


def _images_1d(A, L, alpha, tol):
    """Lattice translations t (integers) kept for one axis (reading R7)."""
    rcut = math.sqrt(math.log(1.0 / tol) / alpha)
    tmax = int(math.ceil((rcut + L) / L)) + 1
    keep = []
    for t in range(-tmax, tmax + 1):
        c = A + t * L
        dist = 0.0 if 0.0 <= c <= L else min(abs(c), abs(c - L))
        if dist <= rcut:
            keep.append(t)
    return keep


def _periodic_gaussian_1d(x, A, L, alpha, l, tol):
    out = np.zeros_like(x)
    for t in _images_1d(A, L, alpha, tol):
        u = x - A - t * L
        out += (u ** l) * np.exp(-alpha * u * u)
    return out


def grid_points_1d(system, lev):
    n = system["grids"][lev]
    return [np.arange(n[a]) * (system["edges"][a] / n[a]) for a in range(3)]


def basis_on_level(system, funcs, idx, lev):
    """Phi[f, g] = phi_idx[f](r_g) on level ``lev``; g = i + nx (j + ny k).

    The image-summed Cartesian Gaussian on an orthorhombic lattice is a
    product of three 1-D image sums (the Gaussian and the monomial both
    separate over x, y, z and the kept translations form a box), so each
    function is the outer product of three 1-D periodic factors.  Pinned
    against ``basis_direct`` (literal 3-D image sum) and against the
    Poisson-summation Fourier series.
    """
    xs = grid_points_1d(system, lev)
    n = system["grids"][lev]
    tol = system["image_tol"]
    out = np.empty((len(idx), int(n[0] * n[1] * n[2])))
    for r, mu in enumerate(idx):
        A = system["xyz"][funcs["atom"][mu]]
        a = funcs["alpha"][mu]
        f = [
            _periodic_gaussian_1d(xs[ax], A[ax], system["edges"][ax], a, funcs["lvec"][mu][ax], tol)
            for ax in range(3)
        ]
        # array index [k, j, i] -> flat g = i + nx (j + ny k)
        out[r] = funcs["norm"][mu] * np.einsum("k,j,i->kji", f[2], f[1], f[0]).ravel()
    return out


def basis_direct(system, funcs, idx, lev):
    """Literal 3-D image sum of each function over the kept translations."""
    xs = grid_points_1d(system, lev)
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    tol = system["image_tol"]
    E = system["edges"]
    out = np.zeros((len(idx), P.shape[0]))
    for r, mu in enumerate(idx):
        A = system["xyz"][funcs["atom"][mu]]
        a = funcs["alpha"][mu]
        lv = funcs["lvec"][mu]
        T = [_images_1d(A[ax], E[ax], a, tol) for ax in range(3)]
        for tx in T[0]:
            for ty in T[1]:
                for tz in T[2]:
                    u = P - (A + np.array([tx * E[0], ty * E[1], tz * E[2]]))
                    poly = (u[:, 0] ** lv[0]) * (u[:, 1] ** lv[1]) * (u[:, 2] ** lv[2])
                    out[r] += poly * np.exp(-a * np.sum(u * u, axis=1))
        out[r] *= funcs["norm"][mu]
    return out


def fft_sizes(limit=4096):
    """Even grid sizes of the form 2^a 3^b (a >= 1), ascending."""
    out = []
    for a in range(1, 13):
        for b in range(0, 8):
            n = (2 ** a) * (3 ** b)
            if n <= limit:
                out.append(n)
    return sorted(out)


def grid_for_threshold(length, alpha, eps_K):
    """Points per axis that resolve exp(-alpha r^2) to eps_K in Fourier space
    (Section III, Eq. 6): the function's Fourier transform exp(-G^2/4 alpha)
    falls to eps_K at G_max = sqrt(-4 alpha ln eps_K), and a grid of n points
    over ``length`` carries wave numbers up to pi n / length (Nyquist).
    Smallest even 2^a 3^b size with pi n / length >= G_max."""
    gmax = math.sqrt(-4.0 * alpha * math.log(eps_K))
    for n in fft_sizes():
        if math.pi * n / length >= gmax:
            return n
    raise ValueError("threshold needs more than 4096 points per axis")


def grids_for_threshold(system, eps_K):
    """Grid of every level from eps_K (Section III, Eq. 6): level l must
    resolve its sharpest function -- the largest exponent among the functions
    of level l (reading R1), or, when it has none, among the coarser ones.
    Per axis the counts must then fall strictly from level to level (a
    coarser level's mode set inside every finer one): going from the coarsest
    level up, a level's count is raised to the next size above the coarser
    level's where needed.  Returns an int array (nlevel, 3)."""
    edges = np.asarray(system["level_min_exp"], dtype=np.float64)
    nlev = edges.size + 1
    exps = np.asarray(system["shell_exp"], dtype=np.float64)
    lev_of = np.array([int(np.sum(e < edges)) for e in exps])
    sizes = fft_sizes()
    out = np.zeros((nlev, 3), dtype=np.int64)
    for lev in range(nlev):
        own = exps[lev_of == lev]
        coarser = exps[lev_of > lev]
        alpha = own.max() if own.size else (coarser.max() if coarser.size else None)
        for ax in range(3):
            out[lev, ax] = 2 if alpha is None else grid_for_threshold(system["edges"][ax], alpha, eps_K)
    for lev in range(nlev - 2, -1, -1):
        for ax in range(3):
            if out[lev, ax] <= out[lev + 1, ax]:
                out[lev, ax] = next(n for n in sizes if n > out[lev + 1, ax])
    return out


def level_weight(system, lev):
    """w_l = dV_l = Omega / N_g,l (reading R2)."""
    n = system["grids"][lev]
    return float(np.prod(system["edges"]) / np.prod(n))


# ---------------------------------------------------------------------------
# Point selection: pivoted Cholesky on M (Section II.A, Eq. 2; readings R1-R3)
# ---------------------------------------------------------------------------


def _level_data(system, funcs):
    nlev = len(system["grids"])
    out = []
    for lev in range(nlev):
        L, N, G = level_sets(funcs, lev)
        out.append(
            {
                "L": L,
                "N": N,
                "PhiL": basis_on_level(system, funcs, L, lev),
                "PhiN": basis_on_level(system, funcs, N, lev),
                "w": level_weight(system, lev),
            }
        )
    return out


def m_columns(ld, cols):
    """M_l[:, cols] = A_L o (A_L + 2 A_N) at the given grid points (reading R1, Eq. 2)."""
    AL = ld["PhiL"].T @ ld["PhiL"][:, cols]
    AN = ld["PhiN"].T @ ld["PhiN"][:, cols]
    return AL * (AL + 2.0 * AN)


def initial_diagonal(ld):
    """w_l * M_l(g, g) on one level."""
    aL = np.sum(ld["PhiL"] ** 2, axis=0)
    aN = np.sum(ld["PhiN"] ** 2, axis=0)
    return ld["w"] * aL * (aL + 2.0 * aN)


def select_points(levels, nip, tol=0.0, tie_rel=1e-9, tie_abs=1e-13, cand=None):
    """Greedy pivoted Cholesky over (+)_l w_l M_l (Eq. 2; readings R2, R3).

    At step k: d_max = max residual; p = smallest (level, g) with
    d(p) >= d_max - max(tie_rel d_max, tie_abs d_0) and d(p) > 0; new factor column on
    p's level  L[:, k] = (w M[:, p] - L[:, :k] L[p, :k]^T) / sqrt(d_p) with
    L[p, k] = sqrt(d_p); d -= L[:, k]^2; d(p) = 0.  Stops after ``nip``
    pivots or when d_max < tol * d_0.  ``cand`` optionally restricts the
    candidate points: a list of pivot codes (level << 40 | g).
    Returns pivot codes, pivot values d_k and the per-level factor columns.
    """
    nlev = len(levels)
    d = [initial_diagonal(ld) for ld in levels]
    active = [np.ones(di.shape[0], dtype=bool) for di in d]
    if cand is not None:
        active = [np.zeros(di.shape[0], dtype=bool) for di in d]
        for c in np.asarray(cand, dtype=np.int64):
            active[int(c >> PIVOT_SHIFT)][int(c & ((1 << PIVOT_SHIFT) - 1))] = True
    for lev in range(nlev):
        d[lev] = np.where(active[lev], d[lev], 0.0)
    # factor columns of each level, stored [g, column] with growing capacity
    fac = [np.zeros((di.shape[0], min(64, nip))) for di in d]
    nk = [0] * nlev
    pivots, dvals = [], []
    d0 = None
    for _k in range(nip):
        dmax = max(float(np.max(di)) if di.size else 0.0 for di in d)
        if d0 is None:
            d0 = dmax
        if dmax <= 0.0 or dmax < tol * d0:
            break
        thr = dmax - max(tie_rel * dmax, tie_abs * d0)
        lev, p = None, None
        for l in range(nlev):
            hit = np.flatnonzero((d[l] >= thr) & (d[l] > 0.0))
            if hit.size:
                lev, p = l, int(hit[0])
                break
        dp = float(d[lev][p])
        ld = levels[lev]
        mcol = ld["w"] * m_columns(ld, [p])[:, 0]
        kl = nk[lev]
        if kl:
            Lprev = fac[lev][:, :kl]
            mcol = mcol - Lprev @ Lprev[p, :]
        col = mcol / math.sqrt(dp)
        col[p] = math.sqrt(dp)
        col = np.where(active[lev], col, 0.0) if cand is not None else col
        d[lev] = d[lev] - col * col
        d[lev][p] = 0.0
        if kl == fac[lev].shape[1]:
            grown = np.zeros((fac[lev].shape[0], min(2 * kl, nip)))
            grown[:, :kl] = fac[lev]
            fac[lev] = grown
        fac[lev][:, kl] = col
        nk[lev] = kl + 1
        pivots.append((lev << PIVOT_SHIFT) | p)
        dvals.append(dp)
    return {
        "pivots": np.array(pivots, dtype=np.int64),
        "dvals": np.array(dvals),
        "factor": [fac[l][:, :nk[l]] for l in range(nlev)],
        "residual": d,
    }


# ---------------------------------------------------------------------------
# Least-squares fit of the interpolation vectors (Section II.A, Eq. 3; R4)
# ---------------------------------------------------------------------------


def split_pivots(pivots, nlev):
    pivots = np.asarray(pivots, dtype=np.int64)
    lev = pivots >> PIVOT_SHIFT
    g = pivots & ((1 << PIVOT_SHIFT) - 1)
    return [g[lev == l] for l in range(nlev)]


def fit(levels, pivots, reg_rel=1e-14, col_batch=None):
    """Xi_l = (ZC^T)_l (CC^T + lambda I)^-1 on every level (Eq. 3).

    With Z the pair densities of level l (pairs x grid) and C = Z[:, P], the
    normal equations of min || Z - C Xi^T || give (ZC^T)_l = M_l[:, P] and
    (CC^T)_l = M_l[P, P].  Solved with an FP64 Cholesky (LAPACK).
    ``col_batch`` only bounds memory: the columns of (ZC^T)_l are formed that
    many at a time, each by the same expression as all at once.
    """
    out = []
    for ld, P in zip(levels, split_pivots(pivots, len(levels))):
        if P.size == 0:
            out.append(np.zeros((ld["PhiL"].shape[1], 0)))
            continue
        if col_batch is None or P.size <= col_batch:
            ZCt = m_columns(ld, P)
        else:
            ZCt = np.empty((ld["PhiL"].shape[1], P.size))
            for c0 in range(0, P.size, col_batch):
                ZCt[:, c0:c0 + col_batch] = m_columns(ld, P[c0:c0 + col_batch])
        CCt = ZCt[P, :]
        lam = reg_rel * np.trace(CCt) / P.size
        cf = scipy.linalg.cho_factor(CCt + lam * np.eye(P.size), lower=True)
        out.append(scipy.linalg.cho_solve(cf, ZCt.T).T)
    return out


# ---------------------------------------------------------------------------
# Coulomb matrix (xi|xi') by FFT (Section II, Eq. 1; Section III; reading R5)
# ---------------------------------------------------------------------------


def fourier_coeffs(cols, grid):
    """f~(m) = (1/N_g) sum_g f(r_g) exp(-i G_m . r_g); array [c, mz, my, mx]."""
    nx, ny, nz = (int(v) for v in grid)
    F = np.fft.fftn(cols.T.reshape(-1, nz, ny, nx), axes=(1, 2, 3))
    return F / float(nx * ny * nz)


def _interp_coeff(F, grid, mz, my, mx):
    """Coefficient of the trigonometric interpolant at extended modes (R5)."""
    nx, ny, nz = (int(v) for v in grid)
    c = F[:, mz % nz][:, :, my % ny][:, :, :, mx % nx]
    fz = np.where(np.abs(mz) * 2 == nz, 0.5, 1.0)
    fy = np.where(np.abs(my) * 2 == ny, 0.5, 1.0)
    fx = np.where(np.abs(mx) * 2 == nx, 0.5, 1.0)
    return c * (fz[:, None, None] * fy[None, :, None] * fx[None, None, :])[None]


def coulomb_pair(Fa, grid_a, Fb, grid_b, edges):
    """(f_a | f_b) for all column pairs; grid_b must be the coarser (or same).

    Sum over the extended modes m of the coarser grid, -n/2 <= m <= n/2 per
    axis, m != 0:  4 pi Omega Re[conj c_a(m) c_b(m)] / |G_m|^2.
    The sum is accumulated plane by plane in m_z (same sum, bounded memory).
    """
    nx, ny, nz = (int(v) for v in grid_b)
    omega = float(np.prod(edges))
    my = np.arange(-(ny // 2), ny // 2 + 1)
    mx = np.arange(-(nx // 2), nx // 2 + 1)
    V = np.zeros((Fa.shape[0], Fb.shape[0]))
    for mzv in range(-(nz // 2), nz // 2 + 1):
        mz = np.array([mzv])
        ca = _interp_coeff(Fa, grid_a, mz, my, mx).reshape(Fa.shape[0], -1)
        cb = _interp_coeff(Fb, grid_b, mz, my, mx).reshape(Fb.shape[0], -1)
        Gz = 2 * math.pi * mzv / edges[2]
        Gy = 2 * math.pi * my / edges[1]
        Gx = 2 * math.pi * mx / edges[0]
        G2 = (Gz * Gz + Gy[:, None] ** 2 + Gx[None, :] ** 2).ravel()
        kern = np.zeros_like(G2)
        nz_mask = G2 > 0
        kern[nz_mask] = 4.0 * math.pi * omega / G2[nz_mask]
        V += np.real(np.conj(ca) @ (cb * kern[None, :]).T)
    return V


def coulomb(system, Xi, col_batch=None):
    """V = (xi_P | xi_Q) over all levels, in global pivot order per level blocks.

    Returns the full symmetric matrix ordered level by level (level 0 pivots
    first, each level's pivots in selection order).  ``col_batch`` only bounds
    memory: the Fourier coefficients are taken that many columns at a time and
    V is filled block by block; every entry is the same sum as without it.
    """
    nlev = len(Xi)
    sizes = [x.shape[1] for x in Xi]
    off = np.concatenate([[0], np.cumsum(sizes)])
    V = np.zeros((off[-1], off[-1]))
    if col_batch is None:
        F = [fourier_coeffs(Xi[l], system["grids"][l]) for l in range(nlev)]
        for a in range(nlev):
            for b in range(a, nlev):
                if sizes[a] == 0 or sizes[b] == 0:
                    continue
                blk = coulomb_pair(F[a], system["grids"][a], F[b], system["grids"][b], system["edges"])
                V[off[a]:off[a + 1], off[b]:off[b + 1]] = blk
                V[off[b]:off[b + 1], off[a]:off[a + 1]] = blk.T
        return V
    for a in range(nlev):
        for a0 in range(0, sizes[a], col_batch):
            a1 = min(a0 + col_batch, sizes[a])
            Fa = fourier_coeffs(Xi[a][:, a0:a1], system["grids"][a])
            for b in range(a, nlev):
                for b0 in range(a0 if b == a else 0, sizes[b], col_batch):
                    b1 = min(b0 + col_batch, sizes[b])
                    Fb = Fa if (b == a and b0 == a0) else fourier_coeffs(Xi[b][:, b0:b1], system["grids"][b])
                    blk = coulomb_pair(Fa, system["grids"][a], Fb, system["grids"][b], system["edges"])
                    V[off[a] + a0:off[a] + a1, off[b] + b0:off[b] + b1] = blk
                    V[off[b] + b0:off[b] + b1, off[a] + a0:off[a] + a1] = blk.T
    return V


# ---------------------------------------------------------------------------
# Exchange matrix from the four-term multigrid THC form (Section III.A, Eq. 8)
# ---------------------------------------------------------------------------


def level_ordered(pivots, nlev):
    """Permutation that orders pivots level by level, selection order within."""
    pivots = np.asarray(pivots, dtype=np.int64)
    lev = pivots >> PIVOT_SHIFT
    return np.concatenate([np.flatnonzero(lev == l) for l in range(nlev)]).astype(np.int64)


def pivot_factors(system, funcs, pivots):
    """X^L and X^N (N x N_ip, level-ordered pivot columns), reading R6."""
    nlev = len(system["grids"])
    per = split_pivots(pivots, nlev)
    nfun = funcs["level"].shape[0]
    XL = np.zeros((nfun, sum(p.size for p in per)))
    XN = np.zeros_like(XL)
    c0 = 0
    for lev in range(nlev):
        P = per[lev]
        if P.size == 0:
            continue
        L, N, _ = level_sets(funcs, lev)
        XL[L, c0:c0 + P.size] = basis_on_level(system, funcs, L, lev)[:, P]
        XN[N, c0:c0 + P.size] = basis_on_level(system, funcs, N, lev)[:, P]
        c0 += P.size
    return XL, XN


def exchange(XL, XN, V, C):
    """K_{mu nu} = sum_{lam sig} D_{lam sig} (mu lam|sig nu), D = C C^T (Eq. 8, R6).

    With c(P) the N x N matrix c_{mu lam}(P), E(P) = c(P) C and
    K = sum_PQ V_PQ c(P) D c(Q) = sum_P E(P) (sum_Q V_PQ E(Q))^T.
    E_x = -Tr(D K).
    """
    XG = XL + XN
    yG = C.T @ XG  # (n, nip): y_G(P) = C^T x_G(P)
    yL = C.T @ XL
    # E[P, mu, i] = XL[mu,P] yG[i,P] + XN[mu,P] yL[i,P]
    E = XL.T[:, :, None] * yG.T[:, None, :] + XN.T[:, :, None] * yL.T[:, None, :]
    Fv = np.tensordot(V, E, axes=(1, 0))  # sum_Q V_PQ E(Q)
    K = np.einsum("pmi,pni->mn", E, Fv)
    D = C @ C.T
    Ex = -float(np.sum(D * K))
    return K, Ex


# ---------------------------------------------------------------------------
# The coarsest level as the paper's sparse universal grid (Section III and
# III.A: every point of the universal grid U is an ISDF point, its fitting
# function the grid's sinc function, so the pair densities of that grid are
# represented exactly; (R_U|R_U') is only ever applied)
# ---------------------------------------------------------------------------


def coarse_points(system):
    """Pivot codes of every point of the coarsest level, in grid order."""
    lev = len(system["grids"]) - 1
    ng = int(np.prod(system["grids"][lev]))
    return (np.int64(lev) << PIVOT_SHIFT) | np.arange(ng, dtype=np.int64)


def run_sinc(system, C, nip, tol=0.0, tie_rel=1e-9, tie_abs=1e-13, reg_rel=1e-14, pivots=None):
    """Multigrid ISDF with the coarsest level as the universal sinc grid.

    The greedy selection (Eq. 2) and the least-squares fit (Eq. 3) run on the
    finer levels only (``nip`` counts their pivots).  On the coarsest level
    every grid point is an interpolation point and its interpolation vector is
    the unit vector of that point (Xi = I): a grid function is its own
    interpolant, so no fit is needed.  V (Eq. 1) and K (Eq. 8) are then the
    same definitions over all interpolation points -- fitted and coarse.
    """
    funcs = expand_functions(system)
    levels = _level_data(system, funcs)
    fine = levels[:-1]
    sel = None
    if pivots is None:
        sel = select_points(fine, nip, tol, tie_rel, tie_abs)
        pivots = sel["pivots"]
    pivots = np.asarray(pivots, dtype=np.int64)
    Xi = fit(fine, pivots, reg_rel)
    ngc = levels[-1]["PhiL"].shape[1]
    Xi.append(np.eye(ngc))
    V = coulomb(system, Xi)
    allp = np.concatenate([pivots, coarse_points(system)])
    XL, XN = pivot_factors(system, funcs, allp)
    K, Ex = exchange(XL, XN, V, C)
    return {"pivots": pivots, "dvals": None if sel is None else sel["dvals"], "all_pivots": allp,
            "order": level_ordered(allp, len(levels)), "levels": levels, "funcs": funcs, "Xi": Xi, "V": V,
            "XL": XL, "XN": XN, "K": K, "Ex": Ex}


# ---------------------------------------------------------------------------
# Atom-centred local dense grids (Section III, Eq. 5, the local ISDF of Eq. 7
# on each atom's grid, Fig. Grids; readings R10-R12)
# ---------------------------------------------------------------------------

LOCAL_ATOM_SHIFT = 24  # local pivot code on level 0: (atom << 24) | box index


def local_radius(alpha_min, eps_r):
    """r_max = sqrt(-ln(eps_r) / alpha_min) (Eq. 5): beyond it a Gaussian of
    exponent >= alpha_min has fallen below eps_r."""
    return math.sqrt(-math.log(eps_r) / alpha_min)


def local_grid(system, atom, r_max):
    """The finest grid's points around one atom (reading R10).

    Box: per axis the centre index c = floor(x / h + 1/2) and the half-width
    r = floor(r_max / h) + 1, so every grid point within r_max of the atom is
    inside; the box's points (i, j, k), i fastest, sit at the unwrapped
    positions (c - r + i) h and map to the parent index (c - r + i) mod n.
    Returns (box dims, parent index of every box point, sphere mask)."""
    n = [int(v) for v in system["grids"][0]]
    E = system["edges"]
    x = system["xyz"][atom]
    h = [E[a] / n[a] for a in range(3)]
    c = [int(math.floor(x[a] / h[a] + 0.5)) for a in range(3)]
    r = [int(math.floor(r_max / h[a])) + 1 for a in range(3)]
    B = [2 * r[a] + 1 for a in range(3)]
    if any(B[a] > n[a] for a in range(3)):
        raise ValueError("local grid wider than the cell")
    ax = [np.arange(B[a]) + c[a] - r[a] for a in range(3)]
    K, J, I = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")  # box order: i fastest
    d2 = (I * h[0] - x[0]) ** 2 + (J * h[1] - x[1]) ** 2 + (K * h[2] - x[2]) ** 2
    parent = np.mod(I, n[0]) + n[0] * (np.mod(J, n[1]) + n[1] * np.mod(K, n[2]))
    return B, parent.ravel().astype(np.int64), (d2 <= r_max * r_max).ravel()


def local_sets(funcs, atom):
    """(L_A, N_A) of one atom's grid (reading R11): L_A the finest-level
    functions of the atom; N_A the finest-level functions of atoms with a
    larger index and every function of the coarser levels."""
    fl, fa = funcs["level"], funcs["atom"]
    L = np.flatnonzero((fl == 0) & (fa == atom))
    N = np.flatnonzero(((fl == 0) & (fa > atom)) | (fl > 0))
    return L, N


def local_blocks(system, funcs, eps_r):
    """Per atom the block data of its local grid: the sphere's points (box
    order), their parent indices, Phi_L and Phi_N there, w = dV of the finest
    grid.  alpha_min is the finest level's edge (every function of level 0 has
    alpha >= alpha_min)."""
    r_max = local_radius(float(system["level_min_exp"][0]), eps_r)
    nfun = funcs["level"].shape[0]
    Phi0 = basis_on_level(system, funcs, np.arange(nfun), 0)
    out = []
    for A in range(system["xyz"].shape[0]):
        B, parent, inside = local_grid(system, A, r_max)
        L, N = local_sets(funcs, A)
        pts = parent[inside]
        out.append({"L": L, "N": N, "PhiL": Phi0[L][:, pts], "PhiN": Phi0[N][:, pts], "w": level_weight(system, 0),
                    "box": B, "box_index": np.flatnonzero(inside).astype(np.int64), "parent": pts})
    return out, r_max


def run_local(system, C, nip, tol=0.0, local_tol=1e-8, local_cap=64, eps_r=1e-5, sinc=False, tie_rel=1e-9,
              tie_abs=1e-13, reg_rel=1e-14):
    """Multigrid ISDF with the finest level on atom-centred local grids.

    Per atom (reading R12): the greedy pivoted Cholesky of Eq. 2 on its own
    block w M_A over the sphere's points, at most ``local_cap`` pivots,
    stopping once the largest residual is below ``local_tol`` times the atom's
    largest initial residual; the least-squares fit of Eq. 3 on the block.
    The coarser levels are selected together by the usual greedy (``nip``
    pivots, ``tol``) and fitted as usual; with ``sinc`` the coarsest of them
    is the universal sinc grid (Xi = I, see run_sinc).  The local xi_A are
    zero off their sphere; placed on the finest full grid they enter the
    Coulomb matrix of Eq. 1 like any finest-level vector, and K follows from
    Eq. 8 with X^L_{mu P} = phi_mu(P) for mu in L_A and X^N for mu in N_A.
    Pivot codes: (atom << 24) | box index on level 0, then (level << 40) | g.
    """
    funcs = expand_functions(system)
    nlev = len(system["grids"])
    blocks, r_max = local_blocks(system, funcs, eps_r)
    levels = _level_data(system, funcs)
    hi = nlev - 1 if sinc else nlev
    # local selections and fits, atom by atom
    loc_codes, loc_dv, Xi0_cols, XL_cols, XN_cols = [], [], [], [], []
    nfun = funcs["level"].shape[0]
    ng0 = int(np.prod(system["grids"][0]))
    Phi0 = basis_on_level(system, funcs, np.arange(nfun), 0)
    for A, blk in enumerate(blocks):
        sel = select_points([blk], local_cap, local_tol, tie_rel, tie_abs)
        P = sel["pivots"] & ((1 << PIVOT_SHIFT) - 1)  # indices into the sphere's points
        loc_codes += [(A << LOCAL_ATOM_SHIFT) | int(blk["box_index"][i]) for i in P]
        loc_dv += list(sel["dvals"])
        Xi_A = fit([blk], P, reg_rel)[0]
        emb = np.zeros((ng0, P.size))
        emb[blk["parent"], :] = Xi_A
        Xi0_cols.append(emb)
        g = blk["parent"][P]
        xl = np.zeros((nfun, P.size))
        xn = np.zeros((nfun, P.size))
        xl[blk["L"]] = Phi0[blk["L"]][:, g]
        xn[blk["N"]] = Phi0[blk["N"]][:, g]
        XL_cols.append(xl)
        XN_cols.append(xn)
    # the full-cell levels
    main = levels[1:hi]
    sel = select_points(main, nip, tol, tie_rel, tie_abs)
    mp = sel["pivots"]
    main_codes = ((mp >> PIVOT_SHIFT) + 1) << PIVOT_SHIFT | (mp & ((1 << PIVOT_SHIFT) - 1))
    Xi = [np.concatenate(Xi0_cols, axis=1)] + fit(main, mp, reg_rel)
    per = split_pivots(main_codes, nlev)
    if sinc:
        Xi.append(np.eye(int(np.prod(system["grids"][-1]))))
        per[-1] = np.arange(int(np.prod(system["grids"][-1])), dtype=np.int64)
    V = coulomb(system, Xi)
    XL = [np.concatenate(XL_cols, axis=1)]
    XN = [np.concatenate(XN_cols, axis=1)]
    for lev in range(1, nlev):
        P = per[lev]
        L, N, _ = level_sets(funcs, lev)
        xl = np.zeros((nfun, P.size))
        xn = np.zeros((nfun, P.size))
        if P.size:
            xl[L] = basis_on_level(system, funcs, L, lev)[:, P]
            xn[N] = basis_on_level(system, funcs, N, lev)[:, P]
        XL.append(xl)
        XN.append(xn)
    XL = np.concatenate(XL, axis=1)
    XN = np.concatenate(XN, axis=1)
    K, Ex = exchange(XL, XN, V, C)
    return {"local_pivots": np.array(loc_codes, dtype=np.int64), "local_dvals": np.array(loc_dv),
            "pivots": main_codes, "dvals": sel["dvals"], "blocks": blocks, "r_max": r_max, "funcs": funcs,
            "Xi": Xi, "V": V, "XL": XL, "XN": XN, "K": K, "Ex": Ex}


# ---------------------------------------------------------------------------
# Whole path
# ---------------------------------------------------------------------------


def run(system, C, nip, tol=0.0, tie_rel=1e-9, tie_abs=1e-13, reg_rel=1e-14, pivots=None, cand=None):
    """Selection -> fit -> Coulomb -> exchange, all FP64 on the CPU.

    If ``pivots`` is given the selection is skipped and those pivots are fitted
    (used to check the later steps on their own).
    """
    funcs = expand_functions(system)
    levels = _level_data(system, funcs)
    sel = None
    if pivots is None:
        sel = select_points(levels, nip, tol, tie_rel, tie_abs, cand)
        pivots = sel["pivots"]
    pivots = np.asarray(pivots, dtype=np.int64)
    Xi = fit(levels, pivots, reg_rel)
    V = coulomb(system, Xi)
    order = level_ordered(pivots, len(levels))
    XL, XN = pivot_factors(system, funcs, pivots)
    K, Ex = exchange(XL, XN, V, C)
    return {
        "pivots": pivots,
        "dvals": None if sel is None else sel["dvals"],
        "sel": sel,
        "levels": levels,
        "funcs": funcs,
        "Xi": Xi,
        "V": V,
        "order": order,
        "XL": XL,
        "XN": XN,
        "K": K,
        "Ex": Ex,
    }
