"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to the paper's definitions or to
mathematics: closed forms (Poisson summation, analytic Gaussian Coulomb
series), textbook routines (pivoted QR / LAPACK dpstrf, least squares),
brute force (the 4-index tensor), exact reproduction at full pair rank, and
invariants (symmetry, PSD, monotone fall, interpolation identity).
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import isdf as O
from paper_2404_09373_gb300 import systems as S

ONE_ATOM = np.array([[0.11, 0.23, 0.31]])
TWO_ATOMS = np.array([[0.1, 0.2, 0.3], [0.55, 0.6, 0.7]])


def tiny(levels=1, n=(16, 8, 4), sites=ONE_ATOM, a=4.0, tol=1e-10):
    grids = tuple((m, m, m) for m in n[:levels])
    edges = (1.6, 0.4)[: levels - 1]
    return S.make_system((1, 1, 1), 0.0, None, grids, edges, a=a, sites=sites, image_tol=tol)


def orbitals(sysd, n_occ=2, seed=1):
    return S.make_orbitals(sysd, n_occ, np.random.default_rng(seed))


# --------------------------------------------------------------------------- basis


def test_basis_separable_equals_direct_image_sum():
    sysd = tiny(sites=TWO_ATOMS, n=(10,), a=4.5)
    f = O.expand_functions(sysd)
    idx = np.arange(f["level"].size)
    a = O.basis_on_level(sysd, f, idx, 0)
    b = O.basis_direct(sysd, f, idx, 0)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


@pytest.mark.parametrize("alpha,lx", [(0.1, 0), (1.6, 0), (6.4, 0), (0.6, 1), (2.4, 1)])
def test_basis_matches_poisson_summation(alpha, lx):
    """Image sum of exp(-a|r-A|^2) (and x times it) equals its Fourier series
    (1/Omega)(pi/a)^{3/2} sum_G exp(-G^2/4a) cos G.(r-A)  (s),
    (1/Omega)(pi/a)^{3/2} sum_G (G_x/2a) exp(-G^2/4a) sin G.(r-A)  (p_x)."""
    L = 5.0
    sysd = S.make_system((1, 1, 1), 0.0, None, ((6, 6, 6),), (), a=L, sites=ONE_ATOM,
                         s_exps=(alpha,) if lx == 0 else (), p_exps=(alpha,) if lx == 1 else (), image_tol=1e-16)
    f = O.expand_functions(sysd)
    phi = O.basis_on_level(sysd, f, [0], 0)[0] / f["norm"][0]
    xs = O.grid_points_1d(sysd, 0)
    A = sysd["xyz"][0]
    mmax = int(math.ceil(math.sqrt(4 * alpha * 40) * L / (2 * math.pi))) + 1
    m = np.arange(-mmax, mmax + 1)
    Gx = 2 * math.pi * m / L
    # separable series: product of 1-D series (cell is cubic)
    def series_1d(x, A0, deriv):
        ph = np.outer(x - A0, Gx)
        w = np.exp(-Gx ** 2 / (4 * alpha)) * math.sqrt(math.pi / alpha) / L
        if deriv:
            return (np.sin(ph) * (Gx / (2 * alpha)) * w).sum(axis=1)
        return (np.cos(ph) * w).sum(axis=1)
    fx = series_1d(xs[0], A[0], lx == 1)
    fy = series_1d(xs[1], A[1], False)
    fz = series_1d(xs[2], A[2], False)
    ref = np.einsum("k,j,i->kji", fz, fy, fx).ravel()
    assert np.max(np.abs(phi - ref)) <= 1e-12 * np.max(np.abs(ref))


# --------------------------------------------------------------------------- Coulomb


def _gauss_coeff_exact(alpha, A, L, m):
    G = [2 * math.pi * mi / L for mi in m]
    G2 = sum(g * g for g in G)
    return (math.pi / alpha) ** 1.5 / L ** 3 * math.exp(-G2 / (4 * alpha)) * np.exp(-1j * sum(g * a for g, a in zip(G, A))), G2


def _analytic_coulomb(alpha, A, beta, B, L, mmax=20):
    tot = 0.0
    rng = range(-mmax, mmax + 1)
    for mx in rng:
        for my in rng:
            for mz in rng:
                if mx == my == mz == 0:
                    continue
                fa, G2 = _gauss_coeff_exact(alpha, A, L, (mx, my, mz))
                fb, _ = _gauss_coeff_exact(beta, B, L, (mx, my, mz))
                tot += (np.conj(fa) * fb).real / G2
    return 4 * math.pi * L ** 3 * tot


def _periodic_gauss_on_grid(alpha, A, L, n):
    sysd = S.make_system((1, 1, 1), 0.0, None, ((n, n, n),), (), a=L, sites=np.array([A]) / L,
                         s_exps=(alpha,), p_exps=(), image_tol=1e-16)
    f = O.expand_functions(sysd)
    return O.basis_on_level(sysd, f, [0], 0)[0] / f["norm"][0]


@pytest.mark.parametrize("na,nb", [(32, 32), (32, 16), (16, 16)])
def test_coulomb_fft_matches_analytic_gaussian_series(na, nb):
    """(f|g) by FFT on one or two grid levels equals the analytic series
    4 pi Omega sum_{G != 0} Re[conj f~(G) g~(G)] / G^2 for resolved Gaussians."""
    L = 7.0
    A = np.array([1.0, 2.0, 2.5])
    B = np.array([4.0, 3.5, 5.0])
    alpha, beta = 0.45, 0.3
    fa = _periodic_gauss_on_grid(alpha, A, L, na)
    fb = _periodic_gauss_on_grid(beta, B, L, nb)
    Fa = O.fourier_coeffs(fa[:, None], (na, na, na))
    Fb = O.fourier_coeffs(fb[:, None], (nb, nb, nb))
    got = O.coulomb_pair(Fa, (na, na, na), Fb, (nb, nb, nb), np.array([L, L, L]))[0, 0]
    ref = _analytic_coulomb(alpha, A, beta, B, L)
    assert abs(got - ref) <= 1e-10 * abs(ref)


def test_coulomb_cross_level_equals_fine_level_for_bandlimited():
    """Cross-level (xi|xi') equals the same integral with the coarse function
    resampled (trigonometrically) on the fine grid: reading R5."""
    L = 6.0
    rng = np.random.default_rng(3)
    nc, nf = 8, 16
    f_c = rng.standard_normal(nc ** 3)
    g_f = rng.standard_normal(nf ** 3)
    Fc = O.fourier_coeffs(f_c[:, None], (nc, nc, nc))
    Ff = O.fourier_coeffs(g_f[:, None], (nf, nf, nf))
    cross = O.coulomb_pair(Ff, (nf,) * 3, Fc, (nc,) * 3, np.array([L] * 3))[0, 0]
    # interpolate f_c onto the fine grid by zero padding with split Nyquist
    full = np.zeros((nf, nf, nf), dtype=complex)
    for mz in range(-nc // 2, nc // 2 + 1):
        for my in range(-nc // 2, nc // 2 + 1):
            for mx in range(-nc // 2, nc // 2 + 1):
                w = 1.0
                for mm in (mx, my, mz):
                    if abs(mm) * 2 == nc:
                        w *= 0.5
                full[mz % nf, my % nf, mx % nf] += w * Fc[0, mz % nc, my % nc, mx % nc]
    f_interp = np.fft.ifftn(full * nf ** 3)
    assert np.max(np.abs(f_interp.imag)) < 1e-12
    F_int = O.fourier_coeffs(f_interp.real.ravel()[:, None], (nf,) * 3)
    same = O.coulomb_pair(Ff, (nf,) * 3, F_int, (nf,) * 3, np.array([L] * 3))[0, 0]
    # the interpolant has no mode at the fine Nyquist, so the same-level rule
    # on the fine grid is the plain sum: both must agree
    assert abs(cross - same) <= 1e-12 * max(1.0, abs(same))


# --------------------------------------------------------------------------- selection


def _pair_matrix(levels, lev):
    """Explicit Z (ordered pairs x grid points) of one level, reading R1."""
    ld = levels[lev]
    rows = [ld["PhiL"][i] * ld["PhiL"][j] for i in range(ld["PhiL"].shape[0]) for j in range(ld["PhiL"].shape[0])]
    rows += [ld["PhiL"][i] * ld["PhiN"][j] for i in range(ld["PhiL"].shape[0]) for j in range(ld["PhiN"].shape[0])]
    rows += [ld["PhiN"][j] * ld["PhiL"][i] for i in range(ld["PhiL"].shape[0]) for j in range(ld["PhiN"].shape[0])]
    return np.array(rows)


def _levels(sysd):
    f = O.expand_functions(sysd)
    return f, O._level_data(sysd, f)


def test_m_matches_explicit_pair_gram():
    """M_l = Z_l^T Z_l for the ordered pair set of each level (Eq. 2, R1)."""
    sysd = tiny(levels=3, sites=TWO_ATOMS, n=(8, 4, 2), a=4.0)
    _, levels = _levels(sysd)
    for lev in range(3):
        Z = _pair_matrix(levels, lev)
        ng = levels[lev]["PhiL"].shape[1]
        M = O.m_columns(levels[lev], np.arange(ng))
        assert np.max(np.abs(M - Z.T @ Z)) <= 1e-12 * np.max(np.abs(M))


def test_selection_matches_pivoted_qr_and_dpstrf():
    """Single level: pivoted Cholesky on M picks the same points as pivoted QR
    on the pair matrix (Section II.A) and as LAPACK dpstrf on M."""
    sysd = S.make_system((1, 1, 1), 0.04, np.random.default_rng(11), ((10, 10, 10),), (), a=5.0,
                         sites=TWO_ATOMS, s_exps=(0.3, 1.2), p_exps=(0.8,))
    _, levels = _levels(sysd)
    k = 30
    sel = O.select_points(levels, k, tie_rel=0.0, tie_abs=0.0)
    piv = sel["pivots"] & ((1 << O.PIVOT_SHIFT) - 1)
    Z = _pair_matrix(levels, 0)
    _, _, qr_piv = scipy.linalg.qr(Z, pivoting=True, mode="economic")
    np.testing.assert_array_equal(piv, qr_piv[:k])
    M = levels[0]["w"] * O.m_columns(levels[0], np.arange(Z.shape[1]))
    _, lp, rank, info = scipy.linalg.lapack.dpstrf(M, lower=1, tol=-1.0)
    np.testing.assert_array_equal(piv, (lp - 1)[:k])


def test_selection_tie_rule_smallest_index():
    """Undisplaced symmetric cell: exact ties resolve to the smallest (level, g)."""
    sysd = S.make_system((1, 1, 1), 0.0, None, ((8, 8, 8),), (), a=6.74)
    _, levels = _levels(sysd)
    d = O.initial_diagonal(levels[0])
    dmax = d.max()
    ties = np.flatnonzero(d >= dmax - 1e-9 * dmax)
    assert ties.size > 1  # the symmetric cell really has ties
    sel = O.select_points(levels, 1)
    assert int(sel["pivots"][0]) == int(ties[0])


def test_residual_trace_equals_fit_error():
    """Sum_g d_k(g) = sum_l w_l ||Z_l - C_l Xi_l^T||_F^2 (Schur complement)."""
    sysd = tiny(levels=3, sites=TWO_ATOMS, n=(8, 4, 2), a=4.0)
    _, levels = _levels(sysd)
    sel = O.select_points(levels, 40)
    Xi = O.fit(levels, sel["pivots"], reg_rel=0.0)
    per = O.split_pivots(sel["pivots"], 3)
    err = 0.0
    for lev in range(3):
        Z = _pair_matrix(levels, lev)
        if per[lev].size:
            R = Z - Z[:, per[lev]] @ Xi[lev].T
        else:
            R = Z
        err += levels[lev]["w"] * np.sum(R * R)
    tr = sum(float(np.sum(r)) for r in sel["residual"])
    assert abs(err - tr) <= 1e-9 * abs(err) + 1e-14


def test_fit_matches_lstsq_and_interpolates():
    """Xi = argmin ||Z - Z[:,P] Xi^T|| (Eq. 3) and Xi[P, :] = I."""
    sysd = tiny(levels=3, sites=TWO_ATOMS, n=(8, 4, 2), a=4.0)
    _, levels = _levels(sysd)
    sel = O.select_points(levels, 30)
    Xi = O.fit(levels, sel["pivots"], reg_rel=0.0)
    for lev, P in enumerate(O.split_pivots(sel["pivots"], 3)):
        if P.size == 0:
            continue
        Z = _pair_matrix(levels, lev)
        ref = np.linalg.lstsq(Z[:, P], Z, rcond=None)[0].T
        assert np.max(np.abs(Xi[lev] - ref)) <= 1e-8 * max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(Xi[lev][P, :] - np.eye(P.size))) <= 1e-10


def test_selection_nested_and_residual_monotone():
    sysd = tiny(levels=3, sites=TWO_ATOMS, n=(8, 4, 2), a=4.0)
    _, levels = _levels(sysd)
    prev = None
    traces = []
    for k in (5, 10, 20, 40):
        sel = O.select_points(levels, k)
        if prev is not None:
            np.testing.assert_array_equal(sel["pivots"][: prev.size], prev)
        prev = sel["pivots"]
        traces.append(sum(float(np.sum(r)) for r in sel["residual"]))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(traces, traces[1:]))


# --------------------------------------------------------------------------- exchange


@pytest.mark.parametrize("levels", [1, 3])
def test_nofit_equals_brute_4index(levels):
    sysd = tiny(levels=levels, n=(12, 6, 4))
    C = orbitals(sysd)
    Kn, En = oracle.nofit_exchange(sysd, C)
    Kb, Eb, eri = oracle.brute_exchange(sysd, C)
    assert np.max(np.abs(Kn - Kb)) <= 1e-13 * np.max(np.abs(Kb))
    # ERI symmetries of the exact tensor
    assert np.max(np.abs(eri - eri.transpose(1, 0, 2, 3))) <= 1e-13 * np.max(np.abs(eri))
    assert np.max(np.abs(eri - eri.transpose(2, 3, 0, 1))) <= 1e-13 * np.max(np.abs(eri))


@pytest.mark.parametrize("levels,rank", [(1, 91), (3, 91)])
def test_isdf_exact_at_full_pair_rank(levels, rank):
    """With N_ip at the pair-space rank ISDF reproduces the no-fit exchange."""
    sysd = tiny(levels=levels)
    C = orbitals(sysd)
    Kn, En = oracle.nofit_exchange(sysd, C)
    r = oracle.run(sysd, C, 200, tol=1e-14, reg_rel=0.0)
    assert len(r["pivots"]) == rank
    assert np.max(np.abs(r["K"] - Kn)) <= 1e-9
    assert abs(r["Ex"] - En) <= 1e-9


def test_isdf_eri_four_term_form():
    """exchange() contracts the Eq. 8 tensor: build (mu lam|sig nu) explicitly
    from c(P) V c(Q), check its pair symmetries and K = D-contraction."""
    sysd = tiny(levels=3)
    C = orbitals(sysd)
    r = oracle.run(sysd, C, 40)
    XL, XN = r["XL"], r["XN"]
    XG = XL + XN
    c = np.einsum("mp,lp->pml", XL, XG) + np.einsum("mp,lp->pml", XN, XL)
    eri = np.einsum("pml,pq,qsn->mlsn", c, r["V"], c)
    assert np.max(np.abs(eri - eri.transpose(1, 0, 2, 3))) <= 1e-12 * np.max(np.abs(eri))
    assert np.max(np.abs(eri - eri.transpose(2, 3, 0, 1))) <= 1e-12 * np.max(np.abs(eri))
    D = C @ C.T
    K = np.einsum("ls,mlsn->mn", D, eri)
    assert np.max(np.abs(K - r["K"])) <= 1e-12 * np.max(np.abs(K))


def test_invariants_symmetry_psd_sign():
    sysd, C = S.small_multigrid(per_cell=(12, 6, 4), seed=5)
    r = oracle.run(sysd, C, 120)
    K, V = r["K"], r["V"]
    assert np.max(np.abs(K - K.T)) <= 1e-13 * np.max(np.abs(K))
    assert np.max(np.abs(V - V.T)) <= 1e-13 * np.max(np.abs(V))
    ev = np.linalg.eigvalsh(V)
    assert ev.min() >= -1e-10 * ev.max()
    assert r["Ex"] < 0.0


def test_error_falls_with_nip():
    """|K - K_nofit| falls along N_ip = N, 2N, 4N, 8N (with slack)."""
    sysd = tiny(levels=3, n=(12, 6, 4))
    C = orbitals(sysd)
    Kn, _ = oracle.nofit_exchange(sysd, C)
    N = 13
    errs = [np.max(np.abs(oracle.run(sysd, C, k)["K"] - Kn)) for k in (N, 2 * N, 4 * N, 7 * N)]
    assert errs[-1] < 1e-6
    for a, b in zip(errs, errs[1:]):
        assert b <= 1.5 * a


# --------------------------------------------------------------------------- planted mistakes


def test_planted_mistake_in_m_breaks_exact_reproduction(monkeypatch):
    """Dropping the factor 2 of the cross term in M (reading R1) changes the
    pivots and breaks exact reproduction: the pins above would catch it."""
    sysd = tiny(levels=3)
    C = orbitals(sysd)
    Kn, _ = oracle.nofit_exchange(sysd, C)

    def wrong(ld, cols):
        AL = ld["PhiL"].T @ ld["PhiL"][:, cols]
        AN = ld["PhiN"].T @ ld["PhiN"][:, cols]
        return AL * (AL + AN)

    monkeypatch.setattr(O, "m_columns", wrong)
    try:
        r = oracle.run(sysd, C, 200, tol=1e-14, reg_rel=0.0)
    except np.linalg.LinAlgError:
        return  # the wrong M is not even a Gram matrix: its Cholesky breaks down
    assert np.max(np.abs(r["K"] - Kn)) > 1e-6


def test_planted_mistake_in_eq8_breaks_brute_agreement(monkeypatch):
    """Using X^G on both factors (dropping the L/N bookkeeping of Eq. 8)
    double counts diffuse pairs and no longer matches the exact exchange."""
    sysd = tiny(levels=3)
    C = orbitals(sysd)
    Kn, _ = oracle.nofit_exchange(sysd, C)
    orig = O.exchange

    def wrong(XL, XN, V, C_):
        return orig(XL + XN, XN, V, C_)

    monkeypatch.setattr(O, "exchange", wrong)
    r = oracle.run(sysd, C, 200, tol=1e-14, reg_rel=0.0)
    assert np.max(np.abs(r["K"] - Kn)) > 1e-6


# --------------------------------------------------------------------------- learned proposer network


def test_mlp_gradient_matches_finite_differences():
    from oracle import mlp

    rng = np.random.default_rng(0)
    theta = mlp.init_params(rng)
    X = rng.standard_normal((40, mlp.N_IN))
    y = (rng.random(40) < 0.2).astype(float)
    w = np.where(y > 0, 4.0, 1.0)
    L, g = mlp.loss_and_grad(theta, X, y, w)
    h = 1e-6
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss_and_grad(theta + e, X, y, w)[0] - mlp.loss_and_grad(theta - e, X, y, w)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd))


def test_mlp_closed_form_with_zero_hidden_weights():
    """With W1 = W2 = 0 and biases b1 = b2 = 1, every hidden unit is 1, so
    z = sum(W3) + b3 for every sample: dL/db3 = sum_i w_i (p - y_i) / sum w."""
    from oracle import mlp

    P = {"W1": np.zeros((8, 64)), "b1": np.ones(64), "W2": np.zeros((64, 64)), "b2": np.ones(64),
         "W3": np.full(64, 0.01), "b3": np.array([-0.3])}
    theta = mlp.pack(P)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((10, 8))
    y = np.array([1, 0, 0, 1, 0, 0, 0, 1, 0, 0], dtype=float)
    w = np.where(y > 0, 2.0, 1.0)
    L, g = mlp.loss_and_grad(theta, X, y, w)
    z = 0.64 - 0.3
    p = 1 / (1 + np.exp(-z))
    ref_b3 = np.sum(w * (p - y)) / np.sum(w)
    assert abs(g[-1] - ref_b3) <= 1e-14
    ref_L = -np.sum(w * (y * np.log(p) + (1 - y) * np.log(1 - p))) / np.sum(w)
    assert abs(L - ref_L) <= 1e-14


# --------------------------------------------------------------------------- normalisation, levels, Adam


def _norm_integrals(funcs_hook=None):
    """sum_g phi(r_g)^2 dV for isolated s and p Gaussians in a large cell.

    The normalisation is defined by int phi^2 dr = 1.  On a periodic grid fine
    enough that the aliased Fourier terms of phi^2 are below 1e-12 (spacing
    0.125 bohr for exponents up to 6.4) and a cell large enough that images do
    not overlap (edge 16 bohr for exponents down to 0.4), the grid sum is the
    integral to far better than 1e-10: an independent check of the factors
    (2a/pi)^(3/4) and 2 sqrt(a)."""
    sysd = S.make_system((1, 1, 1), 0.0, None, ((128, 128, 128),), (), a=16.0, sites=np.array([[0.43, 0.51, 0.47]]),
                         s_exps=(0.4, 1.6, 6.4), p_exps=(0.6, 2.4), image_tol=1e-16)
    f = O.expand_functions(sysd)
    if funcs_hook is not None:
        funcs_hook(f)
    phi = O.basis_on_level(sysd, f, np.arange(f["level"].size), 0)
    dV = 16.0 ** 3 / 128 ** 3
    return np.sum(phi * phi, axis=1) * dV


def test_basis_normalisation_is_unit_norm_on_a_fine_grid():
    ints = _norm_integrals()
    assert ints.size == 3 + 2 * 3
    assert np.max(np.abs(ints - 1.0)) <= 1e-10


def test_planted_mistake_in_p_normalisation_breaks_unit_norm():
    """Dropping the 2 of the p factor 2 sqrt(a) (a plausible slip) is caught."""

    def slip(f):
        p = np.sum(f["lvec"], axis=1) == 1
        f["norm"][p] *= 0.5

    ints = _norm_integrals(slip)
    assert np.max(np.abs(ints - 1.0)) > 0.5


# Level of each exponent of the 2x2x2 diamond workload: fine grid for
# exponents >= 1.6, mid grid for 0.4 <= a < 1.6, coarse grid below 0.4 (the
# split the workload prescribes; the paper's rule is by exponent, Section II.B).
LEVEL_TABLE = {0.1: 2, 0.15: 2, 0.4: 1, 0.6: 1, 1.6: 0, 2.4: 0, 6.4: 0}


def _levels_of(level_fn):
    sysd = S.make_system((1, 1, 1), 0.0, None, ((8, 8, 8), (4, 4, 4), (2, 2, 2)), S.LEVEL_EDGES_3)
    f = level_fn(sysd)
    return {float(a): int(l) for a, l in zip(f["alpha"], f["level"])}


def test_level_rule_matches_the_exponent_table_including_edges():
    assert _levels_of(O.expand_functions) == LEVEL_TABLE
    # the L / N / G sets of the 2x2x2 workload: |L| = 320 / 256 / 256, |G| = 832 / 512 / 256
    sysd = S.make_system((2, 2, 2), 0.0, None, ((8, 8, 8), (4, 4, 4), (2, 2, 2)), S.LEVEL_EDGES_3)
    f = O.expand_functions(sysd)
    sizes = [tuple(x.size for x in O.level_sets(f, l)) for l in range(3)]
    assert sizes == [(320, 512, 832), (256, 256, 512), (256, 0, 256)]


def test_planted_mistake_in_level_edges_is_caught():
    """'a <= e' instead of 'a < e' moves the edge exponents 1.6 and 0.4 down a level."""

    def slip(sysd):
        f = O.expand_functions(sysd)
        edges = np.asarray(sysd["level_min_exp"])
        f["level"] = np.array([int(np.sum(a <= edges)) for a in f["alpha"]])
        return f

    assert _levels_of(slip) != LEVEL_TABLE


def _adam_pin_ok(step):
    """Closed forms of bias-corrected Adam (Kingma & Ba, Algorithm 1).
    (i) Constant gradient g: the corrected moments are exactly g and g^2 at
    every step, so each step moves theta by lr g / (|g| + eps).
    (ii) Gradients g1 then g2: m_hat_2 = (b1 g1 + g2) / (1 + b1) and
    v_hat_2 = (b2 g1^2 + g2^2) / (1 + b2)."""
    lr, eps, b1, b2 = 1e-2, 1e-8, 0.9, 0.999
    g = np.array([3.0, -0.5, 1e-3, -2e-6])
    th0 = np.array([0.1, -0.2, 0.3, 0.4])
    th, m, v = th0.copy(), np.zeros(4), np.zeros(4)
    ok = True
    for t in range(1, 6):
        th, m, v = step(th, m, v, g, t, lr)
        ok &= np.allclose(th, th0 - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-13)
    g1, g2 = np.array([1.0, -2.0, 0.5, 4.0]), np.array([-0.5, 1.0, 0.25, 3.0])
    th, m, v = step(th0.copy(), np.zeros(4), np.zeros(4), g1, 1, lr)
    th1 = th.copy()
    th, m, v = step(th, m, v, g2, 2, lr)
    mh = (b1 * g1 + g2) / (1 + b1)
    vh = (b2 * g1 ** 2 + g2 ** 2) / (1 + b2)
    ok &= np.allclose(th, th1 - lr * mh / (np.sqrt(vh) + eps), rtol=0, atol=1e-13)
    return bool(ok)


def test_adam_step_matches_closed_forms():
    from oracle import mlp

    assert _adam_pin_ok(mlp.adam_step)


def test_planted_mistakes_in_adam_are_caught():
    from oracle import mlp

    def no_bias_correction(theta, m, v, grad, t, lr, b1=0.9, b2=0.999, eps=1e-8):
        m = b1 * m + (1 - b1) * grad
        v = b2 * v + (1 - b2) * grad * grad
        return theta - lr * m / (np.sqrt(v) + eps), m, v

    def off_by_one(theta, m, v, grad, t, lr):
        return mlp.adam_step(theta, m, v, grad, t + 1, lr)

    def betas_swapped(theta, m, v, grad, t, lr):
        return mlp.adam_step(theta, m, v, grad, t, lr, b1=0.999, b2=0.9)

    for wrong in (no_bias_correction, off_by_one, betas_swapped):
        assert not _adam_pin_ok(wrong)


# --------------------------------------------------------------------------- threshold-driven grids (Eq. 6)


@pytest.mark.parametrize("length,alpha,eps", [(6.74, 6.4, 1e-8), (13.48, 0.6, 1e-8), (13.48, 0.15, 1e-3),
                                              (5.0, 2.4, 1e-2), (20.0, 0.1, 1e-12)])
def test_grid_for_threshold_is_the_smallest_resolving_size(length, alpha, eps):
    """By definition (Section III, Eq. 6): at the grid's largest wave number
    pi n / L the Gaussian's Fourier transform exp(-G^2 / 4 alpha) is at most
    eps_K, and at the next smaller admissible size it is not."""
    n = O.grid_for_threshold(length, alpha, eps)
    sizes = O.fft_sizes()
    assert n in sizes and n % 2 == 0
    ft = lambda m: math.exp(-((math.pi * m / length) ** 2) / (4.0 * alpha))  # noqa: E731
    assert ft(n) <= eps
    smaller = [m for m in sizes if m < n]
    if smaller:
        assert ft(smaller[-1]) > eps


def test_grid_for_threshold_worked_case():
    """a = 6.74 bohr, alpha = 6.4, eps_K = 1e-8: G_max = sqrt(4 * 6.4 * ln 1e8)
    = 21.72 bohr^-1, so n >= 6.74 * 21.72 / pi = 46.6 -> 48 (= 2^4 3)."""
    assert O.grid_for_threshold(6.74, 6.4, 1e-8) == 48
    assert O.fft_sizes()[:10] == [2, 4, 6, 8, 12, 16, 18, 24, 32, 36]


def test_level_grids_for_threshold_follow_the_sharpest_function_and_nest():
    sysd = S.make_system((2, 2, 1), 0.0, None, ((8, 8, 8), (4, 4, 4), (2, 2, 2)), S.LEVEL_EDGES_3)
    g = O.grids_for_threshold(sysd, 1e-8)
    E = sysd["edges"]
    for ax in range(3):
        assert g[0, ax] == O.grid_for_threshold(E[ax], 6.4, 1e-8)
        assert g[1, ax] == O.grid_for_threshold(E[ax], 0.6, 1e-8)
        assert g[2, ax] == O.grid_for_threshold(E[ax], 0.15, 1e-8)
        assert g[0, ax] > g[1, ax] > g[2, ax]
    # a loose threshold that gives two levels the same size: the finer one is raised
    g = O.grids_for_threshold(sysd, 0.5)
    assert np.all(g[:-1] > g[1:])


# --------------------------------------------------------------------------- coarse level as the sinc grid (Section III)


@pytest.mark.parametrize("levels,sites,a,rel", [(2, ONE_ATOM, 4.0, 1e-10), (3, ONE_ATOM, 4.0, 1e-10),
                                                (3, TWO_ATOMS, 4.5, 5e-8)])
def test_sinc_coarse_level_is_exact_at_full_rank(levels, sites, a, rel):
    """With every finer level fitted to its full pair rank and every coarse
    point an interpolation point (Xi = I), the four-term exchange reproduces
    the exact no-fit exchange: the coarse pair densities are grid functions
    of the coarse grid, represented exactly by its sinc functions.  (With two
    atoms the full-rank fit is ill-conditioned and the agreement stops near
    1e-8 relative; a wrong coarse treatment is off by orders of magnitude.)"""
    sysd = tiny(levels=levels, sites=sites, a=a)
    C = orbitals(sysd)
    Kn, En = oracle.nofit_exchange(sysd, C)
    npts = int(sum(np.prod(g) for g in sysd["grids"][:-1]))
    r = oracle.run_sinc(sysd, C, npts, tol=1e-14, reg_rel=0.0)
    assert np.max(np.abs(r["K"] - Kn)) <= rel * np.max(np.abs(Kn))
    assert abs(r["Ex"] - En) <= rel * abs(En)


def test_planted_mistake_in_the_sinc_coarse_level_is_caught(monkeypatch):
    """Xi = 2 I instead of I on the coarse level breaks the exactness pin."""
    sysd = tiny(levels=2)
    C = orbitals(sysd)
    Kn, _ = oracle.nofit_exchange(sysd, C)
    orig = np.eye
    monkeypatch.setattr(O.np, "eye", lambda n, *a, **k: 2.0 * orig(n, *a, **k))
    r = oracle.run_sinc(sysd, C, int(np.prod(sysd["grids"][0])), tol=1e-14, reg_rel=0.0)
    monkeypatch.setattr(O.np, "eye", orig)
    assert np.max(np.abs(r["K"] - Kn)) > 1e-3 * np.max(np.abs(Kn))


def test_sinc_identity_is_the_least_squares_fit_with_all_coarse_points():
    """Xi = I on the coarse level is what the fit of Eq. 3 gives when every
    coarse point is a pivot and M_c is nonsingular (a 2^3 coarse grid with
    more pair functions than points)."""
    sysd = tiny(levels=2, n=(8, 2), sites=TWO_ATOMS, a=4.5)
    funcs = O.expand_functions(sysd)
    levels = O._level_data(sysd, funcs)
    allc = oracle.coarse_points(sysd)
    Xi = O.fit(levels, allc, reg_rel=0.0)
    assert np.max(np.abs(Xi[1] - np.eye(8))) <= 1e-8


def test_sinc_coarse_coulomb_block_is_a_circulant():
    """(R_U|R_U') depends only on the difference of the two grid points
    (periodic), so it can be applied by FFT without being stored; it is PSD
    and has the constant vector (G = 0) in its null space."""
    sysd = tiny(levels=2, n=(8, 4), sites=TWO_ATOMS, a=4.5)
    C = orbitals(sysd)
    r = oracle.run_sinc(sysd, C, 20)
    k = r["pivots"].size
    Vu = r["V"][k:, k:]
    n = 4
    idx = np.arange(n ** 3)
    ijk = np.stack([idx % n, (idx // n) % n, idx // (n * n)], axis=1)
    for g in range(0, n ** 3, 7):
        for h in range(0, n ** 3, 5):
            d = (ijk[h] - ijk[g]) % n
            h0 = d[0] + n * (d[1] + n * d[2])
            assert abs(Vu[g, h] - Vu[0, h0]) <= 1e-12 * np.abs(Vu).max()
    ev = np.linalg.eigvalsh(Vu)
    assert ev.min() >= -1e-10 * ev.max()
    assert np.max(np.abs(Vu @ np.ones(n ** 3))) <= 1e-10 * np.abs(Vu).max()


# --------------------------------------------------------------------------- atom-centred local grids (Section III)


def test_local_radius_closed_form():
    """Eq. 5 at the paper's own thresholds: eps_r = 1e-5, alpha_min = 2.8
    bohr^-2 gives r_max = sqrt(ln(1e5) / 2.8) = 2.0277... bohr."""
    assert abs(O.local_radius(2.8, 1e-5) - 2.027748) <= 1e-6
    # a Gaussian of exponent alpha_min has fallen to eps_r exactly at r_max
    r = O.local_radius(1.6, 1e-3)
    assert abs(math.exp(-1.6 * r * r) - 1e-3) <= 1e-15


@pytest.mark.parametrize("a,n,atom", [(4.5, 16, 0), (4.5, 16, 1), (6.74, 24, 1)])
def test_local_grid_is_the_minimum_image_sphere(a, n, atom):
    """The box construction returns exactly the finest-grid points whose
    minimum-image distance to the atom is at most r_max (brute force over
    every point of the cell), each once."""
    sysd = tiny(levels=2, n=(n, n // 2), sites=TWO_ATOMS, a=a)
    r_max = O.local_radius(1.6, 1e-2)
    B, parent, inside = O.local_grid(sysd, atom, r_max)
    got = np.sort(parent[inside])
    assert np.unique(got).size == got.size
    h = a / n
    idx = np.arange(n ** 3)
    pos = np.stack([idx % n, (idx // n) % n, idx // (n * n)], axis=1) * h
    d = pos - sysd["xyz"][atom]
    d -= a * np.round(d / a)
    want = np.flatnonzero(np.sum(d * d, axis=1) <= r_max * r_max)
    assert np.array_equal(got, want)


CLOSE_ATOMS = np.array([[0.1, 0.2, 0.3], [0.3, 0.35, 0.45]])  # 1.3 bohr apart at a = 4.5


def _local_case(levels=2):
    sysd = tiny(levels=levels, n=(16, 8, 4), sites=CLOSE_ATOMS, a=4.5)
    return sysd, orbitals(sysd)


@pytest.mark.parametrize("levels", [2, 3])
def test_local_isdf_exact_at_full_rank(levels):
    """With every atom's local ISDF and the coarser levels at full pair rank,
    the four-term exchange reproduces the 4-index tensor of the local pair
    partition built pair by pair (brute_exchange_local).  The agreement is
    limited by the conditioning of the full-rank fits (about 1e-9 of max|K|);
    a wrong pair partition is off by 1e-3 or more (next test)."""
    sysd, C = _local_case(levels)
    Kb, Eb = oracle.brute_exchange_local(sysd, C, 1e-2)
    r = oracle.run_local(sysd, C, 400, tol=1e-14, local_tol=1e-14, local_cap=400, eps_r=1e-2, reg_rel=0.0)
    assert np.max(np.abs(r["K"] - Kb)) <= 2e-8 * np.max(np.abs(Kb))
    assert abs(r["Ex"] - Eb) <= 2e-8 * abs(Eb)


@pytest.mark.parametrize("slip", ["double", "missing"])
def test_planted_mistake_in_the_local_sets_is_caught(monkeypatch, slip):
    """N_A holding the sharp functions of every other atom (the pair counted
    on both atoms' grids) or of none (the pair dropped) breaks the pin."""
    sysd, C = _local_case(2)
    Kb, _ = oracle.brute_exchange_local(sysd, C, 1e-2)

    def wrong(funcs, atom):
        fl, fa = funcs["level"], funcs["atom"]
        L = np.flatnonzero((fl == 0) & (fa == atom))
        other = (fl == 0) & (fa != atom) if slip == "double" else np.zeros_like(fl, dtype=bool)
        return L, np.flatnonzero(other | (fl > 0))

    monkeypatch.setattr(O, "local_sets", wrong)
    r = oracle.run_local(sysd, C, 400, tol=1e-14, local_tol=1e-14, local_cap=400, eps_r=1e-2, reg_rel=1e-12)
    assert np.max(np.abs(r["K"] - Kb)) > 1e-3 * np.max(np.abs(Kb))


def test_local_partition_tends_to_the_full_cell_partition():
    """As eps_r falls the spheres take in the sharp products' tails and the
    local partition's exact exchange approaches the full-cell one."""
    sysd, C = _local_case(2)
    Kn, _ = oracle.nofit_exchange(sysd, C)
    errs = [np.max(np.abs(oracle.brute_exchange_local(sysd, C, e)[0] - Kn)) for e in (1e-1, 1e-2, 5e-3)]
    assert errs[1] < 0.2 * errs[0] and errs[2] < 0.6 * errs[1]
    assert errs[2] < 2e-3 * np.max(np.abs(Kn))


def test_local_selection_threshold_is_relative_per_atom():
    """The local selection stops on each atom once its largest residual falls
    below local_tol times that atom's own largest initial residual: the last
    pivot value of every atom sits above the threshold and the atom's
    remaining residual below it (or the cap was reached)."""
    sysd, C = _local_case(2)
    tol = 1e-6
    r = oracle.run_local(sysd, C, 20, local_tol=tol, local_cap=400, eps_r=1e-2)
    codes = r["local_pivots"]
    atoms = codes >> O.LOCAL_ATOM_SHIFT
    for A, blk in enumerate(r["blocks"]):
        dv = r["local_dvals"][atoms == A]
        d0 = np.max(O.initial_diagonal(blk))
        assert dv.size and dv[0] == pytest.approx(d0)
        assert np.all(dv >= tol * d0)
        sel = O.select_points([blk], dv.size + 1, 0.0)
        assert sel["dvals"][-1] < tol * d0


def test_local_grids_with_the_sinc_coarse_level_exact_at_full_rank():
    """Local grids on the finest level and the coarsest level as the sinc
    grid together: at full rank the exchange is again the 4-index exchange of
    the local pair partition (the coarse pairs are exact on the sinc grid)."""
    sysd, C = _local_case(3)
    Kb, Eb = oracle.brute_exchange_local(sysd, C, 1e-2)
    r = oracle.run_local(sysd, C, 400, tol=1e-14, local_tol=1e-14, local_cap=400, eps_r=1e-2, sinc=True, reg_rel=0.0)
    assert np.max(np.abs(r["K"] - Kb)) <= 2e-8 * np.max(np.abs(Kb))
    assert abs(r["Ex"] - Eb) <= 2e-8 * abs(Eb)
