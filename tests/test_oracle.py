"""Pins of the CPU oracle against facts the paper and mathematics fix.

Each test targets a plausible mistake: a dropped stencil term, a wrong sign,
a transposed offset, a misplaced half-node stretch, a wrong transfer weight,
a broken Krylov minimiser, a wrong adjoint or gradient.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import hz_workloads as W
from oracle import gradient as og
from oracle import iofd
from oracle import threegrid as tg

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(f"{GOLDEN}/{name}"):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def small_problem(n=16, n_pml=4, kind="homogeneous", gamma_max=1.119058, seed=0):
    if kind == "homogeneous":
        w = W.homogeneous(n=n, n_pml=n_pml)
        c = w.c
    else:
        w = W.random_field(n=n, n_pml=n_pml, nsrc=2, nrec_side=4)
        c = w.c
    return w, iofd.make_problem(c, n_pml, w.h, w.omega, gamma_max)


# ---------------------------------------------------------------- tables
def test_hermite_reproduces_cubic():
    """Cubic Hermite interpolation is exact for a cubic polynomial."""
    s = np.linspace(0, 0.4, 17)
    f = lambda x: 1.5 - 2 * x + 3 * x ** 2 - 7 * x ** 3
    df = lambda x: -2 + 6 * x - 21 * x ** 2
    x = np.linspace(0, 0.4, 101)
    v, dv = iofd.hermite(s, f(s)[:, None], df(s)[:, None], x)
    assert np.allclose(v[:, 0], f(x), atol=1e-13)
    assert np.allclose(dv[:, 0], df(x), atol=1e-11)


def test_table_bounds_from_paper():
    """a1 >= 0.588 and h^2 d_h^0 >= 3.519 on nu in [6, 24] (Sec. 4.3); the mass
    symbol stays positive so the shifted symbols are invertible."""
    g = _golden("symbol_bounds.txt")
    T = iofd.load_tables()
    eta = np.linspace(0, 0.4, 801)
    a, _ = iofd.hermite(T.s, T.alpha, T.dalpha, eta)
    assert a[:, 0].min() >= g["a1_min"]
    nu = np.linspace(6, 24, 361)
    kap = 2 * math.pi / nu
    a, _ = iofd.hermite(T.s, T.alpha, T.dalpha, kap / (2 * math.pi))
    d0 = 6 * a[:, 3] - kap ** 2 * a[:, 0]
    # the paper prints 3.519 (four digits); our independently fitted interior
    # operator gives 3.5185, equal at the printed precision
    assert d0.min() >= g["h2d0_min"] - 1e-3
    for zeta in itertools.product((-1.0, 1.0), repeat=3):
        a1, a2, a3 = a[:, 0], a[:, 1], a[:, 2]
        m = a1 + a2 / 3 * sum(zeta) + a3 / 3 * (zeta[0] * zeta[1] + zeta[0] * zeta[2] + zeta[1] * zeta[2]) \
            + (1 - a1 - a2 - a3) * zeta[0] * zeta[1] * zeta[2]
        assert m.min() > 0.3


# ---------------------------------------------------------------- set-up
def test_pml_profile_values():
    """gamma = gamma_max [1 - cos(pi d / 2L)] (Eq. pml-profile): 0 in the box,
    gamma_max at the outer face, gamma_max (1 - 1/sqrt 2) half way."""
    n, p, gm = 32, 8, 1.119058
    g = iofd.pml_gamma(n, p, gm, np.array([8, 16, 24, 0, 32, 4, 28, -1]))
    ref = [0, 0, 0, gm, gm, gm * (1 - math.cos(math.pi / 4)), gm * (1 - math.cos(math.pi / 4)), gm]
    assert np.allclose(g, ref, atol=1e-15)
    xin, xih = iofd.pml_1d(n, p, gm)
    # half node between 4 and 5 averages gamma before inverting
    g4, g5 = iofd.pml_gamma(n, p, gm, np.array([4, 5]))
    assert abs(xih[5] - 1 / (1 + 0.5j * (g4 + g5))) < 1e-15
    assert abs(xin[4] - 1 / (1 + 1j * g4)) < 1e-15


def test_velocity_extension_nearest_interior():
    c = np.random.default_rng(0).uniform(1, 2, (17, 17, 17))
    ce = iofd.extend_velocity(c, 4)
    assert np.array_equal(ce[4:13, 4:13, 4:13], c[4:13, 4:13, 4:13])
    assert ce[0, 0, 0] == c[4, 4, 4] and ce[16, 2, 9] == c[12, 4, 9]


# ---------------------------------------------------------------- coarse levels
def _same_level(la, lb):
    """True when two levels define the same rows: intervals, PML layers,
    spacing, kappa and the per-axis stretch factors at nodes and half nodes."""
    return (tuple(la.n) == tuple(lb.n) and la.n_pml == lb.n_pml and la.ell == lb.ell
            and np.array_equal(la.kappa, lb.kappa)
            and all(np.array_equal(pa[0], pb[0]) and np.array_equal(pa[1], pb[1])
                    for pa, pb in zip(la.pml, lb.pml)))


def _coarse_case(shape=(40, 24, 32), n_pml=8, seed=3):
    rng = np.random.default_rng(seed)
    c = rng.uniform(1.5, 3.0, tuple(m + 1 for m in shape))   # values in the PML too
    h, omega = 1.0 / (min(shape) - 2 * n_pml), 17.0
    return c, n_pml, h, omega


@pytest.mark.parametrize("L", [1, 2])
def test_coarse_level_is_the_problem_rediscretised_on_the_coarse_grid(L):
    """Sec. 3.1: level L is the same PML problem discretised on the grid of
    spacing 2^L h -- the velocity (extended into the PML from the physical box)
    sampled at the coarse nodes, i.e. fine node 2^L j; a PML of the same
    physical thickness, i.e. n_pml / 2^L layers; kappa = omega 2^L h / c.  So
    the oracle's level L must be level 0 of a problem built directly on the
    coarse grid from the raw velocity at every 2^L-th fine node, with spacing
    2^L h and n_pml / 2^L layers, at the same omega; and its operator rows the
    same.  Independent spot values: kappa at one node from the velocity of the
    fine node it sits on, and the stretch at a coarse PML node and half node
    from gamma evaluated at their physical distance into the layer."""
    c, p, h, omega = _coarse_case()
    f = 1 << L
    prob = iofd.make_problem(c, p, h, omega)
    coarse = iofd.make_problem(c[::f, ::f, ::f], p // f, f * h, omega, nlevels=1)
    lev = prob.levels[L]
    assert _same_level(lev, coarse.levels[0])
    x = W.random_complex(lev.shape, 11)
    for sigma in (0.0, 0.9):
        assert np.array_equal(iofd.operator_A(prob, L, sigma)(x), iofd.operator_A(coarse, 0, sigma)(x))
    # kappa at coarse node (iz, iy, ix): the fine node (f iz, f iy, f ix), moved to
    # the nearest physical node when it lies in the PML
    n = tuple(m - 1 for m in c.shape)
    for j in [(0, 1, 2), (2, 3, 1), (lev.shape[0] - 1, 1, lev.shape[2] - 2)]:
        fine = [min(max(f * jj, p), nn - p) for jj, nn in zip(j, n)]
        assert lev.kappa[j] == pytest.approx(omega * (f * h) / c[tuple(fine)], rel=1e-15)
    # stretch at coarse node 1 of the x axis and at the half node between nodes
    # 0 and 1: gamma from the physical distance into the layer of thickness p h
    gm, L_pml = prob.gamma_max, p * h
    gamma = lambda x_pos: gm * (1 - math.cos(math.pi * max(L_pml - x_pos, 0.0) / (2 * L_pml)))
    xin, xih = lev.pml[2]
    assert abs(xin[1] - 1 / (1 + 1j * gamma(1 * f * h))) < 1e-14
    assert abs(xih[1] - 1 / (1 + 0.5j * (gamma(0.0) + gamma(f * h)))) < 1e-14


def test_coarse_level_pin_rejects_planted_mistakes():
    """The comparison above is sharp: levels built with kappa = omega h / c
    (spacing not scaled), with the PML layers not halved, or with the velocity
    of the odd fine nodes all differ from the rediscretised level."""
    c, p, h, omega = _coarse_case()
    prob = iofd.make_problem(c, p, h, omega)
    ref = iofd.make_problem(c[::2, ::2, ::2], p // 2, 2 * h, omega, nlevels=1).levels[0]
    lev = prob.levels[1]
    assert _same_level(lev, ref)
    wrong_ell = dataclasses_replace(lev, kappa=omega * h / prob.c_ext[::2, ::2, ::2])
    wrong_pml = dataclasses_replace(lev, pml=tuple(iofd.pml_1d(m, p, prob.gamma_max) for m in lev.n))
    odd = np.ix_(*[np.minimum(2 * np.arange(m) + 1, 2 * (m - 1)) for m in lev.shape])
    wrong_c = dataclasses_replace(lev, kappa=omega * 2 * h / prob.c_ext[odd])
    assert wrong_c.kappa.shape == lev.kappa.shape
    for bad in (wrong_ell, wrong_pml, wrong_c):
        assert not _same_level(bad, ref)


def dataclasses_replace(obj, **kw):
    import dataclasses
    return dataclasses.replace(obj, **kw)


def test_point_source_normalisation():
    w, prob = small_problem()
    F = iofd.point_sources(prob, [(3, 4, 5, 2.0 + 1.0j)])
    assert F.sum() == pytest.approx((2.0 + 1.0j) / w.h ** 3)
    assert F[0, 5, 4, 3] == pytest.approx((2.0 + 1.0j) / w.h ** 3)


# ---------------------------------------------------------------- operator
def paper_shell_symbol(a, kap2, theta):
    """Eq. shifted-iofd-symbol with C_m from Eq. iofd-shell-coefficients (ell = 1)."""
    a1, a2, a3, a4, a5 = a
    C0 = 6 * a4 - kap2 * a1
    C1 = -a4 + a5 - kap2 * a2 / 6
    C2 = -a5 / 2 + (1 - a4 - a5) / 2 - kap2 * a3 / 12
    C3 = -0.75 * (1 - a4 - a5) - kap2 * (1 - a1 - a2 - a3) / 8
    z = np.cos(theta)
    return C0 + 2 * C1 * z.sum() + 4 * C2 * (z[0] * z[1] + z[0] * z[2] + z[1] * z[2]) + 8 * C3 * z.prod()


@pytest.mark.parametrize("sigma", [0.0, 0.9])
@pytest.mark.parametrize("L", [0, 1])
def test_interior_symbol_matches_closed_form(L, sigma):
    """Applied to a plane wave exp(i theta.n) at an interior node, the
    tensor-product PML stencil (gamma_max > 0 elsewhere) reproduces the
    closed-form shell symbol of Sec. 4.3 to rounding."""
    w, prob = small_problem(n=24, n_pml=4)
    lev = prob.levels[L]
    A = iofd.operator_A(prob, L, sigma, cache=False)
    rng = np.random.default_rng(5)
    nz, ny, nx = lev.shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c = tuple(s // 2 for s in lev.shape)
    for _ in range(4):
        th = rng.uniform(-math.pi, math.pi, 3)      # (theta_z, theta_y, theta_x)
        pw = np.exp(1j * (th[0] * Z + th[1] * Y + th[2] * X))
        val = A(pw)[c] / pw[c] * lev.ell ** 2
        a, _ = iofd.hermite(prob.tables.s, prob.tables.alpha, prob.tables.dalpha, lev.eta_star[c])
        ref = paper_shell_symbol(a, (1 + 1j * sigma) * lev.kappa[c] ** 2, th)
        assert abs(val - ref) < 1e-12 * max(1, abs(ref))


def test_textbook_limit_is_7point_laplacian():
    """alpha = (1, 0, 0, 1, 0) without PML gives -Laplace_7pt - k^2, assembled
    independently as a Kronecker sum of 1-D second differences."""
    n = 8
    K = 17
    T = iofd.Tables(np.linspace(0, 0.4, K), np.tile([1.0, 0, 0, 1.0, 0], (K, 1)), np.zeros((K, 5)),
                    np.tile([1.0, 0, 0], (K, 1)), np.zeros((K, 3)))
    c = np.full((n + 1,) * 3, 1.0)
    h = 0.1
    omega = 2.0
    prob = iofd.make_problem(c, 0, h, omega, 0.0, T)
    D2 = sp.diags([np.ones(n), -2 * np.ones(n + 1), np.ones(n)], [-1, 0, 1]) / h ** 2
    I = sp.identity(n + 1)
    lap = sp.kron(sp.kron(D2, I), I) + sp.kron(sp.kron(I, D2), I) + sp.kron(sp.kron(I, I), D2)
    ref = -lap - (omega ** 2) * sp.identity((n + 1) ** 3)
    x = W.random_complex((n + 1,) * 3, 3)
    y = iofd.operator_A(prob)(x)
    assert np.allclose(y.ravel(), ref @ x.ravel(), rtol=0, atol=1e-11 * np.abs(ref @ x.ravel()).max())
    Q = iofd.operator_Q(prob)
    assert np.allclose(Q(x), x)


def test_q_operator_shells_and_constants():
    """Q_h of Eq. q-operator with an arbitrary beta table: the four shell
    weights times the shell sizes 1, 6, 12, 8 add up to one, so Q maps a
    constant to itself at every node whose 27 neighbours are inside; on a plane
    wave it multiplies by the shell-sum symbol Q_0 + 2 Q_1 sum cos + 4 Q_2 sum
    cos cos + 8 Q_3 prod cos.  A weight on the wrong shell or a wrong
    denominator breaks one of the two."""
    w, prob0 = small_problem(n=16, n_pml=4, kind="random")
    rng = np.random.default_rng(41)
    T0 = prob0.tables
    beta = rng.uniform(-0.5, 1.5, T0.beta.shape)
    dbeta = rng.uniform(-1.0, 1.0, T0.dbeta.shape)
    T = iofd.Tables(T0.s, T0.alpha, T0.dalpha, beta, dbeta)
    prob = iofd.make_problem(w.c, w.n_pml, w.h, w.omega, w.gamma_max, T)
    Q = iofd.operator_Q(prob)
    shape = prob.levels[0].shape
    one = Q(np.ones(shape, np.complex128))
    assert np.allclose(one[1:-1, 1:-1, 1:-1], 1.0, rtol=0, atol=1e-13)
    Z, Y, X = np.meshgrid(*[np.arange(m) for m in shape], indexing="ij")
    lev = prob.levels[0]
    for k in range(4):
        th = rng.uniform(-math.pi, math.pi, 3)
        pw = np.exp(1j * (th[0] * Z + th[1] * Y + th[2] * X))
        c = tuple(rng.integers(1, m - 1) for m in shape)
        b, _ = iofd.hermite(T.s, T.beta, T.dbeta, lev.eta_star[c])
        q = [b[0], b[1] / 6, b[2] / 12, (1 - b[0] - b[1] - b[2]) / 8]
        z = np.cos(th)
        sym = (q[0] + 2 * q[1] * z.sum() + 4 * q[2] * (z[0] * z[1] + z[0] * z[2] + z[1] * z[2])
               + 8 * q[3] * z.prod())
        assert abs(Q(pw)[c] / pw[c] - sym) < 1e-12 * max(1.0, abs(sym))


@pytest.mark.parametrize("L,sigma", [(0, 0.0), (1, 0.0), (1, 0.9), (2, 0.9)])
def test_matrix_free_equals_kronecker_assembly(L, sigma):
    """Matrix-free rows (inside and outside the PML, variable kh) equal the
    independent Kronecker-product assembly."""
    w, prob = small_problem(n=16, n_pml=4, kind="random")
    A = iofd.operator_A(prob, L, sigma)
    M = iofd.assemble(prob, L, sigma)
    x = W.random_complex(prob.levels[L].shape, 7 + L)
    y = M @ x.ravel()
    assert np.abs(A(x).ravel() - y).max() <= 1e-13 * np.abs(y).max()
    MQ = iofd.assemble(prob, 0, which="Q")
    xq = W.random_complex(prob.levels[0].shape, 9)
    assert np.allclose(iofd.operator_Q(prob)(xq).ravel(), MQ @ xq.ravel(), atol=1e-13)


def test_pointwise_rows_equal_full_grid_rows():
    """The sampled-row evaluator (used for checks at full sizes) gives the same
    rows as the full-grid evaluator, inside and outside the PML."""
    w, prob = small_problem(n=16, n_pml=4, kind="random")
    rng = np.random.default_rng(8)
    for L, sig in [(0, 0.0), (1, 0.9)]:
        lev = prob.levels[L]
        pts = [rng.integers(0, m, 40) for m in lev.shape]
        for d in iofd.OFFSETS[::5]:
            full = iofd.row_coefficient(lev, prob.tables, d, sig)[pts[0], pts[1], pts[2]]
            part = iofd.row_coefficient_points(lev, prob.tables, d, *pts, shift_sigma=sig)
            assert np.allclose(full, part, rtol=1e-14, atol=0)
            lazy = iofd.make_level_points(w.c, w.n_pml, w.h, w.omega, w.gamma_max, L)
            part2 = iofd.row_coefficient_points(lazy, prob.tables, d, *pts, shift_sigma=sig)
            assert np.allclose(full, part2, rtol=1e-14, atol=0)


def test_pml_without_stretch_equals_interior_form():
    """gamma_max = 0 removes every PML term: the stencil is the shell form everywhere."""
    w, prob0 = small_problem(n=16, n_pml=4, gamma_max=0.0)
    A = iofd.operator_A(prob0)
    for d in iofd.OFFSETS:
        cf = A.coeff(d)
        assert np.allclose(cf, cf[8, 8, 8])


def test_adjoint_dot_test():
    """<A u, v> = <u, A^H v> to 1e-13 (A, B_2h, Q)."""
    w, prob = small_problem(n=16, n_pml=4, kind="random")
    for op, shape in [(iofd.operator_A(prob), prob.levels[0].shape),
                      (iofd.operator_A(prob, 1, 0.9), prob.levels[1].shape),
                      (iofd.operator_Q(prob), prob.levels[0].shape)]:
        u = W.random_complex(shape, 11)
        v = W.random_complex(shape, 12)
        lhs = np.vdot(v, op(u))
        rhs = np.vdot(op.adjoint(v), u)
        assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_second_order_consistency_in_pml():
    """Truncation error on a smooth function decreases ~h^2 inside the PML:
    compare ell^2 (A f) with the continuous -sum xi^-1 d(xi^-1 d f) - k^2 f."""
    errs = []
    for n in (32, 64):
        n_pml = n // 4
        h = 1.0 / (n - 2 * n_pml)
        prob = iofd.make_problem(np.ones((n + 1,) * 3), n_pml, h, 3.0, 0.8)
        x = (np.arange(n + 1) - n_pml) * h
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        L = n_pml * h
        f = np.sin(2.1 * X + 0.4) * np.cos(1.3 * Y) * np.exp(0.5 * Z)

        def gam(t):
            d = np.clip(np.maximum(-t, t - (1.0)), 0, L)
            return 0.8 * (1 - np.cos(np.pi * d / (2 * L)))

        def dgam(t):
            d = np.maximum(-t, t - 1.0)
            s = np.where(t < 0, -1.0, 1.0)
            return np.where((d > 0) & (d <= L), 0.8 * np.sin(np.pi * d / (2 * L)) * np.pi / (2 * L) * s, 0.0)
        # -xi^-1 (xi^-1 f')' = -xi^-2 f'' + xi^-3 xi' f'
        terms = 0
        for (t, d1, d2) in ((X, 2.1 * np.cos(2.1 * X + 0.4) * np.cos(1.3 * Y) * np.exp(0.5 * Z),
                             -4.41 * f),
                            (Y, -1.3 * np.sin(2.1 * X + 0.4) * np.sin(1.3 * Y) * np.exp(0.5 * Z),
                             -1.69 * f),
                            (Z, 0.5 * f, 0.25 * f)):
            xi = 1 + 1j * gam(t)
            dxi = 1j * dgam(t)
            terms = terms - d2 / xi ** 2 + dxi * d1 / xi ** 3
        k2 = (3.0) ** 2
        ref = terms - k2 * f
        Af = iofd.operator_A(prob, cache=False)(f)
        # gamma'' jumps at the PML interface and gamma' at the clamped outer
        # face: keep nodes whose stencil stays two nodes clear of both kinks
        ok1 = (np.abs(x) >= 2 * h - 1e-12) & (np.abs(x - 1) >= 2 * h - 1e-12) \
            & (np.abs(x + L) >= 3 * h - 1e-12) & (np.abs(x - 1 - L) >= 3 * h - 1e-12)
        mask = ok1[:, None, None] & ok1[None, :, None] & ok1[None, None, :]
        inpml = (np.abs(gam(X)) + np.abs(gam(Y)) + np.abs(gam(Z))) > 0
        mask &= inpml
        errs.append(np.abs(Af[mask] - ref[mask]).max() / np.abs(ref[mask]).max())
    assert errs[1] < errs[0] / 3.0


# ---------------------------------------------------------------- transfers
def test_restriction_is_scaled_prolongation_adjoint():
    """R = 2^-3 P^* (Sec. 3.1)."""
    v = W.random_complex((17, 17, 17), 1)
    w = W.random_complex((9, 9, 9), 2)
    lhs = np.vdot(w, tg.restrict(v))
    rhs = np.vdot(tg.prolong(w), v) / 8.0
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_prolongation_exact_on_trilinear():
    xc = np.arange(9.0)
    Zc, Yc, Xc = np.meshgrid(xc, xc, xc, indexing="ij")
    f = lambda X, Y, Z: 1 + 2 * X - Y + 0.5 * Z + 0.3 * X * Y - 0.2 * Y * Z + 0.1 * X * Y * Z
    xf = np.arange(17.0) / 2
    Zf, Yf, Xf = np.meshgrid(xf, xf, xf, indexing="ij")
    assert np.allclose(tg.prolong(f(Xc, Yc, Zc)), f(Xf, Yf, Zf))


def test_restriction_of_constant():
    r = tg.restrict(np.ones((17, 17, 17)))
    assert np.allclose(r[1:-1, 1:-1, 1:-1], 1.0)
    assert r[0, 4, 4] == pytest.approx(0.75)   # ghost zero outside


# ---------------------------------------------------------------- Jacobi
def test_jacobi_telescoping_symbol():
    """n_J sweeps from zero: H J(H, g) = (1 - s^nJ) g on a plane wave, away from
    the boundary and the PML, with s = 1 - omega b/d (Eq.
    lfa-bottom-preconditioned-symbol)."""
    w, prob = small_problem(n=24, n_pml=4)
    B = iofd.operator_A(prob, 0, 0.9)
    lev = prob.levels[0]
    Z, Y, X = np.meshgrid(*[np.arange(m) for m in lev.shape], indexing="ij")
    th = np.array([0.7, -1.9, 2.4])
    g = np.exp(1j * (th[0] * Z + th[1] * Y + th[2] * X))
    c = tuple(s // 2 for s in lev.shape)
    bsym = B(g)[c] / g[c]
    d = B.diag()[c]
    for nJ, om in [(1, 0.8), (2, 0.2), (3, 0.8)]:
        y = tg.jacobi(B, g, om, nJ)
        s = 1 - om * bsym / d
        assert abs(B(y)[c] / g[c] - (1 - s ** nJ)) < 1e-12


# ---------------------------------------------------------------- Krylov
def test_gmres_cycle_is_krylov_minimiser():
    """After m right-preconditioned steps from x0 the residual equals the
    minimum over x0 + M K_m(A M, r0), computed by dense least squares on the
    explicit Krylov basis."""
    w, prob = small_problem(n=12, n_pml=4)
    A = iofd.operator_A(prob, 0, 0.3)
    M = lambda v: tg.jacobi(A, v, 0.5, 2)
    g = W.random_complex(prob.levels[0].shape, 21)
    x0 = W.random_complex(prob.levels[0].shape, 22) * 1e-3
    for m in (1, 2, 4):
        x = tg.fgmres_cycle(A, M, g, x0, m)
        r0 = g - A(x0)
        K = [r0]
        for _ in range(m - 1):
            K.append(A(M(K[-1])))
        Zs = np.stack([M(k).ravel() for k in K], axis=1)
        AZ = np.stack([A(M(k)).ravel() for k in K], axis=1)
        y = np.linalg.lstsq(AZ, r0.ravel(), rcond=None)[0]
        rbest = np.linalg.norm(r0.ravel() - AZ @ y)
        rgot = np.linalg.norm((g - A(x)).ravel())
        assert rgot == pytest.approx(rbest, rel=1e-9)
        assert np.allclose(x.ravel(), x0.ravel() + Zs @ y, atol=1e-9 * np.abs(x).max())


def _transfer_matrices_1d(m):
    """Full weighting (1/4, 1/2, 1/4) and linear interpolation between m + 1 fine
    and m/2 + 1 coarse nodes, written from the stencil weights (zero outside)."""
    mc = m // 2
    R1 = np.zeros((mc + 1, m + 1))
    P1 = np.zeros((m + 1, mc + 1))
    for J in range(mc + 1):
        R1[J, 2 * J] = 0.5
        P1[2 * J, J] = 1.0
        if 2 * J + 1 <= m:
            R1[J, 2 * J + 1] = 0.25
            P1[2 * J + 1, J] = 0.5
            P1[2 * J + 1, J + 1] = 0.5
        if J >= 1:
            R1[J, 2 * J - 1] = 0.25
    return R1, P1


@pytest.mark.parametrize("adjoint", [False, True])
def test_shifted_vcycle_is_two_grid_error_operator(adjoint):
    """With an exact 4h solve in place of C_4h, the shifted cycle of Eq.
    shifted-auxiliary-cycle has the textbook two-grid error propagation
    e - V(B e) = S^nJ (I - P B_4h^-1 R B_2h) S^nJ e, S = I - omega D^-1 B_2h,
    on the shifted operators (Eq. shifted-operator) of a PML problem with
    variable kh.  The matrices come from the Kronecker assembly and the
    1-D transfer weights, not from the oracle's matrix-free code; swapping the
    smoothing order, a stale residual before the post-sweeps, the unshifted
    operator or a wrong transfer weight each break it.  The adjoint hierarchy
    uses B^H and conj(D) throughout."""
    w, prob = small_problem(n=16, n_pml=4, kind="random")
    p = tg.Params()
    B2 = iofd.assemble(prob, 1, p.sigma).toarray()
    B4 = iofd.assemble(prob, 2, p.sigma).toarray()
    if adjoint:
        B2, B4 = B2.conj().T, B4.conj().T
    R1, P1 = _transfer_matrices_1d(prob.levels[1].n[0])
    R = np.kron(np.kron(R1, R1), R1)
    P = np.kron(np.kron(P1, P1), P1)
    D = np.diag(B2)
    S = np.eye(len(D)) - p.w_2h * B2 / D[:, None]
    Sn = np.linalg.matrix_power(S, p.nJ_2h)
    E = Sn @ (np.eye(len(D)) - P @ np.linalg.solve(B4, R @ B2)) @ Sn

    M = tg.ThreeGrid(prob, p, adjoint=adjoint)
    shape4 = prob.levels[2].shape
    M.C_4h = lambda g: np.linalg.solve(B4, g.ravel()).reshape(shape4)
    e = W.random_complex(prob.levels[1].shape, 31)
    got = e - M.V_2h((B2 @ e.ravel()).reshape(e.shape))
    ref = E @ e.ravel()
    assert np.linalg.norm(got.ravel() - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("adjoint", [False, True])
def test_algorithm1_step_order_is_two_grid_error_operator(adjoint):
    """Algorithm 1 with its two Krylov solves replaced by linear maps -- S_h(g,
    x0) = x0 + omega D^-1 (g - A_h x0), K_2h = exact A_2h solve -- has the error
    propagation e - M(A_h e) = S (I - P A_2h^-1 R A_h) S e, S = I - omega D^-1
    A_h: steps 1-5 compose pre-smoothing from zero, restriction of the updated
    residual, the 2h correction and post-smoothing from the corrected iterate.
    Sparse matrices from the Kronecker assembly and the 1-D transfer weights."""
    w, prob = small_problem(n=16, n_pml=4, kind="random")
    p = tg.Params()
    A = iofd.assemble(prob, 0).tocsc()
    A2 = iofd.assemble(prob, 1).tocsc()
    if adjoint:
        A, A2 = A.conj().T.tocsc(), A2.conj().T.tocsc()
    R1, P1 = _transfer_matrices_1d(prob.levels[0].n[0])
    R1, P1 = sp.csr_matrix(R1), sp.csr_matrix(P1)
    R = sp.kron(sp.kron(R1, R1), R1, format="csr")
    P = sp.kron(sp.kron(P1, P1), P1, format="csr")
    d = A.diagonal()
    om = p.w_h
    S = lambda v: v - om * (A @ v) / d

    M = tg.ThreeGrid(prob, p, adjoint=adjoint)
    shape, shape2 = prob.levels[0].shape, prob.levels[1].shape
    M.S_h = lambda g, x0: (np.zeros_like(g) if x0 is None else x0) + om * (
        g - (A @ (np.zeros(g.size) if x0 is None else x0.ravel())).reshape(shape)) / d.reshape(shape)
    M.K_2h = lambda r2: spla.spsolve(A2, r2.ravel()).reshape(shape2)
    e = W.random_complex(shape, 32).ravel()
    got = e - M((A @ e).reshape(shape)).ravel()
    ref = S(e)
    ref = S(ref - P @ spla.spsolve(A2, R @ (A @ ref)))
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("adjoint", [False, True])
def test_krylov_solves_use_unshifted_operators(adjoint):
    """S_h (step 1) and K_2h (Eq. unshifted-middle-solve) iterate on the
    unshifted A_h and A_2h: with an exact inverse of that operator as the
    preconditioner, one Krylov step returns the exact solution.  Running either
    on the shifted B or on the wrong level leaves a residual."""
    w, prob = small_problem(n=16, n_pml=4, kind="random")
    p = tg.Params()
    A = iofd.assemble(prob, 0).tocsc()
    A2 = iofd.assemble(prob, 1).tocsc()
    if adjoint:
        A, A2 = A.conj().T.tocsc(), A2.conj().T.tocsc()
    shape, shape2 = prob.levels[0].shape, prob.levels[1].shape
    M = tg.ThreeGrid(prob, p, adjoint=adjoint)
    M.J = lambda H, g, omega, nJ: spla.spsolve(A, g.ravel()).reshape(shape)
    M.V_2h = lambda q: spla.spsolve(A2, q.ravel()).reshape(shape2)
    g = W.random_complex(shape, 33)
    x0 = W.random_complex(shape, 34)
    ref = spla.spsolve(A, g.ravel())
    for start in (None, x0):
        got = M.S_h(g, start).ravel()
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    r2 = W.random_complex(shape2, 35)
    ref2 = spla.spsolve(A2, r2.ravel())
    got2 = M.K_2h(r2).ravel()
    assert np.linalg.norm(got2 - ref2) <= 1e-10 * np.linalg.norm(ref2)


@pytest.mark.parametrize("adjoint", [False, True])
def test_bottom_solve_uses_shifted_operator(adjoint):
    """C_4h iterates on the shifted B_4h = L - (1 + i sigma) M at spacing 4h:
    with an exact inverse of B_4h as its Jacobi stand-in, one step is exact."""
    w, prob = small_problem(n=16, n_pml=4, kind="random")
    p = tg.Params()
    B4 = iofd.assemble(prob, 2, p.sigma).tocsc()
    if adjoint:
        B4 = B4.conj().T.tocsc()
    shape4 = prob.levels[2].shape
    M = tg.ThreeGrid(prob, p, adjoint=adjoint)
    M.J = lambda H, g, omega, nJ: spla.spsolve(B4, g.ravel()).reshape(shape4)
    g = W.random_complex(shape4, 36)
    ref = spla.spsolve(B4, g.ravel())
    assert np.linalg.norm(M.C_4h(g).ravel() - ref) <= 1e-10 * np.linalg.norm(ref)


def _dense_fgmres_minimiser(A, M, r0, k):
    """Residual-minimising correction over span{M r0, M (A M) r0, ...} (k
    directions), by dense least squares on the explicit Krylov basis."""
    K = [r0]
    for _ in range(k - 1):
        K.append(A(M(K[-1])))
    Zs = np.stack([M(v).ravel() for v in K], axis=1)
    AZ = np.stack([A(M(v)).ravel() for v in K], axis=1)
    y = np.linalg.lstsq(AZ, r0.ravel(), rcond=None)[0]
    return (Zs @ y).reshape(r0.shape), np.linalg.norm(r0.ravel() - AZ @ y)


def test_outer_fgmres_counts_and_restarts():
    """Outer FGMRES(m_out) (Eq. relative-residual stopping test, one
    preconditioner call per Arnoldi step): a run capped at one cycle returns the
    dense Krylov minimiser; a second cycle restarts from it; a tolerance met
    inside a cycle stops at the first step whose minimal residual meets it; an
    exact preconditioner needs one call."""
    w, prob = small_problem(n=12, n_pml=4, kind="random")
    A = iofd.operator_A(prob)
    M = lambda v: tg.jacobi(A, v, 0.5, 2)
    b = W.random_complex(prob.levels[0].shape, 37)
    bn = np.linalg.norm(b)
    m = 5
    d1, res1 = _dense_fgmres_minimiser(A, M, b, m)
    x, info = tg.fgmres_solve(A, M, b, tg.Params(tol=1e-30, max_pc=m, m_out=m))
    assert info.pc_calls == m and len(info.history) == 2
    assert np.linalg.norm((x - d1).ravel()) <= 1e-9 * np.linalg.norm(d1)
    assert info.rel_res == pytest.approx(res1 / bn, rel=1e-9)
    d2, res2 = _dense_fgmres_minimiser(A, M, b - A(d1), m)
    x, info = tg.fgmres_solve(A, M, b, tg.Params(tol=1e-30, max_pc=2 * m, m_out=m))
    assert info.pc_calls == 2 * m and len(info.history) == 3
    assert np.linalg.norm((x - d1 - d2).ravel()) <= 1e-8 * np.linalg.norm(d1 + d2)
    mins = [_dense_fgmres_minimiser(A, M, b, k)[1] / bn for k in range(1, m + 1)]
    assert all(mins[k + 1] < mins[k] for k in range(m - 1))
    tol = float(np.sqrt(mins[1] * mins[2]))          # met first at step 3
    x, info = tg.fgmres_solve(A, M, b, tg.Params(tol=tol, max_pc=50, m_out=m))
    assert info.pc_calls == 3 and info.rel_res == pytest.approx(mins[2], rel=1e-8)
    Asp = iofd.assemble(prob).tocsc()
    exact = lambda v: spla.spsolve(Asp, v.ravel()).reshape(v.shape)
    x, info = tg.fgmres_solve(A, exact, b, tg.Params(tol=1e-10, max_pc=50, m_out=m))
    assert info.pc_calls == 1 and info.rel_res <= 1e-10


@pytest.mark.parametrize("adjoint", [False, True])
def test_s_step_bottom_solve_equals_gmres(adjoint):
    """Reading of C_4h (Sec. 3.2): m_4h = 4 CA-GMRES steps -- monomial basis
    p_0 = g / ||g||, p_{k+1} = B J(p_k), the least-squares problem
    min || ||g|| p_0 - [p_1..p_4] y || solved through the 5 x 5 Gram block and
    its Cholesky factor, x = sum_k y_k J(p_k) -- give the iterate of
    GMRES(4) right-preconditioned by J on the same Krylov space, which the
    oracle runs (on the shifted 4h operator of a PML problem)."""
    w, prob = small_problem(n=16, n_pml=4, kind="random")
    p = tg.Params()
    M = tg.ThreeGrid(prob, p, adjoint=adjoint)
    B = M.op(M.B_4h)
    J = lambda v: M.J(M.B_4h, v, p.w_4h, p.nJ_4h)
    g = W.random_complex(prob.levels[2].shape, 38)
    beta = np.linalg.norm(g)
    P = [g / beta]
    for _ in range(p.m_4h):
        P.append(B(J(P[-1])))
    Pm = np.stack([v.ravel() for v in P], axis=1)
    G = Pm.conj().T @ Pm                                   # Gram block (5 x 5)
    L = np.linalg.cholesky(G[1:, 1:])
    y = np.linalg.solve(L.conj().T, np.linalg.solve(L, beta * G[1:, 0]))
    x_ca = sum(y[k] * J(P[k]) for k in range(p.m_4h))
    x_gm = tg.fgmres_cycle(B, J, g, None, p.m_4h)
    assert np.linalg.norm((x_ca - x_gm).ravel()) <= 1e-8 * np.linalg.norm(x_gm)


def test_cgs_selective_reorthogonalisation_and_givens_equal_mgs_lstsq():
    """Reading of the orthogonalisation and small least-squares steps (the
    paper names neither): classical Gram-Schmidt with a second pass only when
    the first removes more than half of ||w||^2 (criterion of Daniel, Gragg,
    Kaufman and Stewart), and Givens rotations on the Hessenberg matrix, give
    the flexible GMRES iterate of the oracle's modified Gram-Schmidt and lstsq
    (outer FGMRES(5) on A_h with a Jacobi preconditioner, from a nonzero x0)."""
    w, prob = small_problem(n=12, n_pml=4, kind="random")
    A = iofd.operator_A(prob)
    Mj = lambda v: tg.jacobi(A, v, 0.8, 2)
    g = W.random_complex(prob.levels[0].shape, 39)
    x0 = 1e-2 * W.random_complex(prob.levels[0].shape, 40)
    m = 5
    r0 = (g - A(x0)).ravel()
    beta = np.linalg.norm(r0)
    V = [r0 / beta]
    Z, H = [], np.zeros((m + 1, m), dtype=np.complex128)
    for j in range(m):
        z = Mj(V[j].reshape(g.shape)).ravel()
        Z.append(z)
        wv = A(z.reshape(g.shape)).ravel()
        Vm = np.stack(V, axis=1)
        h = Vm.conj().T @ wv
        w1 = wv - Vm @ h
        if np.vdot(w1, w1).real <= 0.5 * np.vdot(wv, wv).real:
            h2 = Vm.conj().T @ w1
            w1 = w1 - Vm @ h2
            h = h + h2
        H[:j + 1, j] = h
        H[j + 1, j] = np.linalg.norm(w1)
        V.append(w1 / H[j + 1, j])
    # Givens rotations reduce H to upper triangular form; back substitution
    R = H.copy()
    rhs = np.zeros(m + 1, dtype=np.complex128)
    rhs[0] = beta
    for j in range(m):
        a, b = R[j, j], R[j + 1, j]
        rho = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
        c, s = a / rho, b / rho
        G = np.array([[np.conj(c), np.conj(s)], [-s, c]])
        R[j:j + 2, j:] = G @ R[j:j + 2, j:]
        rhs[j:j + 2] = G @ rhs[j:j + 2]
    y = np.linalg.solve(np.triu(R[:m, :m]), rhs[:m])
    x = x0.ravel() + np.stack(Z, axis=1) @ y
    ref = tg.fgmres_cycle(A, Mj, g, x0, m).ravel()
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    assert abs(abs(rhs[m]) - np.linalg.norm(g.ravel() - A(x.reshape(g.shape)).ravel())) <= 1e-8 * beta


def test_cycle_with_zero_rhs_returns_zero():
    w, prob = small_problem(n=12, n_pml=4)
    A = iofd.operator_A(prob)
    z = np.zeros(prob.levels[0].shape, np.complex128)
    assert np.all(tg.fgmres_cycle(A, lambda v: v, z, None, 3) == 0)
    M = tg.ThreeGrid(prob)
    assert np.all(M(z) == 0)


def test_table4_defaults():
    g = _golden("table4_parameters.txt")
    p = tg.Params()
    for k, v in g.items():
        if k == "gamma_max":
            assert W.Workload.__dataclass_fields__["gamma_max"].default == v
        else:
            assert getattr(p, k) == v, k


def test_full_solve_matches_sparse_direct():
    """FGMRES + Algorithm 1 reaches the sparse direct solution of A_h v = Q f."""
    w, prob = small_problem(n=16, n_pml=4, kind="random")
    Q = iofd.operator_Q(prob)
    b = Q(iofd.point_sources(prob, [(8, 8, 8, 1.0)])[0])
    v, info = tg.solve(prob, b, tg.Params(tol=1e-10))
    assert info.rel_res <= 1e-10
    vd = spla.spsolve(iofd.assemble(prob).tocsc(), b.ravel())
    assert np.linalg.norm(v.ravel() - vd) / np.linalg.norm(vd) < 1e-8
    vadj, info = tg.solve_adjoint(prob, b, tg.Params(tol=1e-10))
    va = spla.spsolve(iofd.assemble(prob).conj().T.tocsc(), b.ravel())
    assert np.linalg.norm(vadj.ravel() - va) / np.linalg.norm(va) < 1e-8


@pytest.mark.slow
def test_green_function_48():
    """Homogeneous 32^3 + 8-point PML, ppw 6, centre source: u = Q v matches the
    outgoing Green function (Err of Sec. 5.1 on the 4h lattice outside one
    wavelength) at the level the paper reports (2.49e-3 at 512^3); we accept
    Err < 6e-3 at this size with our fitted tables."""
    w = W.homogeneous(n=48, n_pml=8)
    prob = iofd.make_problem(w.c, w.n_pml, w.h, w.omega)
    Q = iofd.operator_Q(prob)
    b = Q(iofd.point_sources(prob, w.sources)[0])
    v, info = tg.solve(prob, b, tg.Params(tol=1e-6))
    assert info.rel_res <= 1e-6 and info.pc_calls <= 30
    u = Q(v)
    n, p, h = w.n, w.n_pml, w.h
    k = w.omega
    x = (np.arange(n + 1) - p) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    xs = [(w.sources[0][j] - p) * h for j in range(3)]
    r = np.sqrt((X - xs[0]) ** 2 + (Y - xs[1]) ** 2 + (Z - xs[2]) ** 2)
    G = np.exp(1j * k * r) / (4 * math.pi * np.maximum(r, 1e-300))
    mask = np.zeros(r.shape, bool)
    mask[p:n - p + 1:4, p:n - p + 1:4, p:n - p + 1:4] = True
    mask &= r >= 2 * math.pi / k
    Wt = r[mask]
    err = (np.abs(Wt * (G.real - u.real)[mask]).sum() / np.abs(Wt * G.real[mask]).sum()
           + np.abs(Wt * (G.imag - u.imag)[mask]).sum() / np.abs(Wt * G.imag[mask]).sum())
    assert err < 6e-3


def test_phase_audit_of_tables():
    """Normalised numerical wavenumber of the oracle's interior stencil at
    nu = 6 (fine) and ppw 3 (2h), bisection on [0.9, 1.1] with 50 steps
    (Sec. 4.2), within twice the paper's printed mismatch."""
    g = _golden("phase_audit.txt")
    T = iofd.load_tables()
    prob_h = iofd.make_problem(np.ones((9, 9, 9)), 0, 1.0, 2 * math.pi / 6, 0.0, T, nlevels=1)
    prob_2h = iofd.make_problem(np.ones((9, 9, 9)), 0, 1.0, 2 * math.pi / 3, 0.0, T, nlevels=1)
    c = (4, 4, 4)

    def coeffs(prob):
        lev = prob.levels[0]
        return {d: iofd.row_coefficient(lev, T, d)[c] for d in iofd.OFFSETS}, lev.kappa[c]

    def q_of(cf, kap, dvec):
        f = lambda q: np.real(sum(v * np.exp(1j * q * kap * np.dot(d, dvec)) for d, v in cf.items()))
        lo, hi = 0.9, 1.1
        flo = f(lo)
        for _ in range(50):
            mid = 0.5 * (lo + hi)
            fm = f(mid)
            if np.sign(fm) == np.sign(flo):
                lo, flo = mid, fm
            else:
                hi = mid
        return 0.5 * (lo + hi)
    ch, kh = coeffs(prob_h)
    c2, k2 = coeffs(prob_2h)
    eh = e2 = ed = 0.0
    for th in np.linspace(0, math.pi / 2, 7):
        for ph in np.linspace(0, math.pi / 2, 7):
            dvec = np.array([math.cos(th), math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph)])
            qh = q_of(ch, kh, dvec)
            q2 = q_of(c2, k2, dvec)
            eh, e2, ed = max(eh, abs(qh - 1)), max(e2, abs(q2 - 1)), max(ed, abs(q2 - qh))
    assert eh <= 2 * g["q_h_err"] and e2 <= 2 * g["q_2h_err"] and ed <= 2 * g["q_diff"]


# ---------------------------------------------------------------- gradient
def test_row_derivatives_match_central_differences():
    """d A_i(delta)/d m_i and d Q_i(delta)/d m_i (every offset, inside and
    outside the PML; the PML nodes carry the copied physical value) against
    central differences of the row coefficients under a node-wise random
    perturbation of m = 1/c^2: each row depends on its own node only."""
    n, p = 12, 4
    w = W.random_field(n=n, n_pml=p, nsrc=1, nrec_side=4)
    prob0 = iofd.make_problem(w.c, p, w.h, w.omega, w.gamma_max)
    m0 = 1.0 / prob0.c_ext ** 2
    xi = np.random.default_rng(4).uniform(0.5, 1.5, m0.shape)
    eps = 1e-5
    probs = [iofd.make_problem(1.0 / np.sqrt(m0 * (1 + sgn * eps * xi)), p, w.h, w.omega, w.gamma_max)
             for sgn in (1, -1)]
    dm = 1.0 / probs[0].c_ext ** 2 - 1.0 / probs[1].c_ext ** 2
    assert np.all(np.abs(dm) > 0)
    for d in iofd.OFFSETS:
        fd = (iofd.row_coefficient(probs[0].levels[0], probs[0].tables, d)
              - iofd.row_coefficient(probs[1].levels[0], probs[1].tables, d)) / dm
        ref = og.row_coefficient_dm(prob0, m0, d)
        assert np.abs(fd - ref).max() <= 1e-6 * np.abs(ref).max(), d
        fq = (iofd.q_coefficient(probs[0].levels[0], probs[0].tables, d)
              - iofd.q_coefficient(probs[1].levels[0], probs[1].tables, d)) / dm
        refq = og.q_coefficient_dm(prob0, m0, d)
        assert np.abs(fq - refq).max() <= 1e-6 * np.abs(refq).max() + 1e-12, d


def test_gradient_matches_central_differences():
    """Adjoint-state dJ/dm against central differences of J(m) on random voxels
    (including one next to the PML, whose extension copies fold onto it)."""
    n, p = 12, 4
    w = W.random_field(n=n, n_pml=p, nsrc=2, nrec_side=4)
    rec = w.receivers
    d_obs = og.synthetic_data(w.c_true, p, w.h, w.omega, w.sources, rec)
    m0 = 1.0 / w.c ** 2
    J0, g, _ = og.misfit_and_gradient(w.c, p, w.h, w.omega, w.sources, rec, d_obs)
    assert np.all(g[:p] == 0) and np.all(g[:, :, -p:] == 0)
    rng = np.random.default_rng(3)
    vox = [tuple(rng.integers(p + 1, n - p, 3)) for _ in range(4)] + [(p, p + 1, p + 2)]
    for v in vox:
        eps = 1e-4 * m0[v]
        mp = m0.copy()
        mp[v] += eps
        mm = m0.copy()
        mm[v] -= eps
        Jp = og.misfit(1 / np.sqrt(mp), p, w.h, w.omega, w.sources, rec, d_obs)
        Jm = og.misfit(1 / np.sqrt(mm), p, w.h, w.omega, w.sources, rec, d_obs)
        fd = (Jp - Jm) / (2 * eps)
        assert fd == pytest.approx(g[v], rel=1e-4, abs=1e-8 * np.abs(g).max())
