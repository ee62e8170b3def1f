"""Oracle: PML-truncated IOFD discretisation (paper Sec. 2) -- test infrastructure.

Plain complex128 NumPy.  Grid fields are arrays of shape (nz+1, ny+1, nx+1)
indexed [iz, iy, ix]; nodes outside 0..n carry the Dirichlet value u = 0
(Eq. helmholtz-pml).  Readings of points the paper leaves open:

* PML distance d_j is counted in nodes from the first physical node and
  clamped to L_pml, so the ghost node just outside the box has gamma_max;
  it only enters through the half-node stretch xi_{-1/2}, xi_{n+1/2}.
* Coarse levels use n/2^L intervals and n_pml/2^L PML layers (Sec. 3.1
  halves the layer count with each coarsening), velocity injected from fine node
  2^L j, and gamma evaluated at the coarse node's own position.
* Q_h uses its shell form everywhere, inside the PML too (Sec. 2.2 gives
  only the shell form).
"""
from __future__ import annotations

import dataclasses
import itertools
import math
import os

import numpy as np
import scipy.sparse as sp

OFFSETS = [d for d in itertools.product((-1, 0, 1), repeat=3)]   # (dz, dy, dx)
ETA_MAX = 0.4   # Eq. iofd-clamped-coordinate


# ----------------------------------------------------------------------------
# IOFD tables and cubic Hermite interpolation (Sec. 2.2: each alpha_j and
# beta_j is a piecewise cubic Hermite curve through tabulated node values)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Tables:
    s: np.ndarray        # (K,) uniform nodes on [0, 0.4]
    alpha: np.ndarray    # (K, 5) values
    dalpha: np.ndarray   # (K, 5) d/ds
    beta: np.ndarray     # (K, 3)
    dbeta: np.ndarray    # (K, 3)


def default_table_path():
    here = os.path.dirname(os.path.abspath(__file__))
    return os.path.join(here, "..", "paper_2608_22946_gb300", "tables", "iofd_tables.txt")


def load_tables(path: str | None = None) -> Tables:
    rows = np.loadtxt(path or default_table_path(), comments="#")
    return Tables(rows[:, 0], rows[:, 1:6], rows[:, 6:11], rows[:, 11:14], rows[:, 14:17])


def hermite(s_nodes, vals, ders, s):
    """Cubic Hermite interpolant through (s_k, vals_k, ders_k), evaluated at s.
    Returns (value, d value / ds), each of shape s.shape + vals.shape[1:]."""
    s = np.asarray(s, dtype=np.float64)
    ds = s_nodes[1] - s_nodes[0]
    k = np.clip(np.floor((s - s_nodes[0]) / ds).astype(np.int64), 0, len(s_nodes) - 2)
    t = ((s - s_nodes[k]) / ds)[..., None]
    h00 = 2 * t ** 3 - 3 * t ** 2 + 1
    h10 = t ** 3 - 2 * t ** 2 + t
    h01 = -2 * t ** 3 + 3 * t ** 2
    h11 = t ** 3 - t ** 2
    v = h00 * vals[k] + h10 * ds * ders[k] + h01 * vals[k + 1] + h11 * ds * ders[k + 1]
    g00 = 6 * t ** 2 - 6 * t
    g10 = 3 * t ** 2 - 4 * t + 1
    g01 = -6 * t ** 2 + 6 * t
    g11 = 3 * t ** 2 - 2 * t
    dv = (g00 * vals[k] + g01 * vals[k + 1]) / ds + g10 * ders[k] + g11 * ders[k + 1]
    return v, dv


# ----------------------------------------------------------------------------
# Problem set-up: PML profile (Eq. pml-profile), velocity extension, levels
# ----------------------------------------------------------------------------
def pml_gamma(n: int, n_pml: int, gamma_max: float, idx) -> np.ndarray:
    """gamma_j at integer node indices idx of a level with n intervals and
    n_pml PML layers per side (Eq. pml-profile; d measured into the PML)."""
    idx = np.asarray(idx, dtype=np.float64)
    if n_pml == 0:
        return np.zeros_like(idx)
    dist = np.maximum(np.maximum(n_pml - idx, idx - (n - n_pml)), 0.0)
    dist = np.minimum(dist, n_pml)
    return gamma_max * (1.0 - np.cos(math.pi * dist / (2.0 * n_pml)))


def pml_1d(n: int, n_pml: int, gamma_max: float):
    """xi^{-1} at nodes 0..n and at half nodes -1/2 .. n+1/2 (n+2 values);
    half-node stretch from the average of gamma at the adjacent nodes before
    inversion (Sec. 2.2, after Eq. pml-second-difference)."""
    g_node = pml_gamma(n, n_pml, gamma_max, np.arange(-1, n + 2))   # nodes -1..n+1
    xi_inv_node = 1.0 / (1.0 + 1j * g_node[1:-1])
    g_half = 0.5 * (g_node[:-1] + g_node[1:])                        # (i-1/2) for i=0..n+1
    xi_inv_half = 1.0 / (1.0 + 1j * g_half)
    return xi_inv_node, xi_inv_half


def extend_velocity(c: np.ndarray, n_pml: int) -> np.ndarray:
    """Wave speed in the PML = nearest value in the physical box (Sec. 2.1)."""
    nz, ny, nx = (s - 1 for s in c.shape)
    iz = np.clip(np.arange(nz + 1), n_pml, nz - n_pml)
    iy = np.clip(np.arange(ny + 1), n_pml, ny - n_pml)
    ix = np.clip(np.arange(nx + 1), n_pml, nx - n_pml)
    return c[np.ix_(iz, iy, ix)]


def extension_index(shape, n_pml):
    """Flat index of the physical node each node copies its velocity from."""
    nz, ny, nx = (s - 1 for s in shape)
    iz = np.clip(np.arange(nz + 1), n_pml, nz - n_pml)
    iy = np.clip(np.arange(ny + 1), n_pml, ny - n_pml)
    ix = np.clip(np.arange(nx + 1), n_pml, nx - n_pml)
    Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
    return (Z * (ny + 1) + Y) * (nx + 1) + X


@dataclasses.dataclass
class Level:
    """One grid of the hierarchy (Sec. 3.1): spacing ell = 2^L h."""
    L: int
    n: tuple            # (nz, ny, nx) intervals
    n_pml: int
    ell: float
    kappa: np.ndarray   # k(x_i) * ell on this level's nodes
    pml: tuple          # per axis (z, y, x): (xi_inv_node, xi_inv_half)

    @property
    def shape(self):
        return tuple(m + 1 for m in self.n)

    @property
    def eta_star(self):
        return np.minimum(self.kappa / (2.0 * math.pi), ETA_MAX)


@dataclasses.dataclass
class Problem:
    n: tuple
    n_pml: int
    h: float
    omega: float
    gamma_max: float
    c_ext: np.ndarray
    levels: list
    tables: Tables


def make_problem(c, n_pml, h, omega, gamma_max=1.119058, tables=None, nlevels=3) -> Problem:
    c = np.asarray(c, dtype=np.float64)
    n = tuple(s - 1 for s in c.shape)
    for m in n:
        if m % (1 << (nlevels - 1)):
            raise ValueError("intervals must be divisible by 4")
    if n_pml % (1 << (nlevels - 1)):
        raise ValueError("n_pml must be divisible by 4")
    tables = tables or load_tables()
    c_ext = extend_velocity(c, n_pml)
    levels = []
    for L in range(nlevels):
        f = 1 << L
        cL = c_ext[::f, ::f, ::f]
        nL = tuple(m // f for m in n)
        pL = n_pml // f
        ell = h * f
        pml = tuple(pml_1d(m, pL, gamma_max) for m in nL)
        levels.append(Level(L, nL, pL, ell, omega * ell / cL, pml))
    return Problem(n, n_pml, h, omega, gamma_max, c_ext, levels, tables)


class PointKappa:
    """kappa = omega ell / c_ext evaluated on demand at node indices, for grids
    too large to hold whole; c_ext copies the nearest physical node (Sec. 2.1)
    and level L samples fine node 2^L j (Sec. 3.1)."""

    def __init__(self, c, n_pml, omega, ell, stride):
        self.c, self.n_pml, self.omega, self.ell, self.f = c, n_pml, omega, ell, stride
        self.n = tuple(s - 1 for s in c.shape)

    def __getitem__(self, key):
        idx = []
        for i, m in zip(key, self.n):
            idx.append(np.clip(np.asarray(i, dtype=np.int64) * self.f, self.n_pml, m - self.n_pml))
        return self.omega * self.ell / np.asarray(self.c[idx[0], idx[1], idx[2]], dtype=np.float64)


def make_level_points(c, n_pml, h, omega, gamma_max=1.119058, L=0) -> Level:
    """Level L whose kappa is evaluated only where indexed (use with
    ``row_coefficient_points``)."""
    f = 1 << L
    n = tuple((s - 1) // f for s in c.shape)
    pL = n_pml // f
    pml = tuple(pml_1d(m, pL, gamma_max) for m in n)
    return Level(L, n, pL, h * f, PointKappa(c, n_pml, omega, h * f, f), pml)


# ----------------------------------------------------------------------------
# Row coefficients A_i(delta) of the PML-stretched IOFD operator
# ----------------------------------------------------------------------------
def _pml_d(level: Level, axis: int, dj: int) -> np.ndarray:
    """d_{j,i}(delta_j) along one axis: the coefficients of the 1-D PML second
    difference (Eq. pml-second-difference) times ell^2, as a 1-D array over
    the node index of that axis."""
    xin, xih = level.pml[axis]
    plus = xin * xih[1:]      # xi_i^{-1} xi_{i+1/2}^{-1}
    minus = xin * xih[:-1]    # xi_i^{-1} xi_{i-1/2}^{-1}
    if dj == 1:
        return plus
    if dj == -1:
        return minus
    return -(plus + minus)


def _bcast(v1d, axis):
    shape = [1, 1, 1]
    shape[axis] = -1
    return v1d.reshape(shape)


def row_coefficient(level: Level, tables: Tables, delta, shift_sigma: float = 0.0,
                    mass_scale: float = 1.0):
    """A_i(delta) for every row i of B = L - (1 + i sigma) M  (sigma = 0 gives A).

    Tensor-product IOFD row (Sec. 2.2): each directional second difference
    D_j is replaced by its PML form, with transverse weights a4, a5/4,
    (1-a4-a5)/4 for 0, 1, 2 nonzero transverse offsets, and mass weights
    a1, a2/6, a3/12, (1-a1-a2-a3)/8 on the four shells; alpha is evaluated
    at the row's own eta* (Eq. iofd-clamped-coordinate) and the unclamped
    kappa^2 multiplies the mass (Eq. shifted-iofd-levels for the shift)."""
    a, _ = hermite(tables.s, tables.alpha, tables.dalpha, level.eta_star)
    a1, a2, a3, a4, a5 = (a[..., j] for j in range(5))
    tw = {0: a4, 1: a5 / 4.0, 2: (1.0 - a4 - a5) / 4.0}
    mw = {0: a1, 1: a2 / 6.0, 2: a3 / 12.0, 3: (1.0 - a1 - a2 - a3) / 8.0}
    stiff = np.zeros(level.shape, dtype=np.complex128)
    for axis in range(3):
        others = [delta[k] for k in range(3) if k != axis]
        nnz_t = sum(1 for o in others if o != 0)
        stiff = stiff + _bcast(_pml_d(level, axis, delta[axis]), axis) * tw[nnz_t]
    m = sum(1 for o in delta if o != 0)
    mass = (1.0 + 1j * shift_sigma) * mass_scale * level.kappa ** 2 * mw[m]
    return (-stiff - mass) / level.ell ** 2


def row_coefficient_points(level: Level, tables: Tables, delta, iz, iy, ix, shift_sigma: float = 0.0):
    """A_i(delta) of ``row_coefficient`` at the nodes (iz, iy, ix) only (for
    sampled checks on grids too large to evaluate whole): the same
    tensor-product row with the PML factors of each node's own coordinates."""
    iz, iy, ix = (np.asarray(v, dtype=np.int64) for v in (iz, iy, ix))
    kap = level.kappa[iz, iy, ix]
    eta = np.minimum(kap / (2.0 * math.pi), ETA_MAX)
    a, _ = hermite(tables.s, tables.alpha, tables.dalpha, eta)
    a1, a2, a3, a4, a5 = (a[..., j] for j in range(5))
    tw = {0: a4, 1: a5 / 4.0, 2: (1.0 - a4 - a5) / 4.0}
    mw = {0: a1, 1: a2 / 6.0, 2: a3 / 12.0, 3: (1.0 - a1 - a2 - a3) / 8.0}
    coords = (iz, iy, ix)
    stiff = np.zeros(kap.shape, dtype=np.complex128)
    for axis in range(3):
        others = [delta[k] for k in range(3) if k != axis]
        nnz_t = sum(1 for o in others if o != 0)
        stiff = stiff + _pml_d(level, axis, delta[axis])[coords[axis]] * tw[nnz_t]
    m = sum(1 for o in delta if o != 0)
    mass = (1.0 + 1j * shift_sigma) * kap ** 2 * mw[m]
    return (-stiff - mass) / level.ell ** 2


def apply_points(level: Level, tables: Tables, x_at, iz, iy, ix, shift_sigma: float = 0.0):
    """(A x)_i at the nodes (iz, iy, ix); ``x_at(dz, dy, dx)`` returns x at the
    neighbours (zero outside the grid)."""
    y = 0.0
    for d in OFFSETS:
        y = y + row_coefficient_points(level, tables, d, iz, iy, ix, shift_sigma) * x_at(*d)
    return y


def shift_field(v: np.ndarray, delta) -> np.ndarray:
    """out[i] = v[i + delta], zero where i + delta leaves the grid (u = 0)."""
    out = np.zeros_like(v)
    src = []
    dst = []
    for d, size in zip(delta, v.shape):
        if d >= 0:
            src.append(slice(d, size))
            dst.append(slice(0, size - d))
        else:
            src.append(slice(0, size + d))
            dst.append(slice(-d, size))
    out[tuple(dst)] = v[tuple(src)]
    return out


class StencilOp:
    """Matrix-free 27-point operator y_i = sum_delta C_i(delta) x_{i+delta}."""

    def __init__(self, coeff_fn, shape, cache=True):
        self.coeff_fn = coeff_fn
        self.shape = shape
        self._cache = {d: coeff_fn(d) for d in OFFSETS} if cache else None

    def coeff(self, delta):
        return self._cache[delta] if self._cache is not None else self.coeff_fn(delta)

    def diag(self):
        return self.coeff((0, 0, 0))

    def __call__(self, x):
        x = x.reshape(self.shape)
        y = np.zeros(self.shape, dtype=np.complex128)
        for d in OFFSETS:
            y += self.coeff(d) * shift_field(x, d)
        return y

    def adjoint(self, x):
        """(H^H x)_i = sum_delta conj(C_{i+delta}(-delta)) x_{i+delta}."""
        x = x.reshape(self.shape)
        y = np.zeros(self.shape, dtype=np.complex128)
        for d in OFFSETS:
            md = tuple(-v for v in d)
            y += shift_field(np.conj(self.coeff(md)) * x, d)
        return y


def operator_A(prob: Problem, L: int = 0, sigma: float = 0.0, cache=True) -> StencilOp:
    """A_ell (sigma = 0, Eq. physical-iofd-levels) or B_ell (Eq. shifted-iofd-levels)."""
    lev = prob.levels[L]
    return StencilOp(lambda d: row_coefficient(lev, prob.tables, d, sigma), lev.shape, cache)


def q_coefficient(level: Level, tables: Tables, delta):
    """Q_h row (Eq. q-shell-coefficients, Eq. q-operator): shell weight at the
    row's eta*_h."""
    b, _ = hermite(tables.s, tables.beta, tables.dbeta, level.eta_star)
    b1, b2, b3 = b[..., 0], b[..., 1], b[..., 2]
    qw = {0: b1, 1: b2 / 6.0, 2: b3 / 12.0, 3: (1.0 - b1 - b2 - b3) / 8.0}
    m = sum(1 for o in delta if o != 0)
    return qw[m].astype(np.complex128)


def operator_Q(prob: Problem, cache=True) -> StencilOp:
    lev = prob.levels[0]
    return StencilOp(lambda d: q_coefficient(lev, prob.tables, d), lev.shape, cache)


def point_sources(prob: Problem, sources) -> np.ndarray:
    """f_h = h^{-3} delta_{i, i_s} per source (Eq. point-source); one column per
    source, returned as (nsrc, *shape)."""
    shape = prob.levels[0].shape
    F = np.zeros((len(sources),) + shape, dtype=np.complex128)
    for s, (ix, iy, iz, amp) in enumerate(sources):
        F[s, iz, iy, ix] = amp / prob.h ** 3
    return F


# ----------------------------------------------------------------------------
# Independent assembled builder: Kronecker products of 1-D matrices
# ----------------------------------------------------------------------------
def _shift_sum_1d(m):
    """S = forward + backward shift on m+1 nodes (zero outside)."""
    e = np.ones(m)
    return sp.diags([e, e], [-1, 1], shape=(m + 1, m + 1), format="csr")


def _pml_second_difference_1d(level: Level, axis: int):
    """ell^2 D^pml_j as an (m+1)x(m+1) matrix (Eq. pml-second-difference)."""
    m = level.n[axis]
    xin, xih = level.pml[axis]
    main = -xin * (xih[1:] + xih[:-1])
    up = (xin * xih[1:])[:-1]      # row i, column i+1
    lo = (xin * xih[:-1])[1:]      # row i, column i-1
    return sp.diags([lo, main, up], [-1, 0, 1], shape=(m + 1, m + 1), format="csr")


def assemble(prob: Problem, L: int = 0, sigma: float = 0.0, which: str = "A") -> sp.csr_matrix:
    """Sparse matrix of A_ell / B_ell (which='A') or Q_h (which='Q'), built as
    sums of Kronecker products: stiffness  -ell^-2 sum_j diag(t) (D_j (x) S_perp),
    mass  -(1+i sigma) ell^-2 diag(kappa^2 w_m) N_m with the shell-sum matrices
    N_0 = I(x)I(x)I, N_1 = S(x)I(x)I + ..., N_3 = S(x)S(x)S.  Independent of the
    row formula used by the matrix-free operator."""
    lev = prob.levels[L]
    nz, ny, nx = lev.n
    I = [sp.identity(m + 1, format="csr", dtype=np.complex128) for m in (nz, ny, nx)]
    S = [_shift_sum_1d(m).astype(np.complex128) for m in (nz, ny, nx)]

    def kron3(mz, my, mx):
        return sp.kron(sp.kron(mz, my), mx, format="csr")

    # shell-sum matrices N_m (number of nonzero offsets = m)
    N = {m: None for m in range(4)}
    for pick in itertools.product((0, 1), repeat=3):
        mats = [S[a] if pick[a] else I[a] for a in range(3)]
        K = kron3(*mats)
        m = sum(pick)
        N[m] = K if N[m] is None else N[m] + K
    if which == "Q":
        b, _ = hermite(prob.tables.s, prob.tables.beta, prob.tables.dbeta, lev.eta_star)
        b1, b2, b3 = b[..., 0], b[..., 1], b[..., 2]
        w = [b1, b2 / 6, b3 / 12, (1 - b1 - b2 - b3) / 8]
        return sum(sp.diags(w[m].ravel().astype(np.complex128)) @ N[m] for m in range(4)).tocsr()
    a, _ = hermite(prob.tables.s, prob.tables.alpha, prob.tables.dalpha, lev.eta_star)
    a1, a2, a3, a4, a5 = (a[..., j].ravel() for j in range(5))
    tw = [a4, a5 / 4, (1 - a4 - a5) / 4]
    mw = [a1, a2 / 6, a3 / 12, (1 - a1 - a2 - a3) / 8]
    D = [_pml_second_difference_1d(lev, ax) for ax in range(3)]
    stiff = None
    for ax in range(3):
        oth = [o for o in range(3) if o != ax]
        for pick in itertools.product((0, 1), repeat=2):
            mats = [None, None, None]
            mats[ax] = D[ax]
            for o, p in zip(oth, pick):
                mats[o] = S[o] if p else I[o]
            K = sp.diags(tw[sum(pick)].astype(np.complex128)) @ kron3(*mats)
            stiff = K if stiff is None else stiff + K
    k2 = (lev.kappa ** 2).ravel()
    mass = sum(sp.diags((k2 * mw[m]).astype(np.complex128)) @ N[m] for m in range(4))
    return ((-stiff - (1 + 1j * sigma) * mass) / lev.ell ** 2).tocsr()
