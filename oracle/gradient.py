"""Oracle: receiver misfit and adjoint-state gradient -- test infrastructure.

Discretise-then-differentiate on the IOFD system of Eq. iofd-complete-system:
for each source s,  A v_s = Q f_s,  u_s = Q v_s,  and the misfit
J(m) = 1/2 sum_s || R u_s - d_s ||^2, with m = 1/c^2 the squared slowness
(so kappa^2 = omega^2 h^2 m) and R the restriction to receiver nodes.

With r_s = R^T (R u_s - d_s) and lambda_s = A^{-H} Q^H r_s,
  dJ/dm_i = sum_s Re[ conj(lambda_s,i) ( (dQ_i f_s) - (dA_i v_s) ) ]
          + Re[ conj(r_s,i) (dQ_i v_s) ],
where dA_i, dQ_i are the derivatives of row i of A and Q with respect to m_i
(each row depends only on its own node, Sec. 2.2).  The velocity in the PML
copies the nearest physical node (Sec. 2.1), so the derivative at a PML node
is added to that node.  The eta* clamp at 0.4 has zero derivative above it.
The preconditioner does not change v, so only A_h and Q_h enter.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse.linalg as spla

from . import iofd


def _eta_dm(level: iofd.Level, m: np.ndarray):
    """d eta* / d m at each node (0 where the clamp is active)."""
    eta = level.kappa / (2 * math.pi)
    d = level.kappa / (4 * math.pi * m)
    return np.where(eta < iofd.ETA_MAX, d, 0.0)


def row_coefficient_dm(prob: iofd.Problem, m: np.ndarray, delta):
    """d A_i(delta) / d m_i on the fine level (A unshifted)."""
    lev = prob.levels[0]
    T = prob.tables
    a, da = iofd.hermite(T.s, T.alpha, T.dalpha, lev.eta_star)
    deta = _eta_dm(lev, m)
    a1, a2, a3, a4, a5 = (a[..., j] for j in range(5))
    d1, d2, d3, d4, d5 = (da[..., j] * deta for j in range(5))
    tw = {0: d4, 1: d5 / 4.0, 2: (-d4 - d5) / 4.0}
    mw = {0: a1, 1: a2 / 6.0, 2: a3 / 12.0, 3: (1.0 - a1 - a2 - a3) / 8.0}
    dmw = {0: d1, 1: d2 / 6.0, 2: d3 / 12.0, 3: (-d1 - d2 - d3) / 8.0}
    stiff = np.zeros(lev.shape, dtype=np.complex128)
    for axis in range(3):
        others = [delta[k] for k in range(3) if k != axis]
        nnz_t = sum(1 for o in others if o != 0)
        stiff = stiff + iofd._bcast(iofd._pml_d(lev, axis, delta[axis]), axis) * tw[nnz_t]
    k = sum(1 for o in delta if o != 0)
    dk2 = (prob.omega * lev.ell) ** 2
    mass = dk2 * mw[k] + lev.kappa ** 2 * dmw[k]
    return (-stiff - mass) / lev.ell ** 2


def q_coefficient_dm(prob: iofd.Problem, m: np.ndarray, delta):
    lev = prob.levels[0]
    T = prob.tables
    _, db = iofd.hermite(T.s, T.beta, T.dbeta, lev.eta_star)
    deta = _eta_dm(lev, m)
    d1, d2, d3 = (db[..., j] * deta for j in range(3))
    qw = {0: d1, 1: d2 / 6.0, 2: d3 / 12.0, 3: (-d1 - d2 - d3) / 8.0}
    k = sum(1 for o in delta if o != 0)
    return qw[k].astype(np.complex128)


def row_local_apply(coeff_fn, x):
    """y_i = sum_delta C_i(delta) x_{i+delta} for a row-local coefficient field."""
    y = np.zeros(x.shape, dtype=np.complex128)
    for d in iofd.OFFSETS:
        y += coeff_fn(d) * iofd.shift_field(x, d)
    return y


def receiver_matrix_apply(u, rec):
    """R u: values at receiver nodes rec (nrec, 3) = (ix, iy, iz)."""
    return u[rec[:, 2], rec[:, 1], rec[:, 0]]


def receiver_adjoint(vals, rec, shape):
    out = np.zeros(shape, dtype=np.complex128)
    np.add.at(out, (rec[:, 2], rec[:, 1], rec[:, 0]), vals)
    return out


def direct_solver(prob: iofd.Problem):
    """Sparse LU of A_h (small grids only): returns (solve, solve_adjoint)."""
    A = iofd.assemble(prob, 0, 0.0).tocsc()
    lu = spla.splu(A)
    shape = prob.levels[0].shape

    def fwd(b):
        return lu.solve(b.ravel()).reshape(shape)

    def adj(b):
        return lu.solve(b.ravel(), trans="H").reshape(shape)
    return fwd, adj


def misfit_and_gradient(c, n_pml, h, omega, sources, rec, d_obs, gamma_max=1.119058,
                        tables=None, solver=None):
    """Return (J, dJ/dm on every fine node, fields) for m = 1/c^2.

    ``solver(prob)`` returns (solve, solve_adjoint) callables; the default is
    the sparse direct solver.  ``d_obs`` has shape (nsrc, nrec)."""
    c = np.asarray(c, dtype=np.float64)
    prob = iofd.make_problem(c, n_pml, h, omega, gamma_max, tables)
    solve, solve_adj = (solver or direct_solver)(prob)
    Q = iofd.operator_Q(prob)
    F = iofd.point_sources(prob, sources)
    m_ext = 1.0 / prob.c_ext ** 2
    shape = prob.levels[0].shape
    g_ext = np.zeros(shape)
    J = 0.0
    fields = []
    dA = {d: row_coefficient_dm(prob, m_ext, d) for d in iofd.OFFSETS}
    dQ = {d: q_coefficient_dm(prob, m_ext, d) for d in iofd.OFFSETS}
    for s in range(F.shape[0]):
        b = Q(F[s])
        v = solve(b)
        u = Q(v)
        res = receiver_matrix_apply(u, rec) - d_obs[s]
        J += 0.5 * float(np.sum(np.abs(res) ** 2))
        r = receiver_adjoint(res, rec, shape)
        lam = solve_adj(Q.adjoint(r))
        dQf = row_local_apply(lambda d: dQ[d], F[s])
        dAv = row_local_apply(lambda d: dA[d], v)
        dQv = row_local_apply(lambda d: dQ[d], v)
        g_ext += np.real(np.conj(lam) * (dQf - dAv)) + np.real(np.conj(r) * dQv)
        fields.append((v, u, lam))
    g = np.zeros(shape).ravel()
    np.add.at(g, iofd.extension_index(shape, n_pml).ravel(), g_ext.ravel())
    return J, g.reshape(shape), fields


def synthetic_data(c_true, n_pml, h, omega, sources, rec, gamma_max=1.119058, tables=None,
                   solver=None):
    """d_s = R Q A^{-1} Q f_s for the true model."""
    prob = iofd.make_problem(np.asarray(c_true, np.float64), n_pml, h, omega, gamma_max, tables)
    solve, _ = (solver or direct_solver)(prob)
    Q = iofd.operator_Q(prob)
    F = iofd.point_sources(prob, sources)
    return np.stack([receiver_matrix_apply(Q(solve(Q(F[s]))), rec) for s in range(F.shape[0])])


def misfit(c, n_pml, h, omega, sources, rec, d_obs, gamma_max=1.119058, tables=None, solver=None):
    d = synthetic_data(c, n_pml, h, omega, sources, rec, gamma_max, tables, solver)
    return 0.5 * float(np.sum(np.abs(d - d_obs) ** 2))
