"""Oracle: three-grid preconditioner and outer FGMRES (paper Sec. 3) -- test infrastructure.

Plain complex128 NumPy, following the definitions in the order the paper
states them: transfers (Eq. linear-prolongation, Eq. full-weighting), damped
Jacobi (Eq. jacobi-map), the bottom Krylov solve C_4h, the shifted V-cycle
(Eq. shifted-auxiliary-cycle), the unshifted 2h solve (Eq.
unshifted-middle-solve), the fine smoother S_h, Algorithm 1 and the outer
FGMRES with the stopping test of Eq. relative-residual.  Parameters default
to Table 4.

Readings:
* The m_4h CA-GMRES steps of C_4h produce, in exact arithmetic, the GMRES
  iterate of the same Krylov space; the oracle runs plain GMRES(m_4h).
* Orthogonalisation is modified Gram-Schmidt and the small least-squares
  problem is solved by a library lstsq (the paper names neither).
* A zero residual (or an exact Arnoldi breakdown) ends a Krylov cycle early
  and returns the current iterate.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import iofd


@dataclasses.dataclass
class Params:
    """Table 4 of the paper."""
    tol: float = 1e-4
    max_pc: int = 500
    m_out: int = 5
    m_h: int = 2
    nJ_h: int = 2
    w_h: float = 0.8
    c_2h: int = 2
    m_2h: int = 10
    nJ_2h: int = 2
    w_2h: float = 0.8
    m_4h: int = 4
    nJ_4h: int = 2
    w_4h: float = 0.2
    sigma: float = 0.9


# ----------------------------------------------------------------------------
# Grid transfers
# ----------------------------------------------------------------------------
def _restrict_axis(v, axis):
    v = np.moveaxis(v, axis, 0)
    m = v.shape[0] - 1
    mc = m // 2
    out = 0.5 * v[0::2]
    out[:mc] += 0.25 * v[1::2]          # v_{2j+1}
    out[1:] += 0.25 * v[1::2]           # v_{2j-1}
    return np.moveaxis(out, 0, axis)


def _prolong_axis(w, axis):
    w = np.moveaxis(w, axis, 0)
    mc = w.shape[0] - 1
    out = np.zeros((2 * mc + 1,) + w.shape[1:], dtype=w.dtype)
    out[0::2] = w
    out[1::2] = 0.5 * (w[:-1] + w[1:])
    return np.moveaxis(out, 0, axis)


def restrict(v):
    """Full weighting (1/4, 1/2, 1/4) per axis, tensorised (Eq. full-weighting)."""
    for ax in range(3):
        v = _restrict_axis(v, ax)
    return v


def prolong(w):
    """Trilinear interpolation (Eq. linear-prolongation), tensorised."""
    for ax in range(3):
        w = _prolong_axis(w, ax)
    return w


# ----------------------------------------------------------------------------
# Damped Jacobi and Krylov cycles
# ----------------------------------------------------------------------------
def jacobi(H, g, omega_J, nJ):
    """n_J damped Jacobi sweeps from zero (Eq. jacobi-map)."""
    D = H.diag()
    y = np.zeros_like(g)
    for _ in range(nJ):
        y = y + omega_J * (g - H(y)) / D
    return y


def dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def norm(a):
    return float(np.sqrt(np.real(dot(a, a))))


def fgmres_cycle(A, M, g, x0, m):
    """One (flexible) right-preconditioned GMRES cycle of m steps for A x = g
    from x0: Arnoldi on A M with the preconditioned directions z_j = M(v_j)
    kept, y = argmin ||beta e_1 - H y||, x = x0 + Z y."""
    r0 = g - A(x0) if x0 is not None else g.copy()
    x0 = np.zeros_like(g) if x0 is None else x0
    beta = norm(r0)
    if beta == 0.0:
        return x0
    V = [r0 / beta]
    Z = []
    Hm = np.zeros((m + 1, m), dtype=np.complex128)
    k = m
    for j in range(m):
        z = M(V[j])
        Z.append(z)
        w = A(z)
        for i in range(j + 1):
            Hm[i, j] = dot(V[i], w)
            w = w - Hm[i, j] * V[i]
        Hm[j + 1, j] = norm(w)
        if Hm[j + 1, j] == 0.0:
            k = j + 1
            break
        V.append(w / Hm[j + 1, j])
    e1 = np.zeros(k + 1, dtype=np.complex128)
    e1[0] = beta
    y = np.linalg.lstsq(Hm[:k + 1, :k], e1, rcond=None)[0]
    x = x0.copy()
    for j in range(k):
        x = x + y[j] * Z[j]
    return x


class ThreeGrid:
    """The three-grid preconditioner z = M_h^{-1} r of Algorithm 1."""

    def __init__(self, prob: iofd.Problem, params: Params = Params(), cache=True, adjoint=False):
        self.p = params
        self.adjoint = adjoint
        s = params.sigma
        self.A_h = iofd.operator_A(prob, 0, 0.0, cache)
        self.A_2h = iofd.operator_A(prob, 1, 0.0, cache)
        self.B_2h = iofd.operator_A(prob, 1, s, cache)
        self.B_4h = iofd.operator_A(prob, 2, s, cache)

    def op(self, H):
        return H.adjoint if self.adjoint else H

    def diag(self, H):
        return np.conj(H.diag()) if self.adjoint else H.diag()

    def J(self, H, g, omega_J, nJ):
        """Jacobi sweeps for H or, for the adjoint hierarchy, H^H (same diagonal
        conjugated)."""
        Hop, D = self.op(H), self.diag(H)
        y = np.zeros_like(g)
        for _ in range(nJ):
            y = y + omega_J * (g - Hop(y)) / D
        return y

    def C_4h(self, g):
        p = self.p
        B = self.op(self.B_4h)
        return fgmres_cycle(B, lambda v: self.J(self.B_4h, v, p.w_4h, p.nJ_4h), g, None, p.m_4h)

    def V_2h(self, q):
        """Shifted 2h-4h cycle, Eq. shifted-auxiliary-cycle."""
        p = self.p
        B = self.op(self.B_2h)
        y = self.J(self.B_2h, q, p.w_2h, p.nJ_2h)
        q4 = restrict(q - B(y))
        e4 = self.C_4h(q4)
        yt = y + prolong(e4)
        return yt + self.J(self.B_2h, q - B(yt), p.w_2h, p.nJ_2h)

    def K_2h(self, r2):
        """c_2h restarted FGMRES(m_2h) cycles on A_2h from zero, Eq. unshifted-middle-solve."""
        p = self.p
        A = self.op(self.A_2h)
        x = None
        for _ in range(p.c_2h):
            x = fgmres_cycle(A, self.V_2h, r2, x, p.m_2h)
        return x

    def S_h(self, g, x0):
        p = self.p
        A = self.op(self.A_h)
        return fgmres_cycle(A, lambda v: self.J(self.A_h, v, p.w_h, p.nJ_h), g, x0, p.m_h)

    def __call__(self, r):
        A = self.op(self.A_h)
        z_pre = self.S_h(r, None)                    # step 1
        r2 = restrict(r - A(z_pre))                  # step 2
        e2 = self.K_2h(r2)                           # step 3
        z_t = z_pre + prolong(e2)                    # step 4
        return self.S_h(r, z_t)                      # step 5


@dataclasses.dataclass
class SolveInfo:
    pc_calls: int
    rel_res: float
    history: list


def fgmres_solve(A, M, b, params: Params = Params(), x0=None):
    """Outer FGMRES(m_out), right preconditioner M, stopping test
    ||A v - b|| / ||b|| <= tol (Eq. relative-residual).  Each Arnoldi step
    calls M once; the estimate from the Givens-reduced Hessenberg decides
    when to leave a cycle and the true residual decides convergence."""
    bn = norm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if bn == 0.0:
        return x, SolveInfo(0, 0.0, [])
    pc = 0
    hist = []
    r = b - A(x)
    rel = norm(r) / bn
    hist.append(rel)
    while rel > params.tol and pc < params.max_pc:
        m = params.m_out
        beta = norm(r)
        V = [r / beta]
        Z = []
        Hm = np.zeros((m + 1, m), dtype=np.complex128)
        k = 0
        for j in range(m):
            if pc >= params.max_pc:
                break
            z = M(V[j])
            pc += 1
            Z.append(z)
            w = A(z)
            for i in range(j + 1):
                Hm[i, j] = dot(V[i], w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = norm(w)
            k = j + 1
            e1 = np.zeros(k + 1, dtype=np.complex128)
            e1[0] = beta
            y = np.linalg.lstsq(Hm[:k + 1, :k], e1, rcond=None)[0]
            est = norm_vec(e1 - Hm[:k + 1, :k] @ y) / bn
            if Hm[j + 1, j] == 0.0 or est <= params.tol:
                break
            V.append(w / Hm[j + 1, j])
        if k == 0:
            break
        e1 = np.zeros(k + 1, dtype=np.complex128)
        e1[0] = beta
        y = np.linalg.lstsq(Hm[:k + 1, :k], e1, rcond=None)[0]
        for j in range(k):
            x = x + y[j] * Z[j]
        r = b - A(x)
        rel = norm(r) / bn
        hist.append(rel)
    return x, SolveInfo(pc, rel, hist)


def norm_vec(v):
    return float(np.sqrt(np.sum(np.abs(v) ** 2)))


# ----------------------------------------------------------------------------
# Block flexible GMRES over s right-hand sides (the block Krylov method for
# multiple right-hand sides named as future work in Sec. 7).  One basis serves
# all right-hand sides: the block residual R_0 = V_0 R_hat (thin QR), then per
# step the preconditioned block Z_j = M(V_j) (column by column: flexible), the
# block W = A Z_j orthogonalised against V_0 .. V_j by block modified
# Gram-Schmidt and factored W = V_{j+1} H_{j+1,j} (thin QR), and the columns
# of Y minimise ||E - H Y|| column by column with E = [R_hat; 0], so each
# right-hand side gets the minimal residual over the whole block space.
# ----------------------------------------------------------------------------
def _block_cycle_steps(A, M, G, X0, m, tol_cols=None, bn=None, on_step=None):
    """Shared body of one block cycle; returns (X, steps, breakdown)."""
    s = G.shape[0]
    shape = G.shape[1:]
    R0 = np.stack([G[c] - A(X0[c]) for c in range(s)]).reshape(s, -1).T   # n x s
    V0, Rh = np.linalg.qr(R0)
    V = [V0]
    Z = []
    Hb = np.zeros(((m + 1) * s, m * s), dtype=np.complex128)
    E = np.zeros(((m + 1) * s, s), dtype=np.complex128)
    E[:s] = Rh
    k = 0
    breakdown = False
    for j in range(m):
        Zj = np.stack([M(V[j][:, c].reshape(shape)).ravel() for c in range(s)], axis=1)
        Z.append(Zj)
        if on_step is not None:
            on_step()
        W = np.stack([A(Zj[:, c].reshape(shape)).ravel() for c in range(s)], axis=1)
        for i in range(j + 1):
            Hij = V[i].conj().T @ W
            W = W - V[i] @ Hij
            Hb[i * s:(i + 1) * s, j * s:(j + 1) * s] = Hij
        Vn, Hn = np.linalg.qr(W)
        Hb[(j + 1) * s:(j + 2) * s, j * s:(j + 1) * s] = Hn
        k = j + 1
        d = np.abs(np.diag(Hn))
        if d.min() <= 1e-14 * max(d.max(), 1e-300):
            breakdown = True
            break
        if tol_cols is not None:
            Y = np.linalg.lstsq(Hb[:(k + 1) * s, :k * s], E[:(k + 1) * s], rcond=None)[0]
            res = E[:(k + 1) * s] - Hb[:(k + 1) * s, :k * s] @ Y
            est = np.sqrt(np.sum(np.abs(res) ** 2, axis=0))
            if np.all(est <= tol_cols):
                break
        V.append(Vn)
    Y = np.linalg.lstsq(Hb[:(k + 1) * s, :k * s], E[:(k + 1) * s], rcond=None)[0]
    Zm = np.concatenate(Z[:k], axis=1)
    X = X0.reshape(s, -1) + (Zm @ Y).T
    return X.reshape(G.shape), k, breakdown


def block_fgmres_cycle(A, M, G, X0, m):
    """One block FGMRES cycle of m block steps for A X = G (G: s fields
    stacked on axis 0) from X0."""
    X0 = np.zeros_like(G) if X0 is None else X0
    return _block_cycle_steps(A, M, G, X0, m)[0]


def block_fgmres_solve(A, M, B, params: Params = Params(), X0=None):
    """Block FGMRES(m_out) for s right-hand sides B (axis 0), right
    preconditioner M applied column by column; stopping test
    ||A x_c - b_c|| / ||b_c|| <= tol for every column c (Eq.
    relative-residual).  pc_calls counts block steps (each applies M to the
    s columns of one basis block)."""
    s = B.shape[0]
    bn = np.array([norm(B[c]) for c in range(s)])
    X = np.zeros_like(B) if X0 is None else X0.copy()
    pc = 0
    hist = []

    def rel_of(X):
        return max((norm(B[c] - A(X[c])) / bn[c]) if bn[c] > 0 else 0.0 for c in range(s))

    rel = rel_of(X)
    hist.append(rel)
    while rel > params.tol and pc < params.max_pc:
        m = min(params.m_out, params.max_pc - pc)
        counter = [0]

        def step():
            counter[0] += 1
        X, k, _ = _block_cycle_steps(A, M, B, X, m, tol_cols=params.tol * bn, bn=bn, on_step=step)
        pc += counter[0]
        rel = rel_of(X)
        hist.append(rel)
        if k == 0:
            break
    return X, SolveInfo(pc, rel, hist)


def solve(prob: iofd.Problem, b, params: Params = Params(), cache=True):
    """v = A_h^{-1} b by FGMRES right-preconditioned with Algorithm 1."""
    M = ThreeGrid(prob, params, cache)
    return fgmres_solve(M.A_h, M, b, params)


def solve_adjoint(prob: iofd.Problem, b, params: Params = Params(), cache=True):
    """lambda = A_h^{-H} b by FGMRES right-preconditioned with the same
    three-grid structure built from the adjoint level operators."""
    M = ThreeGrid(prob, params, cache, adjoint=True)
    return fgmres_solve(M.A_h.adjoint, M, b, params)
