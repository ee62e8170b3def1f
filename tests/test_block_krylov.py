"""Pins of the oracle's block flexible GMRES (block Krylov for multiple
right-hand sides, the future work of Sec. 7) against what the mathematics
fixes: one cycle is the column-wise least-squares minimiser over the block
Krylov space, which contains every column's own Krylov space; an exact
preconditioner solves in one block step; the solve loop reaches the sparse
direct solution of the discrete Helmholtz problem."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import hz_workloads as W
from oracle import iofd
from oracle import threegrid as tg


def _dense_case(n=60, s=3, seed=4):
    rng = np.random.default_rng(seed)
    A = 4.0 * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    d = 1.0 + 0.5 * rng.random(n)                        # fixed diagonal right preconditioner
    G = rng.standard_normal((s, n)) + 1j * rng.standard_normal((s, n))
    X0 = 0.1 * (rng.standard_normal((s, n)) + 1j * rng.standard_normal((s, n)))
    return A, d, G, X0


def _block_minimiser(A, d, G, X0, m):
    """Brute force: the explicit block Krylov matrix K = [R0, (AM) R0, ...,
    (AM)^{m-1} R0] and, per column, Y = argmin ||R0 - A M K Y||."""
    R0 = (G - X0 @ A.T).T                  # n x s
    AM = A * d[None, :]
    blocks = [R0]
    for _ in range(m - 1):
        blocks.append(AM @ blocks[-1])
    K = np.concatenate(blocks, axis=1)
    Y = np.linalg.lstsq(AM @ K, R0, rcond=None)[0]
    return X0 + ((d[:, None] * K) @ Y).T


@pytest.mark.parametrize("m", [1, 2, 4])
def test_block_cycle_is_the_block_krylov_minimiser(m):
    A, d, G, X0 = _dense_case()
    X = tg.block_fgmres_cycle(lambda x: A @ x, lambda v: d * v, G, X0, m)
    ref = _block_minimiser(A, d, G, X0, m)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-11


def test_block_minimiser_pin_is_sharp():
    """The minimiser over m blocks differs clearly from the one over m - 1
    blocks and from each column's own m-step FGMRES iterate (so a dropped
    block, an off-by-one in the steps or a per-column basis fails the pin);
    the block residual is never larger than the column's own."""
    A, d, G, X0 = _dense_case()
    m = 3
    full = _block_minimiser(A, d, G, X0, m)
    short = _block_minimiser(A, d, G, X0, m - 1)
    assert np.linalg.norm(full - short) / np.linalg.norm(full) > 1e-3
    for c in range(G.shape[0]):
        own = tg.fgmres_cycle(lambda x: A @ x, lambda v: d * v, G[c], X0[c], m)
        assert np.linalg.norm(full[c] - own) / np.linalg.norm(own) > 1e-3
        r_block = np.linalg.norm(G[c] - A @ full[c])
        r_own = np.linalg.norm(G[c] - A @ own)
        assert r_block <= r_own * (1 + 1e-12)


def test_block_cycle_with_an_exact_preconditioner_solves_in_one_step():
    A, d, G, X0 = _dense_case()
    X = tg.block_fgmres_cycle(lambda x: A @ x, lambda v: np.linalg.solve(A, v), G, X0, 1)
    ref = np.linalg.solve(A, G.T).T
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-12


def test_block_cycle_single_column_is_fgmres():
    A, d, G, X0 = _dense_case(s=1)
    X = tg.block_fgmres_cycle(lambda x: A @ x, lambda v: d * v, G, X0, 4)
    ref = tg.fgmres_cycle(lambda x: A @ x, lambda v: d * v, G[0], X0[0], 4)
    assert np.linalg.norm(X[0] - ref) / np.linalg.norm(ref) < 1e-12


def test_block_solve_reaches_the_sparse_direct_solution():
    """Block FGMRES(5) right-preconditioned with Algorithm 1 on three point
    sources of a random medium (16^3 + 4 PML) meets tol on every column and
    agrees with the sparse direct solutions."""
    w = W.random_field(n=16, n_pml=4, nsrc=2, nrec_side=4)
    prob = iofd.make_problem(w.c, w.n_pml, w.h, w.omega)
    Q = iofd.operator_Q(prob)
    srcs = [(8, 8, 8, 1.0), (5, 9, 7, 0.5 - 1j), (11, 6, 10, 2.0)]
    B = np.stack([Q(iofd.point_sources(prob, [s])[0]) for s in srcs])
    M = tg.ThreeGrid(prob, tg.Params(tol=1e-10))
    X, info = tg.block_fgmres_solve(M.A_h, M, B, tg.Params(tol=1e-10))
    assert info.rel_res <= 1e-10
    Ad = iofd.assemble(prob).tocsc()
    for c in range(len(srcs)):
        vd = spla.spsolve(Ad, B[c].ravel())
        assert np.linalg.norm(X[c].ravel() - vd) / np.linalg.norm(vd) < 1e-8
