"""Oracle: local Fourier analysis of the IOFD hierarchy (paper Sec. 4) -- test
infrastructure.

Plain NumPy / SciPy restatement of the source-independent diagnostics of
Sec. 4.3-4.4, evaluated with the same IOFD tables as the solver:

* ``shell_coefficients``: C_m^sigma of Eq. iofd-shell-coefficients at
  eta* = min(kappa / 2 pi, 0.4), kappa^2 replaced by (1 + i sigma) kappa^2;
* ``symbol``: the interior symbol b_l^sigma(theta) of Eq. shifted-iofd-symbol,
  in units of ell^-2 (every diagnostic below is a ratio of two symbols of one
  level or carries the level scale explicitly);
* ``smoothing_factor``: mu_l of Eq. lfa-smoothing-factor over the 26 cosine
  vertices of Theta_high;
* ``vcycle_error_norm``: || E_2h^sigma(theta) ||_2 of Eq. lfa-shifted-vcycle
  (8 x 8 harmonic blocks, exact 4h solve, transfers of Eq. lfa-transfer-symbol);
* ``bottom_multiplier``: lambda_4h of Eq. bottom-radius-indicator;
* ``ideal_polynomial_factor``: the degree-m minimax factor of Eq.
  bottom-ideal-gmres-factor by the supporting-half-plane linear program the
  paper describes (64 directions), returning the attained maximum;
* ``threegrid_block``: the 64 x 64 Fourier block of Algorithm 1 over the
  harmonics of Eq. three-grid-harmonics with every Krylov map replaced by a
  prescribed polynomial (closing paragraph of Sec. 4.4; no value printed
  there).

Sampling sets follow the paper's symmetry reduction (sign changes and
coordinate permutations leave every quantity unchanged): angles in
[0, pi/2]^3 (Theta_low) or [0, pi]^3 (full range) with non-decreasing
coordinates, and local samplings nu in [6, 24].
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import iofd

NU_RANGE = (6.0, 24.0)   # Eq. local-ppw-range with contrast <= 4


def kappa_of(level_factor: int, nu):
    """kappa_l = k l = 2 pi (l / h) / nu (Sec. 4.3)."""
    return 2.0 * math.pi * level_factor / np.asarray(nu, dtype=np.float64)


def shell_coefficients(tables: iofd.Tables, kappa, sigma: float = 0.0):
    """C_0..C_3 of Eq. iofd-shell-coefficients (last axis), tables at
    eta* = min(kappa/2pi, 0.4), mass term scaled by (1 + i sigma)."""
    kappa = np.asarray(kappa, dtype=np.float64)
    eta = np.minimum(kappa / (2.0 * math.pi), iofd.ETA_MAX)
    a, _ = iofd.hermite(tables.s, tables.alpha, tables.dalpha, eta)
    a1, a2, a3, a4, a5 = (a[..., j] for j in range(5))
    k2 = (1.0 + 1j * sigma) * kappa ** 2
    c0 = 6 * a4 - k2 * a1
    c1 = -a4 + a5 - k2 * a2 / 6
    c2 = -a5 / 2 + (1 - a4 - a5) / 2 - k2 * a3 / 12
    c3 = -0.75 * (1 - a4 - a5) - k2 * (1 - a1 - a2 - a3) / 8
    return np.stack([c0, c1, c2, c3], axis=-1)


def symbol(C, theta):
    """ell^2 b(theta) of Eq. shifted-iofd-symbol; C (..., 4) broadcast against
    theta (..., 3)."""
    z = np.cos(np.asarray(theta, dtype=np.float64))
    z1, z2, z3 = z[..., 0], z[..., 1], z[..., 2]
    return (C[..., 0] + 2 * C[..., 1] * (z1 + z2 + z3) + 4 * C[..., 2] * (z1 * z2 + z1 * z3 + z2 * z3)
            + 8 * C[..., 3] * z1 * z2 * z3)


def sorted_angles(n_nodes: int, upper: float):
    """One representative per sign-change / permutation orbit: theta_1 <= theta_2
    <= theta_3 on n_nodes uniform nodes of [0, upper]."""
    g = np.linspace(0.0, upper, n_nodes)
    return np.array([(g[i], g[j], g[k]) for i, j, k in
                     itertools.combinations_with_replacement(range(n_nodes), 3)])


def smoothing_factor(tables, level_factor, nu, sigma, omega, n_sweeps):
    """mu_l(nu) of Eq. lfa-smoothing-factor: the modulus of the Jacobi factor
    is separately convex in each cosine, so its supremum over Theta_high is
    attained at the 26 vertices {-1,0,1}^3 minus (1,1,1) of the cosine image."""
    C = shell_coefficients(tables, kappa_of(level_factor, nu), sigma)
    zs = [v for v in itertools.product((-1.0, 0.0, 1.0), repeat=3) if v != (1.0, 1.0, 1.0)]
    theta = np.arccos(np.array(zs))                       # (26, 3)
    b = symbol(C[..., None, :], theta)                   # (..., 26)
    d = C[..., 0][..., None]
    return np.max(np.abs(1.0 - omega * b / d) ** n_sweeps, axis=-1)


def transfer_column(theta):
    """p_hat of Eq. lfa-transfer-symbol: (..., 8) over the harmonics p in {0,1}^3."""
    ps = np.array(list(itertools.product((0, 1), repeat=3)), dtype=np.float64)   # (8, 3)
    th = np.asarray(theta)[..., None, :] + math.pi * ps                           # (..., 8, 3)
    return np.prod((1.0 + np.cos(th)) / 2.0, axis=-1), th


def vcycle_error_norm(tables, nu, theta, sigma, omega, n_sweeps):
    """|| E_2h^sigma(theta; nu) ||_2 of Eq. lfa-shifted-vcycle for theta in
    Theta_low; nu and theta broadcast to a batch (nu (...,), theta (..., 3))."""
    return np.linalg.norm(vcycle_error_block(tables, nu, theta, sigma, omega, n_sweeps), ord=2, axis=(-2, -1))


def vcycle_error_block(tables, nu, theta, sigma, omega, n_sweeps):
    """The 8 x 8 block E_2h^sigma(theta; nu) of Eq. lfa-shifted-vcycle in the
    harmonic basis phi_p, p in {0,1}^3 (itertools.product order)."""
    nu = np.asarray(nu, dtype=np.float64)
    C2 = shell_coefficients(tables, kappa_of(2, nu), sigma)        # 2h level
    C4 = shell_coefficients(tables, kappa_of(4, nu), sigma)        # 4h level
    p, th = transfer_column(theta)                                 # (..., 8), (..., 8, 3)
    # symbols in absolute units: the 2h symbol carries (2h)^-2, the 4h one (4h)^-2
    B2 = symbol(C2[..., None, :], th) / 4.0                        # (..., 8)
    b4 = symbol(C4, 2.0 * np.asarray(theta)) / 16.0                # (...,)
    d2 = C2[..., 0] / 4.0
    S = 1.0 - omega * B2 / d2[..., None]                           # diagonal Jacobi sweep
    Sn = S ** n_sweeps
    eye = np.eye(8)
    K = eye - (p[..., :, None] * p[..., None, :]) * (B2[..., None, :] / b4[..., None, None])
    return Sn[..., :, None] * K * Sn[..., None, :]


def bottom_multiplier(tables, nu, theta, sigma, omega, n_sweeps):
    """lambda_4h = 1 - s_4h^{n_J} of Eq. bottom-radius-indicator."""
    C4 = shell_coefficients(tables, kappa_of(4, nu), sigma)
    s = 1.0 - omega * symbol(C4, theta) / C4[..., 0]
    return 1.0 - s ** n_sweeps


def ideal_polynomial_factor(lam, degree, n_dirs=64):
    """Degree-m minimax factor over the sample set lam (complex, 1-D): minimise t
    subject to Re(e^{-i phi_j} p(lam_i)) <= t for n_dirs supporting directions,
    p(z) = 1 + sum_k c_k z^k (the supporting-half-plane LP of Sec. 4.4).  Returns
    (t, attained max |p(lam)|, coefficients)."""
    from scipy.optimize import linprog
    lam = np.asarray(lam, dtype=np.complex128).ravel()
    phis = 2.0 * math.pi * np.arange(n_dirs) / n_dirs
    powers = np.stack([lam ** k for k in range(1, degree + 1)], axis=1)    # (n, m)
    rows, rhs = [], []
    for phi in phis:
        e = np.exp(-1j * phi)
        # Re(e (1 + sum c_k z^k)) = Re(e) + sum_k [Re(e z^k) Re c_k - Im(e z^k) Im c_k]
        ez = e * powers
        A = np.concatenate([ez.real, -ez.imag, -np.ones((len(lam), 1))], axis=1)
        rows.append(A)
        rhs.append(-np.full(len(lam), e.real))
    A_ub = np.concatenate(rows)
    b_ub = np.concatenate(rhs)
    cost = np.zeros(2 * degree + 1)
    cost[-1] = 1.0
    res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * (2 * degree + 1), method="highs")
    if not res.success:
        raise RuntimeError("minimax LP failed: " + res.message)
    c = res.x[:degree] + 1j * res.x[degree:2 * degree]
    p = 1.0 + powers @ c
    return float(res.x[-1]), float(np.max(np.abs(p))), c


# ----------------------------------------------------------------------------
# the full h - 2h - 4h hierarchy (closing paragraph of Sec. 4.4)
# ----------------------------------------------------------------------------
def harmonics64(theta):
    """q in {0,1,2,3}^3 (itertools.product order) and the fine-grid angles
    theta + (pi/2) q of Eq. three-grid-harmonics, theta in (-pi/4, pi/4]^3."""
    qs = np.array(list(itertools.product(range(4), repeat=3)))
    return qs, np.asarray(theta, dtype=np.float64)[None, :] + 0.5 * math.pi * qs


def neumann_coefficients(m):
    """Coefficients c_0..c_{m-1} of the fixed m-step map x = M sum_j c_j (H M)^j g
    whose residual polynomial is (1 - z)^m (m Richardson steps); one
    right-hand-side-independent choice for the prescribed polynomials."""
    return np.array([math.comb(m, j + 1) * (-1) ** j for j in range(m)], dtype=np.float64)


def _jacobi_block(b, d, omega, n_sweeps):
    """n sweeps of damped Jacobi from zero on one harmonic space: the diagonal
    omega/d sum_{k<n} (1 - omega b/d)^k (Eq. lfa-jacobi-symbol), as a matrix."""
    s = 1.0 - omega * b / d
    return np.diag(omega / d * sum(s ** k for k in range(n_sweeps)))


def _polynomial_map(H, M, coeffs):
    """g -> M sum_j c_j (H M)^j g: a right-preconditioned Krylov map from zero
    with its coefficients prescribed (closing paragraph of Sec. 4.4)."""
    HM = H @ M
    acc = np.zeros_like(HM)
    power = np.eye(len(H), dtype=HM.dtype)
    for c in coeffs:
        acc = acc + c * power
        power = HM @ power
    return M @ acc


def _threegrid_parts(tables, nu, theta, sigma, omega, n_sweeps, m, coeffs):
    """Per-level blocks on the harmonics of theta: symbols (units h^-2),
    transfers, Jacobi maps and the bottom-solve and V-cycle maps."""
    ch, c2, c4 = coeffs or (neumann_coefficients(m[0]), neumann_coefficients(m[1]), neumann_coefficients(m[2]))
    qs, th = harmonics64(theta)
    rs = np.array(list(itertools.product((0, 1), repeat=3)))
    r_index = (qs % 2) @ np.array([4, 2, 1])                   # alias of theta_q among the 8 2h harmonics
    th2 = 2.0 * np.asarray(theta, dtype=np.float64)[None, :] + math.pi * rs
    th4 = 4.0 * np.asarray(theta, dtype=np.float64)
    Ch = shell_coefficients(tables, kappa_of(1, nu), 0.0)
    A2c = shell_coefficients(tables, kappa_of(2, nu), 0.0)
    B2c = shell_coefficients(tables, kappa_of(2, nu), sigma)
    B4c = shell_coefficients(tables, kappa_of(4, nu), sigma)
    a_h = symbol(Ch, th)
    a_2 = symbol(A2c, th2) / 4.0
    b_2 = symbol(B2c, th2) / 4.0
    b_4 = np.atleast_1d(symbol(B4c, th4) / 16.0)
    rho = lambda ang: np.prod((1.0 + np.cos(ang)) / 2.0, axis=-1)
    P1 = np.zeros((64, 8), dtype=np.complex128)
    P1[np.arange(64), r_index] = rho(th)
    P2 = rho(th2).astype(np.complex128)[:, None]                # (8, 1)
    B2, B4 = np.diag(b_2), np.diag(b_4)
    J2 = _jacobi_block(b_2, B2c[0] / 4.0, omega[1], n_sweeps[1])
    J4 = _jacobi_block(b_4, B4c[0] / 16.0, omega[2], n_sweeps[2])
    I8 = np.eye(8)
    C4 = _polynomial_map(B4, J4, c4)                            # bottom solve C_4h
    Y = J2                                                      # shifted cycle V_2h^sigma
    Yt = Y + P2 @ C4 @ P2.T @ (I8 - B2 @ Y)
    V = Yt + J2 @ (I8 - B2 @ Yt)
    return dict(a_h=a_h, Ah=np.diag(a_h), A2=np.diag(a_2), P1=P1, V=V, c2=c2, ch=ch,
                Jh=_jacobi_block(a_h, Ch[0], omega[0], n_sweeps[0]))


def threegrid_block(tables, nu, theta, sigma=0.9, omega=(0.8, 0.8, 0.2), n_sweeps=(2, 2, 2), m=(2, 10, 4),
                    c_2h=2, coeffs=None):
    """64 x 64 Fourier block of the preconditioner M_h of Algorithm 1 on the
    harmonics of Eq. three-grid-harmonics, every Krylov map replaced by a
    prescribed polynomial (S_h: m_h steps, each 2h FGMRES cycle: m_2h steps,
    C_4h: m_4h steps; `coeffs` = (c_h, c_2h, c_4h), default Neumann).

    Levels: A_h, A_2h unshifted, B_2h, B_4h shifted (Eq. shifted-iofd-levels),
    symbols in units of h^-2; the fine harmonic theta_q aliases on the 2h grid
    to 2 theta + pi (q mod 2), every 2h harmonic on the 4h grid to 4 theta;
    transfers between aliases carry prod (1 + cos)/2 of the finer angle (Eq.
    lfa-transfer-symbol), full weighting the adjoint column.  Returns M with
    the fine symbol a (so that I - M diag(a) is the error propagation)."""
    d = _threegrid_parts(tables, nu, theta, sigma, omega, n_sweeps, m, coeffs)
    Ah, A2, P1, V = d["Ah"], d["A2"], d["P1"], d["V"]
    R1 = P1.T
    I8, I64 = np.eye(8), np.eye(64)
    G2 = _polynomial_map(A2, V, d["c2"])                        # K_2h: c_2h cycles from zero
    K = np.zeros((8, 8), dtype=np.complex128)
    for _ in range(c_2h):
        K = K + G2 @ (I8 - A2 @ K)
    Gh = _polynomial_map(Ah, d["Jh"], d["ch"])                  # S_h(g; x0) = x0 + Gh (g - A x0)
    Zpre = Gh                                                   # Algorithm 1, steps 1-5
    Zt = Zpre + P1 @ K @ R1 @ (I64 - Ah @ Zpre)
    return Zt + Gh @ (I64 - Ah @ Zt), d["a_h"]


def report(tables=None, n_low=28, n_full=33, n_nu=145, n_nu_poly=25, n_poly=12):
    """The diagnostics of Sec. 4.3-4.4 at the paper's fixed parameters
    (sigma, omega_2h, omega_4h) = (0.9, 0.8, 0.2), n_J = 2, on the paper's
    sampling sizes (the polynomial LP on a coarser set, its attained factor on
    the full one)."""
    T = tables or iofd.load_tables()
    nu = np.linspace(*NU_RANGE, n_nu)
    out = {"min_h2_d_h": float(shell_coefficients(T, kappa_of(1, nu))[..., 0].real.min())}
    for name, lev, sig, om in (("mu_h", 1, 0.0, 0.8), ("mu_2h", 2, 0.9, 0.8), ("mu_4h", 4, 0.9, 0.2)):
        out[name] = float(smoothing_factor(T, lev, nu, sig, om, 2).max())
    thl = sorted_angles(n_low, math.pi / 2)
    NU, TH = np.meshgrid(nu, np.arange(len(thl)), indexing="ij")
    out["q_V"] = float(vcycle_error_norm(T, NU.ravel(), thl[TH.ravel()], 0.9, 0.8, 2).max())
    th = sorted_angles(n_full, math.pi)
    NU, TH = np.meshgrid(np.linspace(*NU_RANGE, 73), np.arange(len(th)), indexing="ij")
    lam = bottom_multiplier(T, NU.ravel(), th[TH.ravel()], 0.9, 0.2, 2)
    out["rho_4h"], out["delta_4h"] = float(np.abs(lam).max()), float(np.abs(lam).min())
    thp = sorted_angles(n_poly, math.pi)
    NUp, THp = np.meshgrid(np.linspace(*NU_RANGE, n_nu_poly), np.arange(len(thp)), indexing="ij")
    t, _, c = ideal_polynomial_factor(bottom_multiplier(T, NUp.ravel(), thp[THp.ravel()], 0.9, 0.2, 2), 4)
    out["gamma4_lp"] = t
    out["gamma4_attained"] = float(np.max(np.abs(1.0 + sum(c[k] * lam ** (k + 1) for k in range(4)))))
    return out


def _spectral_sweep(tables, coeffs, n_theta, n_nu):
    """sup |1 - lambda| and inf |lambda| of M_h A_h over theta in [0, pi/4]^3
    (sorted representatives) and nu in [6, 24]."""
    worst, sep = 0.0, np.inf
    for nu in np.linspace(*NU_RANGE, n_nu):
        for th in sorted_angles(n_theta, math.pi / 4):
            M, a = threegrid_block(tables, nu, th, coeffs=coeffs)
            lam = np.linalg.eigvals(M * a[None, :])
            worst = max(worst, float(np.abs(1.0 - lam).max()))
            sep = min(sep, float(np.abs(lam).min()))
    return worst, sep


def threegrid_report(tables=None, n_theta=7, n_nu=19):
    """The linearised three-grid map at (sigma, omega_2h, omega_4h) = (0.9, 0.8,
    0.2) and the Table 4 step counts, with two right-hand-side-independent
    choices of the polynomials: Neumann (residual (1 - z)^m) at every level,
    and minimax at every level -- the degree-4 bottom factor of the LP above,
    then the degree-10 and degree-2 minimax factors over the sampled spectra of
    A_2h V_2h and A_h J_h that the levels below produce."""
    T = tables or iofd.load_tables()
    out = {}
    neumann = (neumann_coefficients(2), neumann_coefficients(10), neumann_coefficients(4))
    out["neumann_sup_1_minus_lambda"], out["neumann_inf_lambda"] = _spectral_sweep(T, neumann, n_theta, n_nu)
    thp = sorted_angles(12, math.pi)
    NUp, THp = np.meshgrid(np.linspace(*NU_RANGE, 25), np.arange(len(thp)), indexing="ij")
    _, _, c4 = ideal_polynomial_factor(bottom_multiplier(T, NUp.ravel(), thp[THp.ravel()], 0.9, 0.2, 2), 4)
    # residual polynomial 1 + sum_k c_k z^k  <->  map coefficients q_j = -c_{j+1}
    q4 = -c4
    lam2, lamh = [], []
    for nu in np.linspace(*NU_RANGE, 10):
        for th in sorted_angles(5, math.pi / 4):
            AV, AJ = _level_operators(T, nu, th, q4)
            lam2.append(np.linalg.eigvals(AV))
            lamh.append(AJ)
    _, _, c2 = ideal_polynomial_factor(np.concatenate(lam2), 10)
    _, _, ch = ideal_polynomial_factor(np.concatenate(lamh), 2)
    out["minimax_sup_1_minus_lambda"], out["minimax_inf_lambda"] = _spectral_sweep(T, (-ch, -c2, q4), n_theta, n_nu)
    return out


def _level_operators(tables, nu, theta, q4, sigma=0.9, omega=(0.8, 0.8, 0.2), n_sweeps=(2, 2, 2)):
    """A_2h V_2h (8 x 8, with the bottom map q4) and the diagonal of A_h J_h
    (64 values) on the harmonics of theta: the operators whose spectra the
    2h and h polynomials act on."""
    d = _threegrid_parts(tables, nu, theta, sigma, omega, n_sweeps, (2, 10, 4),
                         (neumann_coefficients(2), neumann_coefficients(10), q4))
    return d["A2"] @ d["V"], d["a_h"] * np.diag(d["Jh"])


if __name__ == "__main__":
    import sys
    rep = threegrid_report() if "--threegrid" in sys.argv else report()
    for k, v in rep.items():
        print(f"{k:28s} {v:.4g}")
