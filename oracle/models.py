"""Data-driven system-matrix models M0, M1, M2 and the distance measures.

Test infrastructure (see ``oracle/__init__``).

Section 2.2 builds system matrices from a dictionary of simulated signals
phi_hat and fits them to a measured system matrix S_calib; Section 2.3 defines
how far a model is from the measurement.  Every array here is laid out
[voxel, channel, k] (complex), the layout of the solver's phi_hat.

* ``equilibrium_trace`` -- model M0: the equilibrium mean moment
  m_equ / m0 = L(bT |B|) B / |B| (Eq. Langevin with beta H = bT B) at the
  sample times, and its time derivative by the complex-step rule
  d/dt f(t) = Im f(t + i h) / h (f analytic in t; no difference quotient, so
  no cancellation).  Its phi_hat follows from ``solve.phi_hat``.
* ``m1_fit`` -- model M1 (and M0): per row k the least-squares filter value
  a_k = S_k conj(Phi_k)^T / ||Phi_k||^2 (closed form of the M0/M1 fit in the
  "Technical details" paragraph of Section 2.2) and the row error of
  Eq. error1 for S_model = diag(a) Phi.
* ``mixing_order`` / ``freq_index_set`` -- Eq. mix, the frequency index set
  I_freq of Section 2.3.
* ``eps_row`` / ``eps_freq`` / ``eps_global`` -- Eq. error1, the per-frequency
  measure and eq. globalMeasure (quadratic sums also over the receive
  channels, as the last remark of Section 2.3 states).
* ``m2_weights`` -- model M2 second step: the Sigma-weighted dictionary
  matrix M (eq. LSfitM2_alternative), its SVD, the truncated problem
  (eq. approx_low_rank) with complex data and real weights stacked as real
  and imaginary parts, solved for w >= 0 by a library non-negative least
  squares routine (the problem the paper's interior-point QP solves).

Parity status: pinned (tests/test_oracle_models.py) -- Langevin values and
series, complex-step derivative against central differences, closed-form
filter against a library least-squares solve, NRMSE special cases, mixing
orders against brute-force enumeration, M2 against a planted exact
superposition and against full-rank NNLS.
"""
import numpy as np
from scipy.optimize import nnls


# ------------------------------------------------------------------ M0 -----
# Taylor coefficients of L(x) = sum_n c_n x^(2n-1), c_n = 2^(2n) B_2n / (2n)!
# (B_2n Bernoulli numbers, exact rationals from the recurrence
# sum_{k<=m} C(m+1, k) B_k = 0), n = 1..11: 1/3, -1/45, 2/945, -1/4725, ...
def _langevin_series_coefficients(nterms=11):
    from fractions import Fraction
    from math import comb, factorial
    B = [Fraction(1)]
    for m in range(1, 2 * nterms + 1):
        B.append(-sum(comb(m + 1, k) * B[k] for k in range(m)) / (m + 1))
    return [float(Fraction(2 ** (2 * n)) * B[2 * n] / factorial(2 * n)) for n in range(1, nterms + 1)]


_LSER = _langevin_series_coefficients()
_LSER_MAX = 0.5      # closed form loses ~3 eps / x^2 relative; series term 12 is ~(x/pi)^22 smaller


def langevin_c(xi):
    """L(xi) = coth(xi) - 1/xi for real or complex xi (Eq. Langevin); its
    Taylor series (11 terms) where |xi| < 0.5, where the closed form cancels."""
    xi = np.asarray(xi)
    small = np.abs(xi) < _LSER_MAX
    safe = np.where(small, 1.0, xi)
    closed = np.cosh(safe) / np.sinh(safe) - 1.0 / safe
    x2 = xi * xi
    acc = np.zeros_like(x2)
    for c in reversed(_LSER):
        acc = acc * x2 + c
    return np.where(small, xi * acc, closed)


def equilibrium_moment(bT, B):
    """m_equ / m0 = L(bT |B|) B / |B| for fields B (..., 3) [T] (Eq. Langevin
    with beta H = bT B).  |B| is continued analytically (sqrt(B.B), no
    conjugate) so that the complex-step derivative applies."""
    B = np.asarray(B)
    nb = np.sqrt(np.sum(B * B, axis=-1))
    xi = bT * nb
    small = np.abs(xi) < 1e-12
    ratio = np.where(small, bT / 3.0, langevin_c(np.where(small, 1.0, xi)) / np.where(small, 1.0, nb))
    return ratio[..., None] * B


def equilibrium_trace(mat, drive, d, h_off, t, h_cs=None):
    """Model M0 trace of one voxel: <m>(t_j) and d<m>/dt(t_j) (per unit m0) of
    the equilibrium model under B(t) = h_off + drive (Section 2.2, M0)."""
    from .physics import derive
    P = derive(mat, 0.0, d)
    t = np.asarray(t, dtype=np.float64)
    off = np.asarray(h_off, dtype=np.float64)
    m = equilibrium_moment(P.bT, drive.field(t, off))
    h = (h_cs if h_cs is not None else 1e-20 * drive.period)
    tc = t + 1j * h
    Bc = np.empty(t.shape + (3,), dtype=np.complex128)
    for k in range(3):
        Bc[..., k] = off[k] + drive.amp[k] * np.sin(2.0 * np.pi * drive.freq[k] * tc + drive.phase[k])
    dm = np.imag(equilibrium_moment(P.bT, Bc)) / h
    return m, dm


# ------------------------------------------------------------------ M1 -----
def m1_fit(Phi, S):
    """Closed-form M1 (or M0) fit per channel and row.  Phi, S: [N, C, K]
    complex.  Returns a [C, K] (a_k = S_k conj(Phi_k)^T / ||Phi_k||^2) and the
    row errors eps [C, K] of Eq. error1 for S_model = diag(a) Phi."""
    Phi = np.asarray(Phi)
    S = np.asarray(S)
    a = np.sum(S * np.conj(Phi), axis=0) / np.sum(np.abs(Phi) ** 2, axis=0)
    model = a[None] * Phi
    return a, eps_row(S, model)


def eps_row(S_calib, S_model):
    """Eq. error1 per channel and row: (1/sqrt(N)) ||S_calib,k - S_model,k||_2
    / ||S_calib,k||_inf, arrays [N, C, K]."""
    N = S_calib.shape[0]
    num = np.sqrt(np.sum(np.abs(S_calib - S_model) ** 2, axis=0)) / np.sqrt(N)
    return num / np.max(np.abs(S_calib), axis=0)


def mixing_order(k, n_dens):
    """(m_x, m_y) with k = m_x n_dens + m_y (n_dens + 1) and the smallest
    |m_x| + |m_y| (Eq. mix); ties: smaller |m_x|, then m_x >= 0.  Found by
    enumeration over m_y (every solution has m_y = k mod n_dens + j n_dens)."""
    best = None
    for my in range(-(abs(k) + 2 * n_dens), abs(k) + 2 * n_dens + 1):
        r = k - my * (n_dens + 1)
        if r % n_dens:
            continue
        mx = r // n_dens
        key = (abs(mx) + abs(my), abs(mx), 0 if mx >= 0 else 1)
        if best is None or key < best[0]:
            best = (key, mx, my)
    return best[1], best[2]


def freq_index_set(M_x, M_y, n_dens):
    """I_freq = {k(m_x, m_y) : 0 <= m_x <= M_x, 0 <= m_y <= M_y} without the
    orders (0,0), (0,1), (1,0) (Section 2.3), as sorted distinct k."""
    ks = {mx * n_dens + my * (n_dens + 1) for mx in range(M_x + 1) for my in range(M_y + 1)
          if (mx, my) not in ((0, 0), (0, 1), (1, 0))}
    return np.array(sorted(ks), dtype=np.int64)


def eps_freq(eps_by_angle):
    """Per-frequency measure: RMS of Eq. error1 over the angles (and receive
    channels).  eps_by_angle: [angles, C, K] -> [K]."""
    e = np.asarray(eps_by_angle)
    return np.sqrt(np.mean(e ** 2, axis=(0, 1)))


def eps_global(eps_by_angle, ks):
    """eq. globalMeasure: RMS of the per-frequency measure over k in I_freq."""
    ef = eps_freq(eps_by_angle)
    return float(np.sqrt(np.mean(ef[np.asarray(ks)] ** 2)))


# ------------------------------------------------------------------ M2 -----
def m2_matrix(Psi, S, ks):
    """The Sigma-weighted dictionary matrix M and data y of eq. LSfitM2_alternative.
    Psi: [angles][J] dictionary system matrices psi = diag(a_q) phi_q, each
    [N, C, K]; S: [angles] measured matrices [N, C, K]; ks: rows used (I_freq).
    Sigma_theta = diag(1/||S_theta,k||_inf) per channel and row; M stacks the
    columns vec(Sigma Psi_q) over the angles, y = vec(Sigma S)."""
    ks = np.asarray(ks)
    cols, ys = [], []
    for Pa, Sa in zip(Psi, S):
        Sk = np.asarray(Sa)[:, :, ks]
        sig = 1.0 / np.max(np.abs(Sk), axis=0)                 # [C, K]
        ys.append((sig[None] * Sk).reshape(-1))
        cols.append(np.stack([(sig[None] * np.asarray(p)[:, :, ks]).reshape(-1) for p in Pa], axis=1))
    return np.concatenate(cols, axis=0), np.concatenate(ys)


def m2_weights(Psi, S, ks, s_rank=None):
    """Model M2 weights for the matrix M and data y of ``m2_matrix``.  With
    s_rank the problem is projected on the first s left singular vectors of M
    (eq. approx_low_rank).  Complex residuals with real weights are split into
    real and imaginary parts; w >= 0 by non-negative least squares.  Returns
    (w, ||M w - y||_2, singular values of M, the minimised objective
    ||G w - h||_2^2 of the (projected) problem)."""
    M, y = m2_matrix(Psi, S, ks)
    U, sv, Vh = np.linalg.svd(M, full_matrices=False)
    if s_rank is None:
        G, h = M, y
    else:
        Us = U[:, :s_rank]
        G, h = np.conj(Us.T) @ M, np.conj(Us.T) @ y
    Gr = np.concatenate([G.real, G.imag], axis=0)
    hr = np.concatenate([h.real, h.imag])
    w, _ = nnls(Gr, hr, maxiter=50 * Gr.shape[1])
    return w, float(np.linalg.norm(M @ w - y)), sv, float(np.linalg.norm(Gr @ w - hr) ** 2)
