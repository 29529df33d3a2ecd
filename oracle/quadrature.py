"""Velocity-space quadratures and Hermite bases of the oracle (FP64, numpy).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow reference the CUDA
solver is checked against.  Only tests, the smoke check and the CPU-baseline
leg of the benchmark may import it; the solver never does.

Velocity space is discretised with the mixed quadrature of Sec. III
("HHLB(N_x;Q_x) x HLB(N_y;Q_y)"): full-range Gauss-Hermite rules on the axes
parallel to the walls and a half-range Gauss-Hermite rule on each semi-axis of
the wall-normal axis.  The weight function is the one of Eq. (H_omega),
omega(p) = exp(-p^2/2)/sqrt(2 pi), so a full-range rule has sum(w) = 1 and a
half-range rule (nodes on (0, inf)) has sum(w) = 1/2.

Algorithms (chosen to differ from the solver's own quadrature code):
  * full range: numpy's Gauss-HermiteE rule (library routine), renormalised;
  * half range: Lanczos with full re-orthogonalisation on a fine discretisation
    of omega restricted to (0, inf) (composite 40-point Gauss-Legendre on 80
    panels of [0, 40]), the eigenvalues of the Jacobi matrix (numpy eigh,
    Golub-Welsch) polished by Newton steps on pi_Q, and Christoffel weights
    w_j = 1 / sum_k phat_k(x_j)^2 over the orthonormal polynomials phat_k (this
    keeps the tiny weights of the outermost nodes accurate to full relative
    precision, which the eigenvector form does not).
"""
import math

import numpy as np
from numpy.polynomial import hermite_e as _he

SQRT_2PI = math.sqrt(2.0 * math.pi)


def full_range_rule(Q):
    """Q-point Gauss rule for omega(p) on the whole line; sum(w) = 1 (Eq. H_omega)."""
    x, w = _he.hermegauss(Q)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64) / SQRT_2PI


def _half_range_measure(panels=80, pts=40, pmax=40.0):
    """Discretisation of omega(p) dp on (0, pmax); omega < 1e-340 beyond pmax."""
    t, v = np.polynomial.legendre.leggauss(pts)
    hw = 0.5 * pmax / panels
    x = np.concatenate([a + hw * (t + 1.0) for a in np.arange(panels) * 2.0 * hw])
    w = np.tile(hw * v, panels) * np.exp(-0.5 * x * x) / SQRT_2PI
    return x, w


def half_range_recurrence(n):
    """Recurrence coefficients of the monic polynomials orthogonal w.r.t. omega on (0, inf).

    pi_{k+1}(p) = (p - alpha_k) pi_k(p) - beta_k pi_{k-1}(p), beta_0 = int omega = 1/2.
    Returned: alpha[0..n-1], beta[0..n-1].
    """
    x, w = _half_range_measure()
    M = x.size
    V = np.zeros((n + 1, M))
    v = np.sqrt(w)
    beta0 = float(v @ v)
    V[0] = v / math.sqrt(beta0)
    alpha = np.zeros(n)
    beta = np.zeros(n)
    beta[0] = beta0
    for k in range(n):
        y = x * V[k]
        alpha[k] = V[k] @ y
        y = y - alpha[k] * V[k]
        if k > 0:
            y = y - math.sqrt(beta[k]) * V[k - 1]
        for _ in range(2):  # full re-orthogonalisation
            y = y - V[: k + 1].T @ (V[: k + 1] @ y)
        b = float(np.linalg.norm(y))
        if k + 1 < n:
            beta[k + 1] = b * b
        V[k + 1] = y / b
    return alpha, beta


def _orthonormal_values(x, alpha, beta, n):
    """phat_k(x), k = 0..n-1, orthonormal w.r.t. omega on (0, inf), by the recurrence."""
    P = np.zeros((n, x.size))
    P[0] = 1.0 / math.sqrt(beta[0])
    if n > 1:
        P[1] = (x - alpha[0]) * P[0] / math.sqrt(beta[1])
    for k in range(1, n - 1):
        P[k + 1] = ((x - alpha[k]) * P[k] - math.sqrt(beta[k]) * P[k - 1]) / math.sqrt(beta[k + 1])
    return P


def half_range_rule(Q):
    """Q-point Gauss rule for omega on (0, inf); sum(w) = 1/2 (Sec. III, half-range GH)."""
    alpha, beta = half_range_recurrence(Q + 1)
    a, b = alpha[:Q], beta[:Q]
    J = np.diag(a) + np.diag(np.sqrt(b[1:]), 1) + np.diag(np.sqrt(b[1:]), -1)
    x = np.linalg.eigvalsh(J)
    for _ in range(3):  # Newton on phat_Q, the orthonormal polynomial of degree Q
        P = _orthonormal_values(x, alpha, beta, Q + 1)
        # derivative by differentiating the recurrence
        D = np.zeros_like(P)
        D[1] = P[0] / math.sqrt(beta[1])
        for k in range(1, Q):
            D[k + 1] = (P[k] + (x - alpha[k]) * D[k] - math.sqrt(beta[k]) * D[k - 1]) / math.sqrt(beta[k + 1])
        x = x - P[Q] / D[Q]
    P = _orthonormal_values(x, alpha, beta, Q)
    return x, 1.0 / np.sum(P * P, axis=0)


def half_range_polys(N):
    """Monomial coefficients c[l, m] of the monic half-range polynomials pi_l, l <= N,
    and their norms h_l = int_0^inf omega pi_l^2 dp."""
    alpha, beta = half_range_recurrence(N + 1)
    c = np.zeros((N + 1, N + 1))
    c[0, 0] = 1.0
    if N >= 1:
        c[1, 0] = -alpha[0]
        c[1, 1] = 1.0
    for l in range(1, N):
        c[l + 1, 1:] += c[l, :-1]
        c[l + 1] -= alpha[l] * c[l]
        c[l + 1] -= beta[l] * c[l - 1]
    h = np.cumprod(beta[: N + 1])
    return c, h


def hermite_table(x, N):
    """He_l(x_i) / l!  for l = 0..N (probabilists' Hermite, Eq. H_ortho normalisation)."""
    T = np.zeros((x.size, N + 1))
    for l in range(N + 1):
        e = np.zeros(l + 1)
        e[l] = 1.0
        T[:, l] = _he.hermeval(x, e) / math.factorial(l)
    return T


def half_range_table(xi, c, h):
    """pi_l(xi_m) / h_l for the half-range basis."""
    N = c.shape[0] - 1
    T = np.zeros((xi.size, N + 1))
    for l in range(N + 1):
        T[:, l] = np.polynomial.polynomial.polyval(xi, c[l]) / h[l]
    return T
