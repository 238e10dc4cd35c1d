"""Plain FP64 CPU oracle for the FGFRFT online hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The
product path (the CUDA library and its Python binding) never imports, calls or
links anything under ``oracle/``, and this module imports nothing from the
product package.

What it computes (paper: "FGFRFT: Fast Graph Fractional Fourier Transform via
Exact Spectral Splitting and Fourier-Series Approximation"):

* ``coeffs`` / ``dcoeffs`` / ``phase``      -- Sec. III-A (Fourier coefficients of
  e^{j alpha theta}), the (-1)^n form from the proof of Thm. 1, and the
  derivative of Prop. 3 (Eq. "eqdifferentiability").
* ``spectral``                               -- Sec. III-A: eigen-decomposition of
  the unitary F with principal-branch phases in (-pi, pi], and the index set
  I_{-1} of Sec. III-B.
* ``exact_gfrft``                            -- Sec. II-B / III-A: F^alpha = V
  diag(e^{j alpha theta_k}) V^H.
* ``fgfrft_spectral`` (form S)               -- Def. 1 evaluated per eigenvalue.
* ``projector`` / ``powers``                 -- Algorithm 1, offline part.
* ``fgfrft_power`` (form P)                  -- Algorithm 1, online part, with the
  negative powers taken as M_n^H (Prop. 2, Eq. "eqefficient_computation").
* ``apply_power`` / ``dalpha_apply`` /
  ``adjoint_apply`` / ``grad_alpha``        -- Def. 2 (x~ = Q x) per column,
  Prop. 3 (d/d alpha), Prop. 2 (adjoint symmetry), and the chain rule.
* ``trunc_error`` and the bounds             -- Thm. 1 (pointwise bound),
  Thm. 2 (Frobenius identity and bounds), Props. 4-6.

Numbers are complex128 / float64 throughout.  Readings of the paper where it
is silent (the tolerance that decides theta_k = pi, "alpha in Z" in floating
point, the branch at theta = pi) are documented next to the code that takes
them.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, brute force on DFT and cyclic-shift matrices, bounds, finite
differences and the paper's printed numbers).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

# Reading of Algorithm 1 ("Identify I_{-1} = {k : theta_k = pi}"): the paper
# gives no tolerance.  An eigenvalue counts as -1 when |lambda_k + 1| <= NEG1_TOL.
NEG1_TOL = 1e-8


# ----------------------------------------------------------------------------
# scalar functions of alpha (Sec. III-A, proof of Thm. 1, Prop. 3)
# ----------------------------------------------------------------------------
def _reduce2(a: float) -> float:
    """a - 2*round(a/2), exact in FP64, lies in [-1, 1]."""
    return a - 2.0 * round(a / 2.0)


def sin_pi(a: float) -> float:
    """sin(pi a), exactly 0 at every integer (reading of "alpha in Z")."""
    r = _reduce2(float(a))
    if r > 0.5:
        r = 1.0 - r
    elif r < -0.5:
        r = -1.0 - r
    return math.sin(math.pi * r)


def cos_pi(a: float) -> float:
    """cos(pi a), exactly +-1 at integers and 0 at half-integers."""
    r = abs(_reduce2(float(a)))
    if r <= 0.5:
        return math.sin(math.pi * (0.5 - r))
    return -math.sin(math.pi * (r - 0.5))


def is_integer_order(alpha: float) -> bool:
    """Reading: alpha is an integer order iff alpha == round(alpha) in FP64."""
    return float(alpha) == float(round(alpha))


def coeffs(alpha: float, L: int) -> np.ndarray:
    """c_n(alpha) for n = -L..L (array index n + L).

    Sec. III-A: c_n = sin(pi(alpha - n)) / (pi(alpha - n)); written as
    (-1)^n sin(pi alpha) / (pi(alpha - n)) (proof of Thm. 1, Step 1) so that
    it is exactly the Kronecker delta at integer alpha (Remark 2).
    """
    s = sin_pi(alpha)
    out = np.empty(2 * L + 1, dtype=np.float64)
    for i, n in enumerate(range(-L, L + 1)):
        d = alpha - n
        if d == 0.0:
            out[i] = 1.0
        else:
            sign = -1.0 if (n % 2) else 1.0
            out[i] = sign * s / (math.pi * d)
    return out


def _dsinc(x: float) -> float:
    """d/dx (sin x / x)."""
    if abs(x) < 1e-2:
        x2 = x * x
        return x * (-1.0 / 3.0 + x2 * (1.0 / 30.0 + x2 * (-1.0 / 840.0 + x2 / 45360.0)))
    return (x * math.cos(x) - math.sin(x)) / (x * x)


def dcoeffs(alpha: float, L: int) -> np.ndarray:
    """d c_n / d alpha for n = -L..L (Prop. 3).

    c_n(alpha) = sinc(pi (alpha - n)) with sinc(x) = sin x / x, so
    c_n' = pi * sinc'(pi (alpha - n)); written with the exact sin(pi alpha),
    cos(pi alpha) away from alpha = n and by its Taylor series near it.
    """
    s = sin_pi(alpha)
    c = cos_pi(alpha)
    out = np.empty(2 * L + 1, dtype=np.float64)
    for i, n in enumerate(range(-L, L + 1)):
        d = alpha - n
        if abs(d) < 1e-3:
            out[i] = math.pi * _dsinc(math.pi * d)
        else:
            sign = -1.0 if (n % 2) else 1.0
            out[i] = sign * (math.pi * d * c - s) / (math.pi * d * d)
    return out


def phase(alpha: float) -> complex:
    """e^{j pi alpha}, the exact factor on the lambda = -1 eigenspace (Eq. 16)."""
    return complex(cos_pi(alpha), sin_pi(alpha))


def dphase(alpha: float) -> complex:
    """d/d alpha e^{j pi alpha} = j pi e^{j pi alpha} (Prop. 3)."""
    return 1j * math.pi * phase(alpha)


# ----------------------------------------------------------------------------
# spectral side (Sec. III-A, III-B)
# ----------------------------------------------------------------------------
class Spectral:
    """Unitary eigen-decomposition F = Z diag(lam) Z^H with principal phases."""

    def __init__(self, F: np.ndarray, tol: float = NEG1_TOL):
        F = np.asarray(F, dtype=np.complex128)
        # Complex Schur: for a normal matrix T is diagonal up to round-off and
        # Z is unitary even inside degenerate eigenspaces.
        T, Z = scipy.linalg.schur(F, output="complex")
        lam = np.diag(T).copy()
        theta = np.angle(lam)
        neg1 = np.abs(lam + 1.0) <= tol
        # Principal branch theta in (-pi, pi]: angle() may return -pi for
        # -1 - 0j; eigenvalues counted as -1 get theta = +pi exactly.
        theta[neg1] = math.pi
        theta[(~neg1) & (theta <= -math.pi)] = math.pi
        self.Z = Z
        self.lam = lam
        self.theta = theta
        self.neg1 = neg1
        self.r_neg1 = int(neg1.sum())
        comp = ~neg1
        self.min_gap = float(np.min(np.abs(lam[comp] + 1.0))) if comp.any() else math.inf
        self.cos_c_min = float(np.min(np.abs(np.cos(theta[comp] / 2.0)))) if comp.any() else math.inf
        self.offdiag = float(np.linalg.norm(T - np.diag(lam)))

    def rebuild(self, values: np.ndarray) -> np.ndarray:
        """Z diag(values) Z^H."""
        return (self.Z * values[None, :]) @ self.Z.conj().T


def spectral(F: np.ndarray, tol: float = NEG1_TOL) -> Spectral:
    return Spectral(F, tol)


def exact_gfrft(F: np.ndarray, alpha: float, sp: Spectral | None = None) -> np.ndarray:
    """F^alpha = V diag(e^{j alpha theta_k}) V^H, principal branch (Eq. 9)."""
    sp = sp or spectral(F)
    return sp.rebuild(np.exp(1j * alpha * sp.theta))


def series_value(theta: np.ndarray, alpha: float, L: int) -> np.ndarray:
    """sum_{n=-L}^{L} c_n(alpha) e^{j n theta} (truncated Fourier series)."""
    c = coeffs(alpha, L)
    n = np.arange(-L, L + 1)
    return np.exp(1j * np.outer(np.atleast_1d(theta), n)) @ c


def q_values(sp: Spectral, alpha: float, L: int) -> np.ndarray:
    """Eigenvalues of Q_L^alpha: e^{j pi alpha} on I_{-1}, truncated series elsewhere."""
    vals = series_value(sp.theta, alpha, L)
    vals[sp.neg1] = phase(alpha)
    return vals


def fgfrft_spectral(F: np.ndarray, alpha: float, L: int, sp: Spectral | None = None) -> np.ndarray:
    """Form S: Def. 1 evaluated on the spectrum, Z diag(q_L(theta_k)) Z^H.

    Integer alpha gives F^alpha (Def. 1, second sentence).
    """
    sp = sp or spectral(F)
    if is_integer_order(alpha):
        return sp.rebuild(sp.lam ** int(round(alpha)))
    return sp.rebuild(q_values(sp, alpha, L))


# ----------------------------------------------------------------------------
# power side: Algorithm 1 (offline + online)
# ----------------------------------------------------------------------------
def projector(F: np.ndarray, sp: Spectral | None = None) -> np.ndarray:
    """P_{-1} = W W^H, W = orthonormal eigenvectors with lambda = -1 (Alg. 1, offline)."""
    sp = sp or spectral(F)
    W = sp.Z[:, sp.neg1]
    return W @ W.conj().T


def powers(F: np.ndarray, L: int, P: np.ndarray) -> list[np.ndarray]:
    """[M_0, ..., M_L] with M_0 = P_c and M_n = F M_{n-1} (Alg. 1, offline loop)."""
    F = np.asarray(F, dtype=np.complex128)
    N = F.shape[0]
    M = [np.eye(N, dtype=np.complex128) - P]
    for _ in range(L):
        M.append(F @ M[-1])
    return M


def integer_power(F: np.ndarray, k: int) -> np.ndarray:
    """F^k by repeated products; F^{-k} = (F^H)^k for unitary F."""
    F = np.asarray(F, dtype=np.complex128)
    base = F if k >= 0 else F.conj().T
    out = np.eye(F.shape[0], dtype=np.complex128)
    for _ in range(abs(k)):
        out = base @ out
    return out


def fgfrft_power(F: np.ndarray, alpha: float, L: int, P: np.ndarray | None = None,
                 M: list[np.ndarray] | None = None) -> np.ndarray:
    """Form P: Algorithm 1, online part.

    Q = e^{j pi alpha} P_{-1} + c_0 P_c + sum_{n=1}^{L} (c_n M_n + c_{-n} M_n^H).
    Integer alpha returns F^alpha (Algorithm 1 returns early; Def. 1).
    """
    if is_integer_order(alpha):
        return integer_power(F, int(round(alpha)))
    if P is None:
        P = projector(F)
    if M is None:
        M = powers(F, L, P)
    c = coeffs(alpha, L)
    Q = phase(alpha) * P + c[L] * M[0]
    for n in range(1, L + 1):
        Q = Q + c[L + n] * M[n] + c[L - n] * M[n].conj().T
    return Q


# ----------------------------------------------------------------------------
# signals: Def. 2 per column, Prop. 3, Prop. 2, chain rule
# ----------------------------------------------------------------------------
def _alphas(alpha, B: int) -> np.ndarray:
    a = np.asarray(alpha, dtype=np.float64).reshape(-1)
    if a.size == 1:
        a = np.full(B, float(a[0]))
    if a.size != B:
        raise ValueError("alpha must be a scalar or have one entry per column")
    return a


def _power_terms(F: np.ndarray, P: np.ndarray, X: np.ndarray, L: int):
    """Z_n = F^n P_c X for n = -L..L by recursion on the signals (no stored powers)."""
    F = np.asarray(F, dtype=np.complex128)
    Z0 = X - P @ X
    pos = [Z0]
    neg = [Z0]
    FH = F.conj().T
    for _ in range(L):
        pos.append(F @ pos[-1])
        neg.append(FH @ neg[-1])
    return [neg[L - i] for i in range(L)] + pos  # index n + L


def apply_power(F: np.ndarray, alpha, L: int, X: np.ndarray, P: np.ndarray | None = None,
                terms=None) -> np.ndarray:
    """Y[:, j] = Q_L^{alpha_j} X[:, j] (Def. 2), power form per column.

    X is (N, B); alpha is a scalar or one order per column.  Integer orders
    give F^alpha x exactly (Def. 1).
    """
    X = np.asarray(X, dtype=np.complex128)
    if X.ndim == 1:
        X = X[:, None]
    N, B = X.shape
    a = _alphas(alpha, B)
    if P is None:
        P = projector(F)
    if terms is None:
        terms = _power_terms(F, P, X, L)
    PX = P @ X
    Y = np.zeros_like(X)
    for j in range(B):
        if is_integer_order(a[j]) and abs(round(a[j])) > L:
            Y[:, j] = integer_power(F, int(round(a[j]))) @ X[:, j]
            continue
        c = coeffs(a[j], L)
        y = phase(a[j]) * PX[:, j]
        for i in range(2 * L + 1):
            y = y + c[i] * terms[i][:, j]
        Y[:, j] = y
    return Y


def dalpha_apply(F: np.ndarray, alpha, L: int, X: np.ndarray, P: np.ndarray | None = None,
                 terms=None) -> np.ndarray:
    """D[:, j] = (dQ/d alpha)(alpha_j) X[:, j] (Prop. 3, Eq. "eqdifferentiability")."""
    X = np.asarray(X, dtype=np.complex128)
    if X.ndim == 1:
        X = X[:, None]
    N, B = X.shape
    a = _alphas(alpha, B)
    if P is None:
        P = projector(F)
    if terms is None:
        terms = _power_terms(F, P, X, L)
    PX = P @ X
    D = np.zeros_like(X)
    for j in range(B):
        dc = dcoeffs(a[j], L)
        d = dphase(a[j]) * PX[:, j]
        for i in range(2 * L + 1):
            d = d + dc[i] * terms[i][:, j]
        D[:, j] = d
    return D


def adjoint_apply(F: np.ndarray, alpha, L: int, G: np.ndarray, P: np.ndarray | None = None) -> np.ndarray:
    """(Q_L^{alpha_j})^H G[:, j] = Q_L^{-alpha_j} G[:, j] (Prop. 2, adjoint symmetry)."""
    a = -_alphas(alpha, np.asarray(G).reshape(np.asarray(G).shape[0], -1).shape[1])
    return apply_power(F, a, L, G, P)


def grad_alpha(G: np.ndarray, D: np.ndarray) -> np.ndarray:
    """d loss / d alpha_j = Re sum_i conj(G_ij) D_ij, G = dloss/dRe Y + j dloss/dIm Y."""
    G = np.asarray(G, dtype=np.complex128)
    D = np.asarray(D, dtype=np.complex128)
    if G.ndim == 1:
        G = G[:, None]
        D = D[:, None]
    return np.real(np.sum(np.conj(G) * D, axis=0))


# ----------------------------------------------------------------------------
# error analysis (Thm. 1, Thm. 2, Props. 4-6, Sec. IV-A)
# ----------------------------------------------------------------------------
def trunc_error(theta: np.ndarray, alpha: float, L: int) -> np.ndarray:
    """R_L(theta) = e^{j alpha theta} - sum_{|n|<=L} c_n e^{j n theta} (Thm. 1)."""
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    return np.exp(1j * alpha * theta) - series_value(theta, alpha, L)


def pointwise_bound(theta: np.ndarray, alpha: float, L: int) -> np.ndarray:
    """|sin(pi a)| / (pi cos(theta/2)) (1/(L+1-a) + 1/(L+1+a)), valid for L > |a| (Thm. 1)."""
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    return abs(sin_pi(alpha)) / (math.pi * np.cos(theta / 2.0)) * (
        1.0 / (L + 1 - alpha) + 1.0 / (L + 1 + alpha))


def frobenius_error_exact(sp: Spectral, alpha: float, L: int) -> float:
    """||E_L||_F = sqrt(sum_{k not in I_-1} |R_L(theta_k)|^2) (Thm. 2, first identity)."""
    comp = ~sp.neg1
    return float(np.sqrt(np.sum(np.abs(trunc_error(sp.theta[comp], alpha, L)) ** 2)))


def frobenius_bound_tight(sp: Spectral, alpha: float, L: int) -> float:
    """Thm. 2, second statement (per-eigenvalue cosines)."""
    comp = ~sp.neg1
    k = 2.0 * (L + 1) * abs(sin_pi(alpha)) / (math.pi * ((L + 1) ** 2 - alpha ** 2))
    return float(k * np.sqrt(np.sum(1.0 / np.cos(sp.theta[comp] / 2.0) ** 2)))


def frobenius_bound_simplified(sp: Spectral, alpha: float, L: int) -> float:
    """Thm. 2, third statement (cos_{c,min})."""
    N = sp.lam.size
    return float(2.0 * (L + 1) * math.sqrt(N - sp.r_neg1) * abs(sin_pi(alpha))
                 / (math.pi * sp.cos_c_min * ((L + 1) ** 2 - alpha ** 2)))


def parseval_tail(alpha: float, L: int, terms: int = 2_000_000) -> float:
    """sum_{|n|>L} |c_n(alpha)|^2 (Sec. IV-A, Parseval prediction), summed in closed form
    sin^2(pi a)/pi^2 * sum 1/(a-n)^2 with a tail integral for n beyond ``terms``."""
    s2 = sin_pi(alpha) ** 2
    n = np.arange(L + 1, L + 1 + terms, dtype=np.float64)
    tot = np.sum(1.0 / (alpha - n) ** 2) + np.sum(1.0 / (alpha + n) ** 2)
    far = L + 1 + terms
    tot += 1.0 / (far - 0.5 - alpha) + 1.0 / (far - 0.5 + alpha)  # Euler-Maclaurin tail
    return float(s2 / math.pi ** 2 * tot)


def nmse(E: np.ndarray) -> float:
    """NMSE = ||E||_F^2 / N (Sec. IV-A)."""
    return float(np.linalg.norm(E) ** 2 / E.shape[0])


def rel_fro(A: np.ndarray, B: np.ndarray) -> float:
    """||A - B||_F / ||B||_F."""
    return float(np.linalg.norm(np.asarray(A) - np.asarray(B)) / np.linalg.norm(np.asarray(B)))
