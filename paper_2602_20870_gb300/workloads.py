"""Seeded synthetic inputs for the FGFRFT hot path.

This module holds no FGFRFT arithmetic: it only builds graphs, their GFT
matrices (Sec. II-A: F = U^H from the eigen-decomposition of a symmetric
graph-shift operator), test unitaries, signals and transform orders.  Both the
CUDA path and the FP64 oracle consume what it returns, so it is the one module
that the two sides share.

Every generator takes an explicit seed and uses ``numpy.random.default_rng``.
The workloads stand in for the paper's datasets (Set12 image patches, the
MVUB point clouds, Sec. V-B), which are not available here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------
# graphs and their GFT matrices (Sec. II-A)
# ----------------------------------------------------------------------------
def knn_gaussian_adjacency(points: np.ndarray, k: int, sigma2: float) -> np.ndarray:
    """Symmetric k-NN adjacency with weights exp(-d^2 / sigma2); A = max(A, A^T)."""
    pts = np.asarray(points, dtype=np.float64)
    n = pts.shape[0]
    d2 = np.sum((pts[:, None, :] - pts[None, :, :]) ** 2, axis=-1)
    np.fill_diagonal(d2, np.inf)
    nbr = np.argpartition(d2, kth=k - 1, axis=1)[:, :k]
    A = np.zeros((n, n), dtype=np.float64)
    rows = np.repeat(np.arange(n), k)
    cols = nbr.reshape(-1)
    A[rows, cols] = np.exp(-d2[rows, cols] / sigma2)
    return np.maximum(A, A.T)


def grid_adjacency(h: int, w: int) -> np.ndarray:
    """4-connected h x w grid with unit weights (row-major node order)."""
    n = h * w
    A = np.zeros((n, n), dtype=np.float64)
    for r in range(h):
        for c in range(w):
            i = r * w + c
            if c + 1 < w:
                A[i, i + 1] = A[i + 1, i] = 1.0
            if r + 1 < h:
                A[i, i + w] = A[i + w, i] = 1.0
    return A


def laplacian(A: np.ndarray) -> np.ndarray:
    """Combinatorial Laplacian D - A."""
    return np.diag(A.sum(axis=1)) - A


def gft_from_gso(Z: np.ndarray, flip_one: bool = False) -> np.ndarray:
    """F = U^H with Z = U diag U^H (Sec. II-A), returned as complex128.

    Eigenvector signs are made canonical (largest-magnitude entry positive) so
    that F does not depend on the LAPACK sign convention; ``flip_one`` negates
    one eigenvector, which flips det F and so toggles whether -1 is an
    eigenvalue of the (real orthogonal) F.
    """
    _, U = np.linalg.eigh(np.asarray(Z, dtype=np.float64))
    idx = np.argmax(np.abs(U), axis=0)
    sgn = np.sign(U[idx, np.arange(U.shape[1])])
    sgn[sgn == 0] = 1.0
    U = U * sgn[None, :]
    if flip_one:
        U[:, 0] = -U[:, 0]
    return np.ascontiguousarray(U.T).astype(np.complex128)


def random_unitary(n: int, seed: int) -> np.ndarray:
    """Haar-like unitary from the QR of a complex Gaussian matrix (Sec. IV-A setup)."""
    rng = np.random.default_rng(seed)
    G = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2.0)
    Qm, R = np.linalg.qr(G)
    d = np.diag(R)
    return Qm * (d / np.abs(d))[None, :]


def dft_matrix(n: int) -> np.ndarray:
    """Unitary DFT matrix F_{mk} = exp(-2 pi j m k / n) / sqrt(n)."""
    m = np.arange(n)
    return np.exp(-2j * math.pi * np.outer(m, m) / n) / math.sqrt(n)


def cyclic_shift(n: int) -> np.ndarray:
    """Cyclic shift (C x)_i = x_{i-1 mod n}, a unitary permutation matrix."""
    C = np.zeros((n, n), dtype=np.complex128)
    C[np.arange(n), (np.arange(n) - 1) % n] = 1.0
    return C


def prescribed_spectrum_unitary(n: int, r_neg1: int, seed: int, margin: float = 0.05) -> np.ndarray:
    """V diag(lambda) V^H with r_neg1 eigenvalues equal to -1 and the other phases
    uniform in (-pi + margin, pi - margin), V Haar-like (Sec. IV-E setup)."""
    rng = np.random.default_rng(seed)
    V = random_unitary(n, seed + 7919)
    th = rng.uniform(-math.pi + margin, math.pi - margin, size=n)
    th[:r_neg1] = math.pi
    lam = np.exp(1j * th)
    lam[:r_neg1] = -1.0
    return (V * lam[None, :]) @ V.conj().T


def unitary_with_phases(theta, seed: int) -> np.ndarray:
    """V diag(e^{j theta_k}) V^H for the given eigenphases, V Haar-like: a test unitary
    whose distances |lambda_k + 1| = 2 |cos(theta_k / 2)| are known exactly."""
    th = np.asarray(theta, dtype=np.float64)
    V = random_unitary(th.size, seed)
    return (V * np.exp(1j * th)[None, :]) @ V.conj().T


# ----------------------------------------------------------------------------
# signals
# ----------------------------------------------------------------------------
def gaussian_random_field(h: int, w: int, ell: float, count: int, rng) -> np.ndarray:
    """White noise filtered by exp(-d^2 / (2 ell^2)) on an h x w torus, unit variance.
    Returns (count, h*w) float64."""
    ky = np.fft.fftfreq(h)[:, None]
    kx = np.fft.fftfreq(w)[None, :]
    # Fourier transform of a unit-width Gaussian kernel of std ell (in pixels)
    kern = np.exp(-2.0 * math.pi ** 2 * ell ** 2 * (kx ** 2 + ky ** 2))
    wn = rng.standard_normal((count, h, w))
    f = np.real(np.fft.ifft2(np.fft.fft2(wn) * kern[None]))
    f = f.reshape(count, -1)
    f = (f - f.mean(axis=1, keepdims=True)) / f.std(axis=1, keepdims=True)
    return f


def complex_normal(shape, rng) -> np.ndarray:
    """Complex N(0, 1): real and imaginary parts iid N(0, 1/2)."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------
@dataclass
class Workload:
    """One synthetic workload: GFT matrix, truncation order, orders and signals.

    ``X`` is (B, N) complex128, one signal per row (each signal contiguous);
    ``alpha`` has one order per signal row.
    """
    name: str
    F: np.ndarray
    L: int
    alpha: np.ndarray
    X: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.F.shape[0]

    @property
    def B(self) -> int:
        return self.X.shape[0]


def tiny(seed: int = 1, flip_one: bool = False) -> Workload:
    """64 uniform points, 8-NN, w = exp(-d^2/0.01), Laplacian GFT; alpha=0.37, L=16, 4 real signals."""
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(64, 2))
    F = gft_from_gso(laplacian(knn_gaussian_adjacency(pts, 8, 0.01)), flip_one)
    X = rng.standard_normal((4, 64)).astype(np.complex128)
    return Workload("tiny N=64 L=16", F, 16, np.full(4, 0.37), X, {"points": pts})


def image_graph(seed: int = 2, n_orders: int = 64, per_order: int = 256, side: int = 32) -> Workload:
    """32x32 4-connected grid (N=1024), L=32, 64 orders in [-2,2], 256 GRF(ell=4)+N(0,0.1^2)
    signals per order (columns grouped by order)."""
    rng = np.random.default_rng(seed)
    F = gft_from_gso(laplacian(grid_adjacency(side, side)))
    alphas = rng.uniform(-2.0, 2.0, size=n_orders)
    sig = gaussian_random_field(side, side, 4.0, n_orders * per_order, rng)
    sig = sig + 0.1 * rng.standard_normal(sig.shape)
    return Workload(f"image-graph N={side*side} L=32 A={n_orders}x{per_order}", F, 32,
                    np.repeat(alphas, per_order), sig.astype(np.complex128),
                    {"orders": alphas, "per_order": per_order})


def surface_points(n: int, rng) -> np.ndarray:
    """n points on z = sum_{i=1}^{8} a_i sin(2 pi k_i . p + phi_i) over [0,1]^2."""
    p = rng.uniform(0.0, 1.0, size=(n, 2))
    a = rng.uniform(0.0, 0.1, size=8)
    k = rng.uniform(-3.0, 3.0, size=(8, 2))
    ph = rng.uniform(0.0, 2 * math.pi, size=8)
    z = np.sin(2 * math.pi * (p @ k.T) + ph[None, :]) @ a
    return np.column_stack([p, z])


def point_cloud(seed: int = 3, n: int = 2048, signals: int = 128, L: int = 48) -> Workload:
    """2048 points on an 8-sinusoid surface, 10-NN Gaussian graph, L=48; 128 three-channel
    (xyz + N(0, 0.02^2)) signals, one order per signal shared by its 3 channels."""
    rng = np.random.default_rng(seed)
    pts = surface_points(n, rng)
    F = gft_from_gso(laplacian(knn_gaussian_adjacency(pts, 10, 0.01)))
    alphas = rng.uniform(-2.0, 2.0, size=signals)
    X = np.empty((signals * 3, n), dtype=np.complex128)
    for s in range(signals):
        X[3 * s:3 * s + 3] = (pts + 0.02 * rng.standard_normal(pts.shape)).T
    return Workload(f"point-cloud N={n} L={L} B={signals}x3", F, L, np.repeat(alphas, 3), X,
                    {"points": pts, "orders": alphas})


def precision(seed: int = 4, n: int = 4096, signals: int = 1024, L: int = 64,
              shared_alpha: float | None = None) -> Workload:
    """4096-point random geometric graph, 12-NN Gaussian, L=64; 1024 complex N(0,1) signals.
    Per-column orders in [-2,2] unless ``shared_alpha`` is given."""
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(n, 2))
    F = gft_from_gso(laplacian(knn_gaussian_adjacency(pts, 12, 0.01)))
    X = complex_normal((signals, n), rng)
    if shared_alpha is None:
        alpha = rng.uniform(-2.0, 2.0, size=signals)
    else:
        alpha = np.full(signals, float(shared_alpha))
    return Workload(f"precision N={n} L={L} B={signals}", F, L, alpha, X)


def rgg_gft(n: int, seed: int, k: int = 12, sigma2: float = 0.01) -> np.ndarray:
    """GFT of a random geometric graph of n uniform points (serving graphs)."""
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(n, 2))
    return gft_from_gso(laplacian(knn_gaussian_adjacency(pts, min(k, n - 1), sigma2)))


@dataclass
class Request:
    """One serving request: graph index, kind, orders, truncation order and signals.

    ``X`` is (cols, N) complex128, or None for "assemble".  Requests made with
    ``lazy=True`` draw their signals from (seed, rid) when ``X`` is first read."""
    rid: int
    arrival_s: float
    graph: int
    kind: str            # "apply" | "grad" | "assemble"
    alpha: np.ndarray    # one per signal column ("assemble": one order)
    L: int
    _X: np.ndarray | None = None
    cols: int = 0
    N: int = 0
    seed: int = 0

    @property
    def X(self):
        if self._X is None and self.kind != "assemble" and self.cols:
            rng = np.random.default_rng([self.seed, self.rid])
            return complex_normal((self.cols, self.N), rng)
        return self._X


def serving_requests(sizes, count: int, rate_per_s: float, seed: int = 5,
                     Ls=(16, 32, 64), max_cols: int = 64, lazy: bool = False) -> list[Request]:
    """Poisson arrivals over resident graphs of the given sizes: graph uniform, alpha in
    [-2,2], L from ``Ls``, 1..max_cols N(0,1) signals, 60% apply / 30% grad / 10% assemble."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
    out = []
    for i in range(count):
        g = int(rng.integers(0, len(sizes)))
        u = rng.uniform()
        kind = "apply" if u < 0.6 else ("grad" if u < 0.9 else "assemble")
        L = int(rng.choice(Ls))
        if kind == "assemble":
            out.append(Request(i, float(t[i]), g, kind, np.array([rng.uniform(-2, 2)]), L))
            continue
        cols = int(rng.integers(1, max_cols + 1))
        a = np.full(cols, rng.uniform(-2.0, 2.0))
        X = None if lazy else complex_normal((cols, sizes[g]), rng)
        out.append(Request(i, float(t[i]), g, kind, a, L, X, cols, sizes[g], seed))
    return out
