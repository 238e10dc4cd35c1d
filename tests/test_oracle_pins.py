"""Pins for the FP64 oracle against facts the paper and mathematics fix.

None of these re-types an oracle formula: each compares the oracle with an
independent route (numerical integration, closed-form spectral projectors of
matrices with F^4 = I, FFT diagonalisation of a cyclic shift, repeated
products, finite differences, torch autograd, the paper's printed numbers,
the paper's bounds).
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

from oracle import fgfrft_oracle as O
from paper_2602_20870_gb300 import workloads as W
from tests.conftest import golden

rng = np.random.default_rng(1234)


# ---------------------------------------------------------------- scalars
@pytest.mark.parametrize("alpha", [0.37, -1.3, 0.5, 1.999, -0.001, 2.75])
def test_coeffs_equal_fourier_integral(alpha):
    """Sec. III-A: c_n = (1/2pi) int_{-pi}^{pi} e^{j(alpha-n)theta} dtheta, by quadrature."""
    L = 12
    c = O.coeffs(alpha, L)
    for i, n in enumerate(range(-L, L + 1)):
        re, _ = scipy.integrate.quad(lambda t: math.cos((alpha - n) * t), -math.pi, math.pi,
                                     limit=200, epsabs=1e-14, epsrel=1e-13)
        im, _ = scipy.integrate.quad(lambda t: math.sin((alpha - n) * t), -math.pi, math.pi,
                                     limit=200, epsabs=1e-14, epsrel=1e-13)
        assert abs(c[i] - re / (2 * math.pi)) < 1e-12
        assert abs(im) < 1e-12


@pytest.mark.parametrize("k", [-5, -1, 0, 1, 3, 7])
def test_coeffs_integer_order_is_kronecker_delta(k):
    """Remark 2: alpha in Z gives c_n = delta_{n, alpha} (exactly)."""
    c = O.coeffs(float(k), 8)
    ref = np.zeros(17)
    if abs(k) <= 8:
        ref[k + 8] = 1.0
    assert np.array_equal(c, ref)
    # the derivative of the sinc vanishes at its own peak
    assert O.dcoeffs(float(k), 8)[k + 8] == 0.0 if abs(k) <= 8 else True


def test_coeffs_reflection():
    """Proof of Prop. 2: c_n(-alpha) = c_{-n}(alpha)."""
    for a in [0.1, 0.37, 1.6, -1.9]:
        assert np.allclose(O.coeffs(-a, 20), O.coeffs(a, 20)[::-1], rtol=0, atol=1e-16)


def test_coeffs_parseval_identity():
    """sum_n |c_n|^2 = (1/2pi) int |e^{j alpha theta}|^2 = 1 (Parseval), so the tail equals
    1 - sum_{|n|<=L} c_n^2, and behaves like 2 sin^2(pi a)/(pi^2 L) (Sec. IV-A)."""
    for a in [0.15, 0.55, 0.95, 1.3]:
        for L in [10, 30, 100]:
            head = np.sum(O.coeffs(a, L) ** 2)
            assert abs(O.parseval_tail(a, L) - (1.0 - head)) < 1e-12
        L = 4000
        assert abs(O.parseval_tail(a, L) / (2 * math.sin(math.pi * a) ** 2 / (math.pi ** 2 * L)) - 1) < 2e-3


def test_sin_cos_pi_exact_points():
    for k in range(-6, 7):
        assert O.sin_pi(k) == 0.0
        assert O.cos_pi(k) == (1.0 if k % 2 == 0 else -1.0)
        assert O.cos_pi(k + 0.5) == 0.0
        assert abs(O.sin_pi(k + 0.5)) == 1.0
    for a in rng.uniform(-3, 3, 200):
        assert abs(O.sin_pi(a) - math.sin(math.pi * a)) < 4e-15
        assert abs(O.cos_pi(a) - math.cos(math.pi * a)) < 4e-15
        assert abs(O.phase(a) - np.exp(1j * math.pi * a)) < 4e-15


def test_series_converges_inside_and_to_midpoint_at_pi():
    """Remark 1: the series tends to e^{j alpha theta} for theta in (-pi, pi) and to
    cos(pi alpha) at theta = pi; the error obeys Thm. 1."""
    a = 0.55
    th = np.array([-2.5, -1.0, 0.0, 0.4, 2.9])
    for L in [50, 400]:
        err = np.abs(O.trunc_error(th, a, L))
        assert np.all(err <= O.pointwise_bound(th, a, L) * (1 + 1e-12))
    big = O.series_value(np.array([math.pi]), a, 20000)[0]
    assert abs(big - math.cos(math.pi * a)) < 1e-4


def _fd(f, a, h):
    return (f(a + h) - f(a - h)) / (2 * h)


@pytest.mark.parametrize("alpha", [0.37, -1.21, 1.5, 0.9995, 2.0004, 3.0])
def test_dcoeffs_against_central_difference(alpha):
    """Prop. 3: dc_n/dalpha, checked by a FP64 central difference of the sinc."""
    L = 10
    dc = O.dcoeffs(alpha, L)
    for i, n in enumerate(range(-L, L + 1)):
        g = lambda a: math.sin(math.pi * (a - n)) / (math.pi * (a - n)) if a != n else 1.0
        fd = _fd(g, alpha, 1e-5)
        assert abs(dc[i] - fd) < 2e-9, (n, dc[i], fd)


def test_dcoeffs_against_torch_autograd():
    torch = pytest.importorskip("torch")
    for alpha in [0.37, -1.7, 1.25]:
        a = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
        n = torch.arange(-8, 9, dtype=torch.float64)
        c = torch.sin(math.pi * (a - n)) / (math.pi * (a - n))
        grads = [torch.autograd.grad(c[i], a, retain_graph=True)[0].item() for i in range(17)]
        assert np.allclose(O.dcoeffs(alpha, 8), grads, rtol=0, atol=1e-13)


# ------------------------------------------- closed forms: F^4 = I (DFT), cyclic shift
def _dft_closed_forms(F, alpha, L):
    """Eigensolver-free spectral projectors of F with F^4 = I: P_lam = 1/4 sum_k lam^-k F^k.
    Returns (exact F^alpha, Q_L^alpha) built from them."""
    N = F.shape[0]
    Fk = [np.eye(N), F, F @ F, F @ F @ F]
    lams = {1: 0.0, -1j: -math.pi / 2, -1: math.pi, 1j: math.pi / 2}
    exact = np.zeros((N, N), complex)
    Q = np.zeros((N, N), complex)
    n = np.arange(-L, L + 1)
    c = O.coeffs(alpha, L)
    for lam, th in lams.items():
        Pl = sum(lam ** (-k) * Fk[k] for k in range(4)) / 4
        exact += np.exp(1j * alpha * th) * Pl
        if lam == -1:
            Q += np.exp(1j * math.pi * alpha) * Pl
        else:
            Q += np.sum(c * np.exp(1j * n * th)) * Pl
    return exact, Q


@pytest.mark.parametrize("N", [4, 12, 16])
@pytest.mark.parametrize("alpha", [0.37, -1.45, 1.0, 2.5])
def test_dft_brute_force(N, alpha):
    """Unitary DFT (F^4 = I): closed-form F^alpha and Q_L from the four spectral projectors."""
    F = W.dft_matrix(N)
    L = 6
    exact, Q = _dft_closed_forms(F, alpha, L)
    sp = O.spectral(F)
    assert np.abs(O.exact_gfrft(F, alpha, sp) - exact).max() < 1e-12
    assert np.abs(O.fgfrft_spectral(F, alpha, L, sp) - Q).max() < 1e-12
    assert np.abs(O.fgfrft_power(F, alpha, L) - Q).max() < 1e-12
    X = W.complex_normal((N, 3), rng)
    assert np.abs(O.apply_power(F, alpha, L, X) - Q @ X).max() < 1e-12
    if N == 4:
        assert sorted(np.round(sp.theta, 12)) == sorted([0.0, 0.0, round(math.pi, 12), round(-math.pi / 2, 12)])


@pytest.mark.parametrize("N", [7, 32])
def test_cyclic_shift_by_fft(N):
    """Cyclic shift: eigenvalues e^{-2 pi j k/N} on Fourier modes; F^alpha x and Q_L x by FFT."""
    C = W.cyclic_shift(N)
    k = np.arange(N)
    th = np.angle(np.exp(-2j * math.pi * k / N))
    if N % 2 == 0:
        th[N // 2] = math.pi
    L = 9
    X = W.complex_normal((N, 4), rng)
    alphas = np.array([0.37, -0.8, 1.7, 0.5])
    Xf = np.fft.fft(X, axis=0)
    ex = np.empty_like(X)
    qx = np.empty_like(X)
    for j, a in enumerate(alphas):
        ex[:, j] = np.fft.ifft(Xf[:, j] * np.exp(1j * a * th))
        q = O.series_value(th, a, L)  # scalar series on each mode; -1 mode exact
        if N % 2 == 0:
            q[N // 2] = np.exp(1j * math.pi * a)
        qx[:, j] = np.fft.ifft(Xf[:, j] * q)
    assert np.abs(O.apply_power(C, alphas, L, X) - qx).max() < 1e-12
    sp = O.spectral(C)
    assert sp.r_neg1 == (1 if N % 2 == 0 else 0)
    for j, a in enumerate(alphas):
        assert np.abs(O.exact_gfrft(C, a, sp) @ X[:, j] - ex[:, j]).max() < 1e-12
        assert np.abs(O.fgfrft_power(C, a, L) @ X[:, j] - qx[:, j]).max() < 1e-12


def test_minus_identity_is_exact_for_every_L():
    """Thm. 2 preamble: r_-1 = N (F = -I) gives Q_L = e^{j pi alpha} I for every L."""
    N = 8
    F = -np.eye(N, dtype=complex)
    for L in [0, 1, 5]:
        for a in [0.3, -1.7]:
            ref = np.exp(1j * math.pi * a) * np.eye(N)
            assert np.abs(O.fgfrft_power(F, a, L) - ref).max() < 1e-14
            assert np.abs(O.fgfrft_spectral(F, a, L) - ref).max() < 1e-14
            assert np.abs(O.exact_gfrft(F, a) - ref).max() < 1e-14


@pytest.mark.parametrize("flip", [False, True])
def test_integer_orders_and_boundaries(flip):
    """Sec. II-B: F^0 = I, F^1 = F; Def. 1: integer alpha gives F^alpha (repeated products)."""
    F = W.tiny(flip_one=flip).F
    N = F.shape[0]
    L = 4
    assert np.abs(O.fgfrft_power(F, 0.0, L) - np.eye(N)).max() < 1e-12
    assert np.abs(O.fgfrft_power(F, 1.0, L) - F).max() < 1e-12
    assert np.abs(O.exact_gfrft(F, 1.0) - F).max() < 1e-12
    assert np.abs(O.exact_gfrft(F, 0.0) - np.eye(N)).max() < 1e-12
    for k in [2, -1, -3, 6]:
        ref = np.linalg.matrix_power(F, k) if k >= 0 else np.linalg.matrix_power(F.conj().T, -k)
        assert np.abs(O.fgfrft_power(F, float(k), L) - ref).max() < 1e-11
        assert np.abs(O.exact_gfrft(F, float(k)) - ref).max() < 1e-11
        X = W.complex_normal((N, 2), rng)
        assert np.abs(O.apply_power(F, float(k), L, X) - ref @ X).max() < 1e-11


# ---------------------------------------------------- identities of Sec. III
def _cases():
    yield "tiny", W.tiny().F
    yield "tiny-flip", W.tiny(flip_one=True).F
    yield "haar64", W.random_unitary(64, 11)
    yield "prescribed", W.prescribed_spectrum_unitary(48, 5, 3)


@pytest.mark.parametrize("name,F", list(_cases()))
def test_form_S_equals_form_P(name, F):
    """Def. 1 on the spectrum vs Algorithm 1 with stored powers: <= 1e-12 relative."""
    sp = O.spectral(F)
    P = O.projector(F, sp)
    for L in [3, 16]:
        M = O.powers(F, L, P)
        for a in [0.37, -1.62, 0.5]:
            assert O.rel_fro(O.fgfrft_power(F, a, L, P, M), O.fgfrft_spectral(F, a, L, sp)) < 1e-12


@pytest.mark.parametrize("name,F", list(_cases()))
def test_adjoint_symmetry(name, F):
    """Prop. 2: Q_L^{-alpha} = (Q_L^alpha)^H, and the signal adjoint is apply at -alpha."""
    L = 7
    for a in [0.37, 1.4]:
        Qp = O.fgfrft_power(F, a, L)
        Qm = O.fgfrft_power(F, -a, L)
        assert np.abs(Qm - Qp.conj().T).max() < 1e-13
        G = W.complex_normal((F.shape[0], 3), rng)
        assert np.abs(O.adjoint_apply(F, a, L, G) - Qp.conj().T @ G).max() < 1e-12


def test_projector_properties():
    """Sec. III-B: P_-1 is an orthogonal projector, F P = -P, rank r_-1; P_c commutes with F."""
    for F in [W.tiny(flip_one=True).F, W.prescribed_spectrum_unitary(40, 6, 9), W.dft_matrix(12)]:
        sp = O.spectral(F)
        P = O.projector(F, sp)
        assert np.abs(P @ P - P).max() < 1e-13
        assert np.abs(P - P.conj().T).max() < 1e-14
        assert np.abs(F @ P + P).max() < 1e-13
        assert abs(np.trace(P).real - sp.r_neg1) < 1e-12
    assert O.spectral(W.dft_matrix(12)).r_neg1 == 3  # DFT_12: multiplicity of -1 is 3


def test_apply_matches_matrix_per_column():
    F = W.tiny(flip_one=True).F
    L = 16
    X = W.complex_normal((64, 5), rng)
    a = np.array([0.37, -1.1, 1.9, 0.0, -2.0])
    Y = O.apply_power(F, a, L, X)
    for j in range(5):
        assert np.abs(Y[:, j] - O.fgfrft_power(F, a[j], L) @ X[:, j]).max() < 1e-12


# ------------------------------------------------ error analysis (Thm. 1-2, Props. 4-6)
def test_frobenius_identity_and_bounds():
    """Thm. 2: ||F^a - Q_L||_F (matrices, power form) equals sqrt(sum |R_L(theta_k)|^2)
    (scalars) and lies below both bounds; all shrink with L."""
    F = W.random_unitary(200, 5)
    sp = O.spectral(F)
    P = O.projector(F, sp)
    M = O.powers(F, 24, P)
    for a in [0.37, 0.55, -1.3]:
        exact = O.exact_gfrft(F, a, sp)
        prev = math.inf
        for L in [4, 8, 16, 24]:
            if L <= abs(a):
                continue
            err = np.linalg.norm(exact - O.fgfrft_power(F, a, L, P, M[:L + 1]))
            ident = O.frobenius_error_exact(sp, a, L)
            assert abs(err - ident) < 1e-10 * max(1.0, ident)
            assert err <= O.frobenius_bound_tight(sp, a, L) * (1 + 1e-12)
            assert O.frobenius_bound_tight(sp, a, L) <= O.frobenius_bound_simplified(sp, a, L) * (1 + 1e-12)
            assert err < prev
            prev = err


def test_pointwise_bound_is_tight_to_its_asymptotic_constant():
    """Thm. 1 from both sides.  Each tail of R_L(theta) = sum_{|n|>L} c_n e^{jn theta} is an
    alternating-sign series with terms sin(pi a)/(pi (a - n)); summed in closed form its
    modulus is asymptotically |sin(pi a)| / (pi L |1 + e^{j theta}|) = |sin(pi a)| /
    (2 pi L cos(theta/2)), and the two tails rotate as e^{+-j(L+1) theta}.  Their moduli add
    somewhere in every theta window of width pi/(L+1), where |R_L| reaches half of the
    bound |sin(pi a)|/(pi cos(theta/2)) (1/(L+1-a) + 1/(L+1+a)) ~ 2|sin(pi a)|/(pi L
    cos(theta/2)).  So the windowed maximum of |R_L| / bound lies just above 1/2: a bound
    with a wrong cosine argument or an extra factor fails one side."""
    for a in [0.5, 0.37, -1.3, 1.9]:
        for L in [10, 30, 60]:
            for t0 in [0.5, 1.5, 2.5, -2.0]:
                th = np.linspace(t0, t0 + math.pi / (L + 1), 400)
                ratio = np.abs(O.trunc_error(th, a, L)) / O.pointwise_bound(th, a, L)
                assert ratio.max() <= 1.0
                assert 0.5 <= ratio.max() <= 0.5 + 0.25 / L, (a, L, t0, ratio.max())


def test_bound_values_by_hand_and_between_the_two_theorems():
    """Hand values: at theta = 0, a = 1/2, L = 1 the Thm. 1 bound is (1/pi)(1/1.5 + 1/2.5);
    at theta = 2 pi/3 (cos(theta/2) = 1/2) twice that.  For F = j I_4 (every theta = pi/2,
    cos(theta/2) = 1/sqrt 2) Thm. 2's two bounds coincide and equal
    2 (L+1) |sin(pi a)| sqrt(N) / (pi cos (L+1)^2 - a^2)) = 8 sqrt 2 / (3.75 pi).
    Across the theorems: the tight Frobenius bound is the root sum of squares of the
    pointwise bounds over the complement (the per-eigenvalue form of Thm. 2)."""
    b = O.pointwise_bound(np.array([0.0, 2 * math.pi / 3]), 0.5, 1)
    v = (1 / 1.5 + 1 / 2.5) / math.pi
    assert abs(b[0] - v) < 1e-15 and abs(b[1] - 2 * v) < 1e-15
    sp = O.spectral(1j * np.eye(4))
    want = 8 * math.sqrt(2) / (3.75 * math.pi)
    assert abs(O.frobenius_bound_tight(sp, 0.5, 1) - want) < 1e-14
    assert abs(O.frobenius_bound_simplified(sp, 0.5, 1) - want) < 1e-14
    for F in [W.random_unitary(60, 3), W.prescribed_spectrum_unitary(50, 2, 9), W.tiny().F]:
        sp = O.spectral(F)
        comp = ~sp.neg1
        for a, L in [(0.37, 8), (-1.3, 20), (1.9, 40)]:
            rss = math.sqrt(np.sum(O.pointwise_bound(sp.theta[comp], a, L) ** 2))
            assert abs(O.frobenius_bound_tight(sp, a, L) - rss) < 1e-12 * rss
            # and the simplified bound replaces every cosine by the smallest one
            n = int(comp.sum())
            worst = O.pointwise_bound(np.array([2 * math.acos(sp.cos_c_min)]), a, L)[0]
            assert abs(O.frobenius_bound_simplified(sp, a, L) - math.sqrt(n) * worst) < 1e-12 * worst * n


def test_bound_pins_catch_planted_mistakes(monkeypatch):
    """cos(theta) for cos(theta/2), or a bound loosened by a constant, fails the pins above."""
    real = O.pointwise_bound
    L, a = 30, 0.37
    th = np.linspace(2.5, 2.5 + math.pi / (L + 1), 400)
    for bad in (lambda t, al, LL: real(2 * np.asarray(t), al, LL),
                lambda t, al, LL: 2.0 * real(t, al, LL)):
        monkeypatch.setattr(O, "pointwise_bound", bad)
        r = np.abs(O.trunc_error(th, a, L)) / O.pointwise_bound(th, a, L)
        assert not (r.max() <= 1.0 and 0.5 <= r.max() <= 0.5 + 0.25 / L)
    monkeypatch.undo()


def test_unitarity_reconstruction_additivity_bounds():
    """Props. 4-6: ||Q^H Q - I|| <= 2e + e^2; ||x^ - x|| <= (2e + e^2)||x||; additivity defect."""
    F = W.random_unitary(120, 8)
    sp = O.spectral(F)
    L = 10
    eps = lambda g: np.linalg.norm(O.exact_gfrft(F, g, sp) - O.fgfrft_spectral(F, g, L, sp))
    for a, b in [(0.37, 0.55), (-1.2, 0.7), (0.9, -0.9)]:
        Qa = O.fgfrft_spectral(F, a, L, sp)
        Qb = O.fgfrft_spectral(F, b, L, sp)
        ea, eb, eab = eps(a), eps(b), eps(a + b)
        assert np.linalg.norm(Qa.conj().T @ Qa - np.eye(120)) <= 2 * ea + ea ** 2 + 1e-12
        x = W.complex_normal(120, rng)
        assert np.linalg.norm(Qa.conj().T @ Qa @ x - x) <= (2 * ea + ea ** 2) * np.linalg.norm(x) + 1e-12
        defect = np.linalg.norm(Qa @ Qb - O.fgfrft_spectral(F, a + b, L, sp))
        assert defect <= eab + ea + eb + ea * eb + 1e-12


@pytest.mark.slow
def test_paper_rate_table_random_unitary():
    """Sec. IV-C, Table tab:rate_verification (N=2000, alpha=0.55): the NMSE of the oracle's
    truncation (Thm. 2 identity on the spectrum of a Haar unitary) matches the printed
    values within 5%, and the Parseval tail within 2%."""
    F = W.random_unitary(2000, 2000)
    th = np.angle(scipy.linalg.eigvals(F))
    a = 0.55
    for Ls, val in golden("rate_verification.txt"):
        L, ref = int(Ls), float(val)
        nm = np.sum(np.abs(O.trunc_error(th, a, L)) ** 2) / th.size
        assert abs(nm / ref - 1) < 0.05, (L, nm, ref)
        assert abs(O.parseval_tail(a, L) / ref - 1) < 0.02
    r = {float(x): float(v) for x, v in golden("alpha_ratio.txt")}
    n15 = np.sum(np.abs(O.trunc_error(th, 0.15, 10)) ** 2) / th.size
    n55 = np.sum(np.abs(O.trunc_error(th, 0.55, 10)) ** 2) / th.size
    assert abs((n15 / n55) / (r[0.15] / r[0.55]) - 1) < 0.05
    assert abs(n55 / r[0.55] - 1) < 0.05


def test_paper_efficiency_table_nmse_at_1000():
    """Sec. IV-D, Table tab:efficiency_accuracy at N=1000 (L=10, alpha=0.5): matrix-level
    NMSE of the power form against the exact GFRFT is ~2.0e-2 (printed 2.05e-2), and
    MSE = NMSE/N, MAE <= sqrt(MSE)."""
    N = 1000
    row = [r for r in golden("efficiency_accuracy.txt") if r[0] == "1000"][0]
    F = W.random_unitary(N, 1000)
    sp = O.spectral(F)
    P = O.projector(F, sp)
    E = O.exact_gfrft(F, 0.5, sp) - O.fgfrft_power(F, 0.5, 10, P)
    nm = O.nmse(E)
    assert abs(nm / float(row[3]) - 1) < 0.06
    mse = nm / N
    assert abs(mse / float(row[1]) - 1) < 0.06
    mae = np.mean(np.abs(E))
    assert mae <= math.sqrt(mse)
    assert abs(mae / float(row[2]) - 1) < 0.1


def test_neg1_block_exact_structure():
    """Sec. IV-E: with r_-1 eigenvalues at -1, the proposed form has E_-1 at round-off and
    E_total = E_c, while the standard truncated form has E_-1 of order sqrt(r)|e^{j pi a} - cos(pi a)|."""
    N, r, a = 160, 8, 0.55
    F = W.prescribed_spectrum_unitary(N, r, 21)
    sp = O.spectral(F)
    assert sp.r_neg1 == r
    P = O.projector(F, sp)
    Pc = np.eye(N) - P
    ex = O.exact_gfrft(F, a, sp)
    for L in [10, 20]:
        prop = O.fgfrft_power(F, a, L, P)
        std = sum(cn * O.integer_power(F, n) for cn, n in zip(O.coeffs(a, L), range(-L, L + 1)))
        e_tot = np.linalg.norm(prop - ex)
        e_m1 = np.linalg.norm(P @ (prop - ex) @ P)
        e_c = np.linalg.norm(Pc @ (prop - ex) @ Pc)
        assert e_m1 < 1e-12
        assert abs(e_tot - e_c) < 1e-12 * e_tot
        s_m1 = np.linalg.norm(P @ (std - ex) @ P)
        # on the -1 block the standard series tends to cos(pi a) instead of e^{j pi a}
        assert abs(s_m1 - math.sqrt(r) * abs(np.exp(1j * math.pi * a) - math.cos(math.pi * a))) < 0.1
        assert np.linalg.norm(std - ex) > e_tot


# ------------------------------------------------------ derivative and gradient
def test_dalpha_apply_against_finite_difference():
    """Prop. 3: D = dQ/dalpha X, against a FP64 central difference of apply_power (h=1e-5)."""
    F = W.tiny(flip_one=True).F
    L = 16
    X = W.complex_normal((64, 4), rng)
    a = np.array([0.37, -1.3, 1.62, 0.5])
    D = O.dalpha_apply(F, a, L, X)
    h = 1e-5
    fd = (O.apply_power(F, a + h, L, X) - O.apply_power(F, a - h, L, X)) / (2 * h)
    assert O.rel_fro(D, fd) < 1e-8


def test_grad_alpha_of_real_loss():
    """Chain rule: d/d alpha_j of sum |Y - T|^2 equals Re sum conj(G) D with G = 2 (Y - T)."""
    F = W.tiny().F
    L = 12
    X = W.complex_normal((64, 3), rng)
    T = W.complex_normal((64, 3), rng)
    a = np.array([0.2, -0.7, 1.1])
    loss = lambda al: np.sum(np.abs(O.apply_power(F, al, L, X) - T) ** 2, axis=0)
    Y = O.apply_power(F, a, L, X)
    g = O.grad_alpha(2 * (Y - T), O.dalpha_apply(F, a, L, X))
    h = 1e-6
    fd = (loss(a + h) - loss(a - h)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-7, atol=1e-7)


# ---------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes(monkeypatch):
    """A wrong index direction, a dropped -1 term or a transposed negative power in the
    oracle each break at least one pin above (mutations are planted on the CPU only)."""
    F = W.dft_matrix(12)
    L, a = 6, 0.37
    _, Q = _dft_closed_forms(F, a, L)
    good = O.fgfrft_power(F, a, L)
    assert np.abs(good - Q).max() < 1e-12
    real = O.coeffs
    monkeypatch.setattr(O, "coeffs", lambda al, LL: real(al, LL)[::-1])
    assert np.abs(O.fgfrft_power(F, a, L) - Q).max() > 1e-3
    monkeypatch.setattr(O, "coeffs", real)
    monkeypatch.setattr(O, "phase", lambda al: 0.0)
    assert np.abs(O.fgfrft_power(F, a, L) - Q).max() > 1e-3
    monkeypatch.undo()
    # transposed powers: the DFT is symmetric, so use the cyclic shift and its FFT form
    N = 16
    C = W.cyclic_shift(N)
    th = np.angle(np.exp(-2j * math.pi * np.arange(N) / N))
    th[N // 2] = math.pi
    q = O.series_value(th, a, L)
    q[N // 2] = np.exp(1j * math.pi * a)
    x = W.complex_normal(N, rng)
    ref = np.fft.ifft(np.fft.fft(x) * q)
    P = O.projector(C)
    assert np.abs(O.fgfrft_power(C, a, L, P) @ x - ref).max() < 1e-12
    Mt = [m.T for m in O.powers(C, L, P)]
    assert np.abs(O.fgfrft_power(C, a, L, P, Mt) @ x - ref).max() > 1e-3
