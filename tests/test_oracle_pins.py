"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks re-types an oracle formula: each compares the oracle with
something independent of it (hand-derived values, numpy's FFT and polynomial
routines, pure-Python brute force, closed forms, identities between different
oracle functions), chosen so that a dropped term, a wrong sign or index, or a
transposed operand in any oracle routine fails at least one of them.
"""
import cmath
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lagrange_p2_p3.txt")


def _golden():
    cases = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            case, qty, idx, re, im = line.split()
            cases.setdefault(case, {}).setdefault(qty, {})[int(idx)] = complex(float(re), float(im))
    out = {}
    for case, q in cases.items():
        out[case] = {k: np.array([v[i] for i in range(len(v))]) for k, v in q.items()}
    return out


def test_golden_hand_derived():
    g = _golden()
    A = g["A"]
    x = 2 * np.pi * A["t"].real
    np.testing.assert_allclose(oracle.inv5(x, A["inv5_s"]), A["inv5_S"], atol=1e-15)
    np.testing.assert_allclose(oracle.inv4(x, A["inv4_A"]), A["inv4_a"], atol=1e-15)
    rho = A["rho"][0].real
    np.testing.assert_allclose(oracle.kernel_samples(x, rho), A["K"], atol=1e-15)
    D = oracle.deriv_samples(x)
    np.testing.assert_allclose(D, A["D"], atol=1e-15)
    np.testing.assert_allclose(oracle.weights(x, rho), A["w"], atol=1e-15)
    B = g["B"]
    x = 2 * np.pi * B["t"].real
    np.testing.assert_allclose(oracle.inv5(x, B["inv5_s"]), B["inv5_S"], atol=1e-15)
    np.testing.assert_allclose(oracle.deriv_samples(x), B["D"], atol=1e-14)


@pytest.mark.parametrize("P", [1, 2, 7, 16, 64, 96])
def test_equispaced_reduces_to_dft(P):
    """t_p = p/P: type-1 is the DFT of Eq. 0, type-2 is P*IDFT, and the
    inverses are DFT/P and IDFT (numpy's FFT is the independent reference)."""
    x = synth.equispaced_nodes(P)
    a = synth.cn01(P, seed=P)
    np.testing.assert_allclose(oracle.type1(x, a), np.fft.fft(a), rtol=0, atol=1e-12 * np.sqrt(P))
    np.testing.assert_allclose(oracle.type2(x, a), P * np.fft.ifft(a), rtol=0, atol=1e-12 * np.sqrt(P))
    np.testing.assert_allclose(oracle.inv5(x, a), np.fft.fft(a) / P, rtol=0, atol=1e-13)
    np.testing.assert_allclose(oracle.inv4(x, a), np.fft.ifft(a), rtol=0, atol=1e-13)


def test_type1_at_matches_type1():
    P = 40
    x = synth.jittered_nodes(P, 0.45, seed=71)
    a = synth.cn01(P, seed=72)
    ks = np.array([0, 3, 39, 7, 1000, -5])
    full = oracle.type1(x, a, k0=-5, M=1006)
    np.testing.assert_allclose(oracle.type1_at(x, a, ks), full[ks + 5], atol=1e-12)


def test_type2_at_matches_type2():
    """Coefficients at a scattered, unordered list of integer frequencies give
    the same sums as the contiguous type-2 with those coefficients placed in
    an otherwise zero vector; one term is the plain exponential."""
    P = 40
    x = synth.jittered_nodes(P, 0.45, seed=73)
    ms = np.array([3, 0, 999, -5, 7, 1000, 41])
    S = synth.cn01(ms.size, seed=74)
    full = np.zeros(1006, complex)
    full[ms + 5] = S
    np.testing.assert_allclose(oracle.type2_at(x, S, ms), oracle.type2(x, full, m0=-5), atol=1e-12)
    t = oracle.canon(x)[1]
    one = oracle.type2_at(x, np.array([1.0 + 0j]), np.array([123456789]))
    ref = np.array([cmath.exp(2j * math.pi * ((123456789 * ti) % 1.0)) for ti in t])
    np.testing.assert_allclose(one, ref, atol=1e-6)


@pytest.mark.parametrize("P", [1, 3, 5, 12])
def test_brute_force_python(P):
    """Pure-Python double loops with cmath.exp (no exact phases) vs the oracle."""
    g = synth.rng(100 + P)
    t = g.uniform(0, 1, size=P)
    x = 2 * np.pi * t
    a = synth.cn01(P, generator=g)
    A_bf = [sum(a[p] * cmath.exp(-2j * math.pi * k * t[p]) for p in range(P)) for k in range(P)]
    s_bf = [sum(a[m] * cmath.exp(2j * math.pi * m * t[q]) for m in range(P)) for q in range(P)]
    np.testing.assert_allclose(oracle.type1(x, a), A_bf, atol=1e-13)
    np.testing.assert_allclose(oracle.type2(x, a), s_bf, atol=1e-13)
    # the system matrix entry by entry
    G = oracle.matrix(x)
    for q in range(P):
        for m in range(P):
            assert abs(G[q, m] - cmath.exp(2j * math.pi * m * t[q])) < 5e-14  # cmath phase m*t rounds


def test_canon_wraps():
    x = np.array([0.0, -np.pi / 2, 2 * np.pi, 5 * np.pi / 2, np.pi])
    T, t = oracle.canon(x)
    np.testing.assert_allclose(t, [0.0, 0.75, 0.0, 0.25, 0.5], atol=1e-16)
    assert T[4] == np.uint64(1 << 63)


@pytest.mark.parametrize("P,umax", [(64, 0.3), (200, 0.45)])
def test_round_trips_known_truth(P, umax):
    """c -> type-2 -> type-5 -> c and a -> type-1 -> type-4 -> a (Eqs. 47, 48)."""
    x = synth.jittered_nodes(P, umax, seed=P)
    c = synth.cn01(P, seed=P + 1)
    np.testing.assert_allclose(oracle.inv5(x, oracle.type2(x, c)), c, atol=1e-12)
    np.testing.assert_allclose(oracle.inv4(x, oracle.type1(x, c)), c, atol=1e-12)
    G = oracle.matrix(x)
    s = synth.cn01(P, seed=P + 2)
    S = oracle.inv5(x, s)
    assert np.linalg.norm(G @ S - s) / np.linalg.norm(s) < 1e-13


def test_type4_type5_duality():
    """The type-4 matrix is the Hermitian of the type-5 matrix (Sec. VI), so
    <inv5 u, v> = <u, inv4 v> and <type2 u, v> = <u, type1 v>."""
    P = 80
    x = synth.jittered_nodes(P, 0.45, seed=7)
    u = synth.cn01(P, seed=8)
    v = synth.cn01(P, seed=9)
    lhs = np.vdot(v, oracle.inv5(x, u))
    rhs = np.vdot(oracle.inv4(x, v), u)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    lhs = np.vdot(v, oracle.type2(x, u))
    rhs = np.vdot(oracle.type1(x, v), u)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_translation_law():
    """Shifting every node by tau multiplies S_m by e^{-j 2 pi m tau} in the
    type-5 solution and A_k by e^{-j 2 pi k tau} in type-1."""
    P = 48
    tau = 0.125
    x = synth.jittered_nodes(P, 0.4, seed=11)
    s = synth.cn01(P, seed=12)
    m = np.arange(P)
    S0 = oracle.inv5(x, s)
    S1 = oracle.inv5(x + 2 * np.pi * tau, s)
    np.testing.assert_allclose(S1, S0 * np.exp(-2j * np.pi * m * tau), atol=1e-12)
    A0 = oracle.type1(x, s)
    A1 = oracle.type1(x + 2 * np.pi * tau, s)
    np.testing.assert_allclose(A1, A0 * np.exp(-2j * np.pi * m * tau), atol=1e-12)


@pytest.mark.parametrize("P", [1, 4, 33, 256])
def test_kernel_closed_forms_equispaced(P):
    """Equispaced nodes: L(z) = z^P - 1, so K_q = rho^P - 1, L'(z_p) z_p = P and
    w_p = 1/(P (rho^P - 1))."""
    rho = oracle.rho_of_gamma(P, 10.0)
    x = synth.equispaced_nodes(P)
    K = oracle.kernel_samples(x, rho)
    np.testing.assert_allclose(K, np.full(P, rho ** P - 1), atol=1e-12)
    D = oracle.deriv_samples(x)
    z = np.exp(2j * np.pi * np.arange(P) / P)
    np.testing.assert_allclose(D * z, np.full(P, P), rtol=1e-12)
    w = oracle.weights(x, rho, D)
    np.testing.assert_allclose(w, np.full(P, 1 / (P * (rho ** P - 1))), rtol=1e-12)


@pytest.mark.parametrize("P", [2, 9, 24])
def test_kernel_vs_numpy_polynomial(P):
    """K and L' against numpy's own expansion of prod (z - z_p) (np.poly) and
    its derivative (np.polyder), evaluated by np.polyval."""
    x = synth.jittered_nodes(P, 0.45, seed=P)
    t = oracle.canon(x)[1]
    z = np.exp(2j * np.pi * t)
    coeffs = np.poly(z)
    rho = oracle.rho_of_gamma(P, 10.0)
    zq = rho * np.exp(2j * np.pi * np.arange(P) / P)
    np.testing.assert_allclose(oracle.kernel_samples(x, rho), np.polyval(coeffs, zq), rtol=1e-9, atol=1e-10)  # expansion of 24 roots rounds ~1e-11
    np.testing.assert_allclose(oracle.deriv_samples(x), np.polyval(np.polyder(coeffs), z), rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("P,gamma", [(50, 10.0), (37, 1000.0)])
def test_lagrange_factorisation_identities(P, gamma):
    """Ties K, L' and w together through Sec. III without using the method:
    (i)  Lagrange formula at the shifted grid (Eq. 30):
         s(q/P + ja) = K_q * sum_p s(t_p) / (L'(z_p) (z_q - z_p));
    (ii) the band-limited kernel rewrite (Eqs. 22-25):
         w_p h1(q/P - t_p) = 1 / (L'(z_p) (z_q - z_p)),
         h1(t) = sum_{k<P} rho^k e^{j 2 pi k t}  (Eq. 36)."""
    x = synth.jittered_nodes(P, 0.45, seed=3 * P)
    t = oracle.canon(x)[1]
    c = synth.cn01(P, seed=5)
    rho = oracle.rho_of_gamma(P, gamma)
    K = oracle.kernel_samples(x, rho)
    D = oracle.deriv_samples(x)
    w = oracle.weights(x, rho, D)
    s = oracle.type2(x, c)
    m = np.arange(P)
    q = np.arange(P)
    zq = rho * np.exp(2j * np.pi * q / P)
    zp = np.exp(2j * np.pi * t)
    s_shift = (np.exp(2j * np.pi * np.outer(q, m) / P) * (rho ** m)) @ c
    cauchy = 1.0 / (D[None, :] * (zq[:, None] - zp[None, :]))
    np.testing.assert_allclose(K * (cauchy @ s), s_shift, rtol=1e-10, atol=1e-10 * np.abs(s_shift).max())
    h1 = (np.exp(2j * np.pi * np.subtract.outer(q / P, t)[:, :, None] * m[None, None, :]) * rho ** m).sum(-1)
    np.testing.assert_allclose(w[None, :] * h1, cauchy, rtol=1e-10, atol=1e-12 * np.abs(cauchy).max())


@pytest.mark.parametrize("P,gamma", [(16, 10.0), (24, 300.0)])
def test_middle_stage_convolution_identity(P, gamma):
    """The middle stage of Eqs. 37, 30, 31, S_m = rho^-m/P DFT(K P IDFT(rho^k A))_m
    (IDFT with 1/P), equals c_m + rho^P c_{m+P} with c the linear convolution of
    the coefficients L_0..L_P of prod (z - z_p) (Eqs. 11, 43) with A, which
    follows from Eqs. 10, 30 and 31 by expanding K_q = L(rho e^{j 2 pi q/P}):
    K from the oracle, L from numpy's own expansion (np.poly, which rounds
    badly beyond ~24 roots on the circle), the products by numpy."""
    x = synth.jittered_nodes(P, 0.45, seed=7 * P)
    t = oracle.canon(x)[1]
    A = synth.cn01(P, seed=11)
    rho = oracle.rho_of_gamma(P, gamma)
    K = oracle.kernel_samples(x, rho)
    k = np.arange(P)
    sigma = P * np.fft.ifft(rho ** k * A)
    S_scaled = rho ** (-k) / P * np.fft.fft(K * sigma)
    L = np.poly(np.exp(2j * np.pi * t))[::-1]          # L_0 .. L_P, L_P = 1
    c = np.convolve(L, A)                               # length 2P
    S_conv = c[:P] + rho ** P * c[P:2 * P]
    np.testing.assert_allclose(S_scaled, S_conv, rtol=1e-9, atol=1e-10 * np.abs(S_conv).max())


@pytest.mark.parametrize("which", ["inv5", "inv4"])
def test_vjp_against_finite_differences(which):
    """The oracle's gradients of L = ||inv(x, d) - c_t||^2 against central
    differences of the oracle itself (h = 1e-6 in x, and in Re/Im of d)."""
    P = 24
    x = synth.jittered_nodes(P, 0.45, seed=31)
    d = synth.cn01(P, seed=32)
    ct = synth.cn01(P, seed=33)
    solve = oracle.inv5 if which == "inv5" else oracle.inv4
    vjp = oracle.inv5_vjp if which == "inv5" else oracle.inv4_vjp

    def loss(xx, dd):
        r = solve(xx, dd) - ct
        return float(np.vdot(r, r).real)

    g_out = 2 * (solve(x, d) - ct)
    g_d, g_x = vjp(x, d, g_out)
    h = 1e-6
    for q in (0, 5, 11, 23):
        e = np.zeros(P)
        e[q] = h
        fd = (loss(x + e, d) - loss(x - e, d)) / (2 * h)
        assert abs(fd - g_x[q]) <= 1e-6 * max(1.0, abs(fd)), (q, fd, g_x[q])
        ed = np.zeros(P, complex)
        ed[q] = h
        fdr = (loss(x, d + ed) - loss(x, d - ed)) / (2 * h)
        fdi = (loss(x, d + 1j * ed) - loss(x, d - 1j * ed)) / (2 * h)
        assert abs(fdr + 1j * fdi - g_d[q]) <= 1e-6 * max(1.0, abs(g_d[q]))
