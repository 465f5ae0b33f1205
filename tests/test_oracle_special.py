"""Pins for the oracle's special functions: elliptic integrals, Q_{n-1/2}, G^(n).

Each test checks the oracle against something other than itself: a library routine
(scipy, mpmath), a textbook closed form, an identity, or brute-force quadrature.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# --- complete elliptic integrals (Carlson 1995, used for Eq. gfunc:Q0) -------------------

@pytest.mark.parametrize("k2", [0.0, 1e-8, 0.1, 0.3, 0.5, 0.7, 0.9, 0.99, 0.999999, 1 - 1e-12])
def test_ellip_ke_vs_scipy(k2):
    sp = pytest.importorskip("scipy.special")
    K, E = oracle.ellip_ke(k2, 1.0 - k2)
    assert abs(K / sp.ellipk(k2) - 1) < 2e-15
    assert abs(E / sp.ellipe(k2) - 1) < 1e-14


def test_ellip_special_values():
    # K(0) = E(0) = pi/2; lemniscatic case k^2 = 1/2 (DLMF 19.6 / 19.20): K = Gamma(1/4)^2/(4 sqrt(pi))
    K, E = oracle.ellip_ke(0.0, 1.0)
    assert abs(K - math.pi / 2) < 1e-15 and abs(E - math.pi / 2) < 1e-15
    g = math.gamma(0.25)
    K, E = oracle.ellip_ke(0.5, 0.5)
    assert abs(K - g * g / (4 * math.sqrt(math.pi))) < 2e-15
    assert abs(E - (g * g / (8 * math.sqrt(math.pi)) + math.pi ** 1.5 / (g * g))) < 2e-15
    # Carlson: R_F(x,x,x) = x^-1/2, R_D(x,x,x) = x^-3/2
    assert abs(oracle.carlson_rf(2.5, 2.5, 2.5) - 2.5 ** -0.5) < 1e-15
    assert abs(oracle.carlson_rd(2.5, 2.5, 2.5) - 2.5 ** -1.5) < 1e-15


@pytest.mark.parametrize("k2", [0.05, 0.25, 0.5, 0.8, 0.97])
def test_legendre_relation(k2):
    # E K' + E' K - K K' = pi/2 (Legendre's relation)
    K, E = oracle.ellip_ke(k2, 1 - k2)
    Kp, Ep = oracle.ellip_ke(1 - k2, k2)
    assert abs(E * Kp + Ep * K - K * Kp - math.pi / 2) < 4e-15


def test_K_logarithmic_limit():
    # K(k) - ln(4/k') -> 0 like k'^2 ln(1/k') as k' -> 0 (DLMF 19.12.1)
    for kp2 in [1e-6, 1e-10, 1e-14]:
        K, _ = oracle.ellip_ke(1 - kp2, kp2)
        kp = math.sqrt(kp2)
        assert abs(K - math.log(4 / kp)) < 2 * kp2 * math.log(1 / kp) + 1e-14


# --- Q_{n-1/2}(chi) (Eqs. gfunc:recursion, gfunc:Q0) ---------------------------------------

T_GRID = [1e-14, 1e-10, 1e-6, 1e-4, 1e-3, 8e-3, 0.03, 0.1, 0.5, 1.0, 3.0, 30.0, 1e3, 1e5]


@pytest.mark.parametrize("N", [1, 2, 16, 32, 64])
def test_Q_vs_mpmath(N):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    worst = 0.0
    for t in T_GRID:
        Q, _ = oracle.legendre_q(t, N)
        for n in range(N + 1):
            ref = mp.re(mp.legenq(n - mp.mpf(1) / 2, 0, 1 + mp.mpf(t), type=3))
            if abs(ref) < 1e-290:
                continue  # underflows in FP64: contributes nothing
            worst = max(worst, abs(float((Q[n] - ref) / ref)))
    assert worst < 2e-13, worst


def test_Q_start_values_closed_forms():
    # Q_{-1/2} = mu K(mu), Q_{1/2} = chi mu K - (1 + chi) mu E, mu^2 = 2/(1+chi), with K, E
    # from scipy (modulus convention: scipy takes m = mu^2)
    sp = pytest.importorskip("scipy.special")
    for t in [1e-6, 1e-3, 0.05, 0.5, 2.0]:
        chi = 1 + t
        m = 2 / (1 + chi)
        mu = math.sqrt(m)
        # ellipkm1 takes the complementary parameter 1 - m = t / (2 + t) without cancellation
        K, E = sp.ellipkm1(t / (2 + t)), sp.ellipe(m)
        Q, _ = oracle.legendre_q(t, 1)
        assert abs(Q[0] / (mu * K) - 1) < 1e-14
        ref1 = chi * mu * K - (1 + chi) * mu * E
        assert abs(Q[1] / ref1 - 1) < 1e-12 * max(1.0, chi * chi)


def test_Q_large_chi_leading_term():
    # Q_{n-1/2}(chi) ~ sqrt(pi) Gamma(n+1/2) / (n! (2 chi)^{n+1/2}) as chi -> infinity
    t = 1e7
    Q, used_miller = oracle.legendre_q(t, 8)
    assert used_miller
    chi = 1 + t
    for n in range(9):
        lead = math.sqrt(math.pi) * math.gamma(n + 0.5) / (math.factorial(n) * (2 * chi) ** (n + 0.5))
        assert abs(Q[n] / lead - 1) < 1e-12


@pytest.mark.parametrize("t", [1e-8, 1e-3, 0.2, 5.0])
def test_Q_recursion_residual(t):
    # (2n-1) Q_n = 4(n-1) chi Q_{n-1} - (2n-3) Q_{n-2}, Eq. gfunc:recursion (with Q_n = Q_{n-1/2})
    N = 40
    Q, _ = oracle.legendre_q(t, N)
    chi = 1 + t
    for n in range(2, N + 1):
        lhs = (2 * n - 1) * Q[n]
        rhs = 4 * (n - 1) * chi * Q[n - 1] - (2 * n - 3) * Q[n - 2]
        assert abs(lhs - rhs) <= 1e-12 * (abs(4 * (n - 1) * chi * Q[n - 1]) + abs(lhs))


def test_paper_rule_constants_and_error():
    # The paper's literal switch (chi = 1.008) and Miller start (N + 80) lose digits near the
    # switch; the default rule does not.  Documents the reading of Appendix A.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    chi_sw = GOLD["legendre_forward_switch_chi"]["value"]
    t = chi_sw - 1.0
    N = 32
    Qp, mp_used = oracle.legendre_q(t, N, rule=oracle.RULE_PAPER)
    Qs, _ = oracle.legendre_q(t, N, rule=oracle.RULE_SAFE)
    assert mp_used  # chi >= 1.008 -> backward recursion under the paper's rule
    ref = [mp.re(mp.legenq(n - mp.mpf(1) / 2, 0, 1 + mp.mpf(t), type=3)) for n in range(N + 1)]
    ep = max(abs(float((Qp[n] - ref[n]) / ref[n])) for n in range(N + 1))
    es = max(abs(float((Qs[n] - ref[n]) / ref[n])) for n in range(N + 1))
    assert 1e-11 < ep < 1e-7
    assert es < 1e-13


# --- modal Green's function (Eqs. analysis:gfunc, gfunc:def) --------------------------------

def _quad_green(r, r1, x, n, m):
    th = 2 * np.pi * np.arange(m) / m
    R = np.sqrt(r * r + r1 * r1 - 2 * r * r1 * np.cos(th) + x * x)
    return np.sum(np.cos(n * th) / (4 * np.pi * R)) * (2 * np.pi / m)


@pytest.mark.parametrize("geom", [(1.0, 0.7, 0.3), (0.5, 0.5, 0.2), (2.0, 0.1, -1.5), (0.3, 1.2, 0.0),
                                  (1.0, 0.95, 0.05)])
def test_green_vs_quadrature(geom):
    # trapezoid rule on the periodic analytic integrand converges exponentially
    r, r1, x = geom
    N = 12
    G = oracle.green(r, r1, x, N)
    for n in range(N + 1):
        ref = _quad_green(r, r1, x, n, 20000)
        assert abs(G[n] - ref) <= 1e-13 * abs(_quad_green(r, r1, x, 0, 20000))


def test_green_n0_is_ring_potential():
    # n = 0: the classical ring potential K(k) / (pi rho_+), k^2 = 4 r r1 / rho_+^2
    sp = pytest.importorskip("scipy.special")
    for r, r1, x in [(1.0, 0.4, 0.7), (0.2, 0.25, 0.01), (3.0, 0.05, 2.0)]:
        rp2 = (r + r1) ** 2 + x * x
        ref = sp.ellipk(4 * r * r1 / rp2) / (math.pi * math.sqrt(rp2))
        assert abs(oracle.green(r, r1, x, 0)[0] / ref - 1) < 1e-14


def test_green_symmetry_parity_homogeneity():
    N = 20
    r, r1, x = 0.8, 0.35, 0.6
    G = oracle.green(r, r1, x, N)
    np.testing.assert_allclose(oracle.green(r1, r, x, N), G, rtol=1e-14, atol=0)
    np.testing.assert_allclose(oracle.green(r, r1, -x, N), G, rtol=1e-14, atol=0)
    for s in [0.01, 3.7, 250.0]:  # Eq. gfunc:scaled: G(s r, s r1, s x) = G / s
        np.testing.assert_allclose(oracle.green(s * r, s * r1, s * x, N) * s, G, rtol=1e-13, atol=0)


def test_green_coincident_is_zero():
    assert np.all(oracle.green(0.5, 0.5, 0.0, 4) == 0.0)


def test_green_gradient_vs_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    N = 6
    for r, r1, x in [(1.1, 0.6, 0.4), (0.3, 0.32, -0.05), (0.2, 1.5, 2.0)]:
        G, Gr, Gx = oracle.green_grad(r, r1, x, N)
        for n in range(N + 1):
            def f(a, b):
                chi = (a * a + r1 * r1 + b * b) / (2 * a * r1)
                return mp.re(mp.legenq(n - mp.mpf(1) / 2, 0, chi, type=3)) / (2 * mp.pi * mp.sqrt(a * r1))
            dr = float(mp.diff(lambda a: f(a, mp.mpf(x)), mp.mpf(r)))
            dx = float(mp.diff(lambda b: f(mp.mpf(r), b), mp.mpf(x)))
            scale = abs(G[0]) / min(r, abs(r - r1) + abs(x))
            assert abs(Gr[n] - dr) < 1e-12 * scale
            assert abs(Gx[n] - dx) < 1e-12 * scale
