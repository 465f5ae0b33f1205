"""Pins for the oracle's Taylor coefficients gbar^(n)_{i,j,k} (Appendix A).

The generator uses the x-recursion, the closed r/r1/mixed forms and the Laplace recursion
(with the x-term the printed formula omits).  It is checked against mpmath numerical
derivatives, Taylor-shift consistency with directly evaluated G, the source-side Laplace
equation (which the field-side recursion never uses), and the symmetries of G.
"""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("geom", [(1.3, 0.7, 0.45), (0.6, 0.6, 0.5), (0.4, 1.1, 0.0)])
def test_gbar_vs_mpmath_derivatives(geom):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    r, r1, x = geom
    N, P = 3, 5
    g = oracle.gbar(r, r1, x, N, P)

    def G(n, a, b, c):
        chi = (a * a + b * b + c * c) / (2 * a * b)
        return mp.re(mp.legenq(n - mp.mpf(1) / 2, 0, chi, type=3)) / (2 * mp.pi * mp.sqrt(a * b))

    scale = abs(g[0, 0, 0, 0])
    for n in range(N + 1):
        for i in range(P + 1):
            for j in range(P + 1 - i):
                for k in range(P + 1 - i - j):
                    if i + j + k > 4 and (i, j) != (0, 0):
                        continue  # keep the mpmath cost down; all index patterns are covered
                    d = mp.diff(lambda a, b, c: G(n, a, b, c), (mp.mpf(r), mp.mpf(r1), mp.mpf(x)), (i, j, k))
                    ref = float(d) / (math.factorial(i) * math.factorial(j) * math.factorial(k))
                    dist = math.hypot(r - r1, x)
                    tol = 2e-13 * scale * dist ** -(i + j + k) * 10 ** (0.5 * (i + j + k) / 4)
                    assert abs(g[n, i, j, k] - ref) <= max(tol, 1e-13 * abs(ref)), (n, i, j, k)


@pytest.mark.parametrize("geom", [(1.0, 0.5, 0.8), (2.0, 1.9, 0.6), (0.3, 0.9, 1.0)])
def test_gbar_taylor_shift(geom):
    # sum_{i+j+k<=P} gbar_{ijk} dr^i dr1^j dx^k reproduces G at the shifted point
    r, r1, x = geom
    N, P = 10, 30
    g = oracle.gbar(r, r1, x, N, P)
    dist = math.hypot(r - r1, x)
    rng = np.random.default_rng(5)
    i, j, k = np.meshgrid(np.arange(P + 1), np.arange(P + 1), np.arange(P + 1), indexing="ij")
    for _ in range(6):
        d = rng.uniform(-0.15 * dist, 0.15 * dist, 3)
        G = oracle.green(r + d[0], r1 + d[1], x + d[2], N)
        S = np.einsum("nijk,ijk->n", g, d[0] ** i * d[1] ** j * d[2] ** k)
        np.testing.assert_allclose(S, G, rtol=1e-12, atol=1e-14 * abs(G[0]))


@pytest.mark.parametrize("geom,frac", [((1.05, 1.05, 2 / 64), 0.35), ((0.6, 0.6, 3 / 64), 0.45),
                                       ((1.05, 1.05 + 2 / 64, 2 / 64), 0.45)])
def test_gbar_taylor_shift_high_modes_axial_neighbours(geom, frac):
    """Modes 0..64 at order 24 for boxes of side h = 1/64 one or two boxes apart along the
    axis (the geometry where G^(n) and G^(n-1) nearly coincide): the Taylor sum at shifts
    of up to frac * h in all three variables must reproduce G at the shifted point.  FP64
    base columns fail this by up to 2e-6 (the cancellation of the x-recursion at high n);
    the binary128 ones pass at 1e-12."""
    r, r1, x = geom
    N, P = 64, 24
    h = 1 / 64
    g = oracle.gbar(r, r1, x, N, P)
    rng = np.random.default_rng(5)
    i, j, k = np.meshgrid(np.arange(P + 1), np.arange(P + 1), np.arange(P + 1), indexing="ij")
    for _ in range(8):
        d = rng.uniform(-frac * h, frac * h, 3)
        G = oracle.green(r + d[0], r1 + d[1], x + d[2], N)
        S = np.einsum("nijk,ijk->n", g, d[0] ** i * d[1] ** j * d[2] ** k)
        assert np.max(np.abs(S - G)) < 1e-12 * abs(G[0])


def test_gbar_source_laplace_on_field_recursed_terms():
    # Coefficients with i >= 2 come from the field-side (r) Laplace recursion.  They must
    # also satisfy the source-side (r1) Laplace equation, written here in its local form:
    # (j+1)(j+2) r1^2 g_{i,j+2,k} + (j+1)(2j+1) r1 g_{i,j+1,k} + (j^2 - n^2) g_{i,j,k}
    #   + (k+1)(k+2) [r1^2 g_{i,j,k+2} + 2 r1 g_{i,j-1,k+2} + g_{i,j-2,k+2}] = 0
    r, r1, x = 1.2, 0.8, 0.5
    N, P = 6, 14
    g = oracle.gbar(r, r1, x, N, P)

    def G(n, i, j, k):
        if i < 0 or j < 0 or k < 0 or i + j + k > P:
            return 0.0
        return g[n, i, j, k]

    worst = 0.0
    for n in range(N + 1):
        for i in range(2, P):
            for j in range(0, P - i - 1):
                for k in range(0, P - i - j - 1):
                    if i + j + 2 + k > P:
                        continue
                    terms = [(j + 1) * (j + 2) * r1 * r1 * G(n, i, j + 2, k),
                             (j + 1) * (2 * j + 1) * r1 * G(n, i, j + 1, k),
                             (j * j - n * n) * G(n, i, j, k),
                             (k + 1) * (k + 2) * (r1 * r1 * G(n, i, j, k + 2) + 2 * r1 * G(n, i, j - 1, k + 2)
                                                  + G(n, i, j - 2, k + 2))]
                    res = abs(sum(terms)) / max(sum(abs(t) for t in terms), 1e-300)
                    worst = max(worst, res)
    assert worst < 1e-11, worst


def _natural_scale(g, r, r1, x, P):
    """|gbar_000| * dist^-(i+j+k): the size a coefficient of that order has before any
    cancellation; rounding errors of the recursions are relative to it."""
    dist = min(math.hypot(r - r1, x), min(r, r1))
    i, j, k = np.meshgrid(np.arange(P + 1), np.arange(P + 1), np.arange(P + 1), indexing="ij")
    return np.abs(g[:, :1, :1, :1]).max() * dist ** (-(i + j + k))[None].astype(float)


def test_gbar_symmetries():
    N, P = 5, 12
    r, r1, x = 0.9, 0.4, 0.7
    g = oracle.gbar(r, r1, x, N, P)
    sc = _natural_scale(g, r, r1, x, P)
    # r <-> r1 symmetry of G: gbar_{ijk}(r, r1, x) = gbar_{jik}(r1, r, x)
    gs = oracle.gbar(r1, r, x, N, P)
    assert np.all(np.abs(g - np.transpose(gs, (0, 2, 1, 3))) <= 1e-13 * sc)
    # parity in x: gbar_{ijk}(r, r1, -x) = (-1)^k gbar_{ijk}(r, r1, x)
    gm = oracle.gbar(r, r1, -x, N, P)
    sign = (-1.0) ** np.arange(P + 1)
    assert np.all(np.abs(gm - g * sign[None, None, None, :]) <= 1e-13 * sc)
    # homogeneity (Eq. gfunc:scaled): gbar_{ijk}(s .) = s^{-1-i-j-k} gbar_{ijk}(.)
    s_ = 2.5
    gh = oracle.gbar(s_ * r, s_ * r1, s_ * x, N, P)
    i, j, k = np.meshgrid(np.arange(P + 1), np.arange(P + 1), np.arange(P + 1), indexing="ij")
    fac = (s_ ** (-1.0 - i - j - k))[None]
    assert np.all(np.abs(gh - g * fac) <= 1e-13 * sc * fac)


def test_gbar_zero_mode_uses_G_minus_one_equals_G_one():
    # the n = 0 x-derivative needs G^(-1) = G^(1); check gbar^(0)_{0,0,1} against dG/dx
    r, r1, x = 1.0, 0.6, 0.3
    g = oracle.gbar(r, r1, x, 0, 3)
    _, _, Gx = oracle.green_grad(r, r1, x, 0)
    assert abs(g[0, 0, 0, 1] - Gx[0]) < 1e-14 * abs(Gx[0])
