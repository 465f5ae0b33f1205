"""GPU parity of the per-pair modal Green's function and of its Taylor coefficients
(afmm_green, afmm_green_expansion) against the oracle, through the C ABI."""
import math

import numpy as np
import pytest

import oracle
from tests.gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def _pairs(seed=3):
    rng = np.random.default_rng(seed)
    rows = []
    # near-coincident pairs (chi - 1 from 1e-14 to 1e-3), moderate and far pairs
    for t in [1e-14, 1e-10, 1e-7, 1e-5, 1e-3]:
        for _ in range(8):
            r = rng.uniform(0.05, 2.0)
            d = math.sqrt(2 * t) * r * rng.uniform(0.3, 1.0)
            ang = rng.uniform(0, 2 * math.pi)
            r1 = r + d * math.cos(ang)
            rows.append((r, r1, d * math.sin(ang)))
    for _ in range(120):
        r, r1 = rng.uniform(0.01, 3.0, 2)
        rows.append((r, r1, rng.normal(0, 1.5)))
    rows.append((0.01, 0.012, 6.0))  # very large chi
    rows.append((1.0, 1.0, 0.0))     # coincident: contributes zero
    return np.array(rows)


@pytest.mark.parametrize("N", [0, 1, 2, 16, 32, 64])
def test_green_matches_oracle(N):
    P = _pairs()
    r, r1, x = to_dev(P[:, 0], P[:, 1], P[:, 2])
    from paper_2301_01179_gb300 import binding
    G, Gr, Gx = to_np(*binding.green(r, r1, x, N + 1, grad=True))
    for p, (a, b, c) in enumerate(P):
        g, gr, gx = oracle.green_grad(a, b, c, N)
        scale = abs(g[0]) + 1e-300
        for n in range(N + 1):
            # forward recursion is used while its error growth exp(2 N acosh chi) <= e^9:
            # about 1e-12 relative on the highest modes
            tol = 1e-11 * abs(g[n]) + 1e-15 * scale
            assert abs(G[n, p] - g[n]) <= tol, (p, n, G[n, p], g[n])
            dist = math.hypot(a - b, c) + 1e-300
            gscale = scale / min(a, dist)
            assert abs(Gr[n, p] - gr[n]) <= 1e-11 * abs(gr[n]) + 1e-14 * gscale, (p, n)
            assert abs(Gx[n, p] - gx[n]) <= 1e-11 * abs(gx[n]) + 1e-14 * gscale, (p, n)


def test_green_expansion_matches_oracle():
    from paper_2301_01179_gb300 import binding
    pts = np.array([[1.3, 0.7, 0.45], [2.5, 2.0, 1.5], [0.6, 0.6, 0.5], [0.4, 1.1, -0.3], [10.5, 8.5, 2.0]])
    N, P = 6, 14
    r, r1, x = to_dev(pts[:, 0], pts[:, 1], pts[:, 2])
    E = to_np(binding.green_expansion(r, r1, x, N + 1, P))[0]
    for p, (a, b, c) in enumerate(pts):
        g = oracle.gbar(a, b, c, N, P)
        dist = min(math.hypot(a - b, c), min(a, b))
        i, j, k = np.meshgrid(np.arange(P + 1), np.arange(P + 1), np.arange(P + 1), indexing="ij")
        sc = np.abs(g[:, 0, 0, 0]).max() * dist ** (-(i + j + k)).astype(float)
        err = np.abs(E[p] - g) / sc[None]
        assert err.max() < 1e-11, (p, err.max(), np.unravel_index(err.argmax(), err.shape))


def test_green_expansion_high_modes_axial_neighbours():
    """Modes 0..64 at Taylor order 24 for boxes of side h = 1/64 one to three boxes apart, in
    plain and in box units (as the S2L expansions are generated): there the x-recursion's
    G^(n) - G^(n-1) cancels, and FP64 start values and base columns lose up to ten digits.
    The GPU forms them in double-double.  Checked two ways:
      - the Taylor sum at shifts of up to 0.35 h in all three variables (the offsets an S2L
        application meets) reproduces the oracle's G at the shifted point, 1e-12 of G^(0),
        for every mode;
      - against the oracle (binary128 base columns) for modes 0..32, normwise per mode and
        total order i + j + k: max |E - g| / max |g| over the order's coefficients <= 1e-11.
        (Mixed coefficients of these geometries exceed |G^(0)| dist^-(i+j+k) by up to 2^24,
        so FP64 rounding alone shows at 1e-8 on that scale.)  Above mode 32 the Laplace
        recursion magnifies even binary128 rounding in the highest mixed coefficients
        (about 6e-19 in the base columns at n = 64), which the S2L weights by (h/2)^(i+j+k)."""
    from paper_2301_01179_gb300 import binding
    h = 1.0 / 64
    pts = np.array([[1.05, 1.05, 2 * h], [0.6, 0.6, 3 * h], [1.05, 1.05 + 2 * h, 2 * h], [1.05 + 3 * h, 1.05, h],
                    [1.05 / h, 1.05 / h, 2.0], [0.3 / h + 2.0, 0.3 / h, 2.0]])
    box = [h, h, h, h, 1.0, 1.0]
    N, P = 64, 24
    r, r1, x = to_dev(pts[:, 0], pts[:, 1], pts[:, 2])
    E = to_np(binding.green_expansion(r, r1, x, N + 1, P))[0]
    i, j, k = np.meshgrid(np.arange(P + 1), np.arange(P + 1), np.arange(P + 1), indexing="ij")
    rng = np.random.default_rng(8)
    for p, (a, b, c) in enumerate(pts):
        for _ in range(6):
            d = rng.uniform(-0.35 * box[p], 0.35 * box[p], 3)
            G = oracle.green(a + d[0], b + d[1], c + d[2], N)
            S = np.einsum("nijk,ijk->n", E[p], d[0] ** i * d[1] ** j * d[2] ** k)
            assert np.max(np.abs(S - G)) < 1e-12 * abs(G[0]), (p, np.max(np.abs(S - G)) / abs(G[0]))
        g = oracle.gbar(a, b, c, 32, P)
        o = i + j + k
        for order in range(P + 1):
            sel = o == order
            den = np.abs(g[:, sel]).max(axis=1)
            err = np.abs(E[p][:33][:, sel] - g[:, sel]).max(axis=1) / np.where(den > 0, den, 1.0)
            assert err.max() < 1e-11, (p, order, err.max(), int(err.argmax()))
