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
