"""GPU parity of the mixed-precision path (AFMM_MIXED) against the FP64 oracle.

MIXED forms the pair geometry (r - r1, r + r1, z - z1) as FP32 pairs, by error-free FP32 sums
of exact FP32 triples of the coordinates (about 2^-47 of each difference, no FP64 arithmetic
per pair); the elliptic (AGM) start values and the Legendre recursion run in FP32-pair
arithmetic (48-bit significands, FP32 exponent range with exact power-of-two rescaling),
not in IEEE FP64; the products with the strengths are FP32 with Kahan-compensated FP32
sums, and the far field (moments, shifts, S2L) is FP32 on box-scaled coordinates.  Its
stated error, per mode (Eq. results:error): near field and direct sums <= 2e-6, FMM <= 2e-5
on top of the FP64 FMM's own truncation error (both measured on these workloads on GB300).
The FP32-pair sequence itself is checked against the native FP64 sequence pair by pair on
near-singular and far pairs (test_fp32_pair_sequence_vs_native_fp64)."""
import numpy as np
import pytest

import oracle
from paper_2301_01179_gb300 import workloads as W
from tests.gpu_util import eps_modes, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL_DIRECT = 2e-6
TOL_FMM = 2e-5


def _plan(w, **kw):
    from paper_2301_01179_gb300 import binding
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    return binding.Plan(sr, sz, tr, tz, w["n_modes"], precision="mixed", **kw)


def test_mixed_direct_matches_oracle():
    w = W.make("cfg3", ns=3000, nf=1500)
    pl = _plan(w, order=8, leaf_size=32)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.direct_grad(q_re, q_im))
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], grad=True)
    for c in range(0, 6, 2):
        e = eps_modes(g[c], g[c + 1], D[c], D[c + 1])
        print("mixed direct comp %d eps max %.3e" % (c, e.max()))
        assert e.max() < TOL_DIRECT, (c, e.max())


def test_mixed_fmm_matches_oracle_fmm():
    w = W.make("cfg1")
    pl = _plan(w, order=w["order"], leaf_size=w["leaf"])
    d = pl.info()["depth"]
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.grad(q_re, q_im))
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=d)
    F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], w["order"], d, geom,
                   grad=True)
    for c in range(0, 6, 2):
        e = eps_modes(g[c], g[c + 1], F[c], F[c + 1])
        print("mixed fmm comp %d eps max %.3e per mode %s" % (c, e.max(), np.array2string(e, precision=1)))
        assert e.max() < TOL_FMM, (c, e.max())


def test_mixed_adjoint_matches_oracle():
    w = W.make("cfg4", ns=1200, nf=1000, n_modes=9, with_targets=True)
    pl = _plan(w, order=10, leaf_size=32)
    d = pl.info()["depth"]
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=d)
    q_re, q_im, T_re, T_im = to_dev(w["q_re"], w["q_im"], w["T_re"], w["T_im"])
    g = to_np(*pl.adjoint(q_re, q_im, T_re, T_im))
    A = oracle.adjoint_fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], w["T_re"], w["T_im"],
                           10, d, geom)
    assert eps_modes(g[0], g[1], A[0], A[1]).max() < TOL_FMM
    assert np.max(np.abs(g[2] - A[2])) / np.max(np.abs(A[2])) < TOL_FMM
    assert np.max(np.abs(g[3] - A[3])) / np.max(np.abs(A[3])) < TOL_FMM


def test_fp32_pair_sequence_vs_native_fp64():
    """The Legendre sequence of the FP32-pair kernels (shared by MIXED and the FP64 path)
    against native FP64 (afmm_green) pair by pair: one ring source on the near-singular
    curve workload's profile and field points at distances 1e-9 .. 3 from it (chi - 1 from
    ~1e-18, the logarithmic near-singularity, to the Miller regime).  With unit strengths
    the direct sum of one source is the sequence G^(n) itself.  Per mode, the error of every
    pair relative to its G^(0) (the scale of the max-normalised per-mode error):
      - FP64 path (FP32-pair sequence, pair products): <= 1e-11;
      - MIXED (the same sequence, FP32 products): <= 2e-6, the FP32 rounding of the product."""
    import torch
    from paper_2301_01179_gb300 import binding
    rng = np.random.default_rng(31)
    r1, z1 = 0.5 + 0.2 * np.cos(1.1), 0.3 * np.sin(1.1)
    dist = 10.0 ** rng.uniform(-9.0, 0.5, 3000)
    ang = rng.uniform(0.0, 2.0 * np.pi, 3000)
    tr = r1 + dist * np.cos(ang)
    tz = z1 + dist * np.sin(ang)
    keep = tr > 1e-3
    tr, tz = tr[keep], tz[keep]
    nm = 65
    sr, sz, dtr, dtz = to_dev(np.array([r1]), np.array([z1]), tr, tz)
    q_re, q_im = to_dev(np.ones((nm, 1)), np.zeros((nm, 1)))
    G = binding.green(dtr, torch.full_like(dtr, r1), dtz - z1, nm).cpu().numpy()
    ref0 = np.abs(G[0])
    worst = {}
    for prec, tol in (("fp64", 1e-11), ("mixed", 2e-6)):
        pl = binding.Plan(sr, sz, dtr, dtz, nm, order=4, leaf_size=64, precision=prec)
        g = to_np(*pl.direct(q_re, q_im))
        pl.close()
        err = np.abs(g[0] - G) / ref0[None, :]
        worst[prec] = err.max(axis=1)
        print(prec, "per-mode max error / G0:", np.array2string(worst[prec], precision=1))
        assert err.max() < tol, (prec, err.max(), np.unravel_index(err.argmax(), err.shape))
        assert np.abs(g[1]).max() == 0.0


def test_mixed_fmm_deep_tree_65_modes():
    """MIXED against the FP64 path (itself oracle-pinned at 1e-10) on the deep tree of the
    4e6-ring workload: its laws (r ~ Exp(mean 0.5) on [0.01, 3], z ~ N(0, 1), |S^(n)| ~
    n^-2), modes 0..64, order 14, depth 10 as the full workload's leaf rule gives, on 1e5
    points.  The Taylor coefficients of the smallest boxes at the highest modes are where
    the base columns cancel most (Eq. analysis:taylor's x-recursion as chi -> 1); the bound
    is MIXED's stated FMM bound, 2e-5 per mode."""
    w = W.make("cfg5", ns=100000, nf=100000)
    assert w["n_modes"] == 65 and w["order"] == 14
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    out = {}
    for prec in ("fp64", "mixed"):
        from paper_2301_01179_gb300 import binding
        sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
        pl = binding.Plan(sr, sz, tr, tz, 65, order=14, leaf_size=64, depth=10, precision=prec)
        assert pl.info()["depth"] == 10
        out[prec] = to_np(*pl.grad(q_re, q_im))
        pl.close()
    for c in range(0, 6, 2):
        e = eps_modes(out["mixed"][c], out["mixed"][c + 1], out["fp64"][c], out["fp64"][c + 1])
        print("component", c // 2, "per-mode eps, modes 56..64:", np.array2string(e[56:], precision=1))
        assert e.max() < TOL_FMM, (c, e.max(), int(e.argmax()))
