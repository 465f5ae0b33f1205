"""GPU parity at the benchmark's own shapes against the oracle FMM on the same tree.

- The headline tile: 2e4 points with the 1e6-point benchmark's laws (r ~ U[0.05, 2],
  z ~ U[-2, 2]), modes 0..32, order 12, leaf 64.  The FP64 path runs its tensor-core S2L
  with the 96-wide tile (91 coefficients) there.  Potential, field gradient and adjoint
  against oracle.fmm / oracle.adjoint_fmm, 1e-10 per mode (Eq. results:error).
- Full 64-box tensor-core units: depth 7 on the same laws (128 boxes per column).
- Full size, in bench.py's launch configuration: the 1e6 x 1e6 benchmark workload and the
  1e6 near-singular curve workload against the sampled oracle FMM at sampled field points
  (1e-10 per mode), the GPU direct sum there against the oracle's direct sum; the
  2.56e5 adjoint workload (order 10) at sampled sources.
- Order 14 with 65 modes on the 4e6-ring workload's laws (r ~ Exp(mean 0.5) on [0.01, 3],
  z ~ N(0, 1), |S^(n)| ~ n^-2), 1.2e4 points: the FP64 path at 1e-10, MIXED within its
  stated bound of the oracle FMM.
- Tree structure (Sec. 2.2): the plan's near and S2L counts equal the oracle's counts
  from the list definitions, and every (field point, source) pair is covered once.
"""
import numpy as np
import pytest

import oracle
from paper_2301_01179_gb300 import workloads as W
from tests.gpu_util import eps_modes, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-10
MIXED_TOL = 2e-5


def _plan(w, order, leaf, depth=0, precision="fp64"):
    from paper_2301_01179_gb300 import binding
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    return binding.Plan(sr, sz, tr, tz, w["n_modes"], order=order, leaf_size=leaf, depth=depth,
                        precision=precision)


def _geom(w, info):
    d, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=info["depth"])
    # same square on both sides (min and max are exact, so is the side)
    assert (geom[0], geom[1], geom[2]) == (info["r0"], info["z0"], info["side"])
    return d, geom


@pytest.fixture(scope="module")
def head():
    return W.make("cfg2", ns=20000, nf=20000, with_targets=True)


def test_headline_tile_potential_and_gradient(head):
    w = head
    pl = _plan(w, 12, 64)
    info = pl.info()
    assert info["s2l_tensor_cores"] and info["n_modes"] == 33 and info["depth"] == 5
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.grad(q_re, q_im))
    pl.close()
    d, geom = _geom(w, info)
    F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], 12, d, geom, grad=True)
    for c in range(0, 6, 2):
        e = eps_modes(g[c], g[c + 1], F[c], F[c + 1])
        assert e.max() < TOL, (c, e.max(), int(e.argmax()))


def test_headline_tile_adjoint(head):
    w = head
    pl = _plan(w, 12, 64)
    info = pl.info()
    assert info["s2l_tensor_cores"]
    q_re, q_im, T_re, T_im = to_dev(w["q_re"], w["q_im"], w["T_re"], w["T_im"])
    g = to_np(*pl.adjoint(q_re, q_im, T_re, T_im))
    pl.close()
    d, geom = _geom(w, info)
    A = oracle.adjoint_fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], w["T_re"],
                           w["T_im"], 12, d, geom)
    assert eps_modes(g[0], g[1], A[0], A[1]).max() < TOL
    for c in (2, 3):
        np.testing.assert_allclose(g[c], A[c], rtol=0, atol=TOL * np.abs(A[c]).max())


def test_full_tensor_core_units_at_depth_7():
    """At depth 7 a column holds 128 boxes, so the tensor-core S2L runs full units of 64
    boxes (128 rows of the MMA tile); checked at sampled field points."""
    w = W.make("cfg2", ns=20000, nf=20000, n_modes=9)
    pl = _plan(w, 12, 64, depth=7)
    info = pl.info()
    # the points fill r in [0.05, 2] of the side-4 square: half of the 128 columns
    assert info["s2l_tensor_cores"] and info["n_boxes"][7] > 0.85 * 4 ** 7 / 2
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.grad(q_re, q_im))
    pl.close()
    d, geom = _geom(w, info)
    idx = W.subset(20000, 64, seed=17)
    S = oracle.fmm_sampled(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], 12, d, geom, idx,
                           grad=True)
    for c in range(0, 6, 2):
        assert eps_modes(g[c][:, idx], g[c + 1][:, idx], S[c], S[c + 1]).max() < TOL, c


@pytest.mark.parametrize("kind", ["cfg2", "cfg3"])
def test_full_size_fmm_vs_sampled_oracle_fmm(kind):
    """The 1e6 x 1e6 workloads (order 12, leaf 64; depth 8 for the uniform box, 9 for the
    curve) as bench.py runs them: FMM potential and gradient at 12 sampled field points
    against the oracle's FMM on the same tree, and the GPU direct sum at 6 of them
    against the oracle's direct sum."""
    from paper_2301_01179_gb300 import binding
    w = W.make(kind)
    sr, sz, tr, tz, qr, qi = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    pl = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=w["order"], leaf_size=w["leaf"])
    info = pl.info()
    assert info["depth"] == (8 if kind == "cfg2" else 9) and info["s2l_tensor_cores"]
    idx = W.subset(w["tgt_r"].size, 12, seed=21)
    ii = to_dev(idx.astype(np.float64))[0].long()
    out = [o[:, ii].cpu().numpy() for o in pl.grad(qr, qi)]
    pl.close()
    d, geom = _geom(w, info)
    S = oracle.fmm_sampled(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], w["order"], d, geom,
                           idx, grad=True)
    for c in range(0, 6, 2):
        e = eps_modes(out[c], out[c + 1], S[c], S[c + 1])
        assert e.max() < TOL, (c, e.max())
    jdx = idx[::2]
    pd = binding.Plan(sr, sz, *to_dev(w["tgt_r"][jdx], w["tgt_z"][jdx]), w["n_modes"], order=4, leaf_size=64)
    g = to_np(*pd.direct_grad(qr, qi))
    pd.close()
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"][jdx], w["tgt_z"][jdx], w["q_re"], w["q_im"], grad=True)
    for c in range(0, 6, 2):
        assert eps_modes(g[c], g[c + 1], D[c], D[c + 1]).max() < TOL, c


def test_full_size_adjoint_vs_sampled_oracle():
    """The 2.56e5 x 2.56e5 adjoint workload (modes 0..24, order 10, leaf 64): dL/dS,
    dL/dr' and dL/dz' at 16 sampled sources against the oracle's transposed FMM."""
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg4", with_targets=True)
    sr, sz, tr, tz, qr, qi, Tr, Ti = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"],
                                            w["T_re"], w["T_im"])
    pl = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=w["order"], leaf_size=w["leaf"])
    info = pl.info()
    g = pl.adjoint(qr, qi, Tr, Ti)
    idx = W.subset(w["src_r"].size, 16, seed=5)
    ii = to_dev(idx.astype(np.float64))[0].long()
    g = [g[0][:, ii].cpu().numpy(), g[1][:, ii].cpu().numpy(), g[2][ii].cpu().numpy(), g[3][ii].cpu().numpy()]
    pl.close()
    d, geom = _geom(w, info)
    A = oracle.adjoint_fmm_sampled(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], w["T_re"],
                                   w["T_im"], w["order"], d, geom, idx)
    assert eps_modes(g[0], g[1], A[0], A[1]).max() < TOL
    for c in (2, 3):
        np.testing.assert_allclose(g[c], A[c], rtol=0, atol=TOL * np.abs(A[c]).max())


def test_order14_65_modes_large_workload_laws():
    """Order 14 and 65 modes (the 4e6-ring workload's) on 1.2e4 points of its laws: the FP64
    path (CUDA-core S2L beyond order 12) at the parity bar, MIXED (tensor-core S2L with
    4-digit slicing) within its stated bound, both against the oracle FMM."""
    w = W.make("cfg5", ns=12000, nf=12000)
    assert w["n_modes"] == 65 and w["order"] == 14
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    F = None
    for prec, tol, tc in (("fp64", TOL, False), ("mixed", MIXED_TOL, True)):
        pl = _plan(w, 14, 64, precision=prec)
        info = pl.info()
        assert info["s2l_tensor_cores"] == tc
        g = to_np(*pl.grad(q_re, q_im))
        pl.close()
        if F is None:
            d, geom = _geom(w, info)
            F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], 14, d, geom,
                           grad=True)
        for c in range(0, 6, 2):
            e = eps_modes(g[c], g[c + 1], F[c], F[c + 1])
            assert e.max() < tol, (prec, c, e.max())


@pytest.mark.parametrize("kind,ns,nf", [("cfg1", None, None), ("paper", None, None), ("cfg2", None, None),
                                        ("cfg3", None, None), ("cfg5", None, None), ("cfg5", 5000, 300)])
def test_tree_counts_match_oracle_lists(kind, ns, nf):
    """Near pairs, S2L box pairs and the point pairs under them, counted by the GPU tree
    build, equal the oracle's counts from the list definitions (exact integers), and the
    near field plus the interaction lists cover all ns * nf pairs once."""
    from paper_2301_01179_gb300 import binding
    w = W.make(kind, ns=ns, nf=nf, n_modes=1)
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    pl = binding.Plan(sr, sz, tr, tz, 1, order=4, leaf_size=w["leaf"])
    info = pl.info()
    pl.close()
    d, geom = _geom(w, info)
    rule_d, _ = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["leaf"])
    assert d == rule_d
    near, box_pairs, far = oracle.tree_counts(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], d, geom)
    assert (info["near_pairs"], info["s2l_pairs"], info["s2l_point_pairs"]) == (near, box_pairs, far)
    assert info["near_pairs"] + info["s2l_point_pairs"] == w["src_r"].size * w["tgt_r"].size
