"""GPU parity of the FMM (afmm_eval, afmm_grad) and of the adjoints (afmm_adjoint,
afmm_adjoint_direct) against the oracle through the C ABI.

The GPU FMM and the oracle FMM follow the same algorithm on the same tree (same depth,
same square), so they must agree to rounding: bar 1e-10 per mode (Eq. results:error).
Against the direct sum the FMM carries its truncation error, which must fall with M."""
import numpy as np
import pytest

import oracle
from paper_2301_01179_gb300 import workloads as W
from tests.gpu_util import eps_modes, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _plan(w, order=None, leaf=None, depth=0):
    from paper_2301_01179_gb300 import binding
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    return binding.Plan(sr, sz, tr, tz, w["n_modes"], order=order or w["order"], leaf_size=leaf or w["leaf"],
                        depth=depth)


def _oracle_fmm(w, M, d, grad=False):
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=d)
    return oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], M, d, geom, grad=grad)


def test_fmm_cfg1_matches_oracle_fmm():
    w = W.make("cfg1")
    pl = _plan(w)
    d = pl.info()["depth"]
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.eval(q_re, q_im))
    F = _oracle_fmm(w, w["order"], d)
    e = eps_modes(g[0], g[1], F[0], F[1])
    assert e.max() < TOL, e


@pytest.mark.parametrize("kind,ns,nf,M,d", [("cfg1", 3000, 2500, 6, 5), ("cfg3", 4000, 3000, 5, 5),
                                             ("cfg5", 3000, 1000, 4, 4), ("paper", 1024, 700, 10, 3)])
def test_fmm_other_shapes_match_oracle_fmm(kind, ns, nf, M, d):
    w = W.make(kind, ns=ns, nf=nf, n_modes=9)
    pl = _plan(w, order=M, depth=d)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.eval(q_re, q_im))
    F = _oracle_fmm(w, M, d)
    assert eps_modes(g[0], g[1], F[0], F[1]).max() < TOL


def test_fmm_converges_to_direct():
    w = W.make("cfg1", ns=3000, nf=3000)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    errs = []
    D = None
    for M in (4, 8, 12):
        pl = _plan(w, order=M)
        if D is None:
            D = to_np(*pl.direct(q_re, q_im))
        g = to_np(*pl.eval(q_re, q_im))
        errs.append(eps_modes(g[0], g[1], D[0], D[1]).max())
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10, errs


def test_fmm_grad_matches_oracle_fmm():
    w = W.make("cfg1", ns=1500, nf=1000)
    pl = _plan(w)
    d = pl.info()["depth"]
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.grad(q_re, q_im))
    F = _oracle_fmm(w, w["order"], d, grad=True)
    for c in range(0, 6, 2):
        assert eps_modes(g[c], g[c + 1], F[c], F[c + 1]).max() < TOL, c


def test_adjoint_direct_matches_oracle():
    w = W.make("cfg4", ns=900, nf=700, n_modes=9, with_targets=True)
    pl = _plan(w)
    q_re, q_im, T_re, T_im = to_dev(w["q_re"], w["q_im"], w["T_re"], w["T_im"])
    g = to_np(*pl.adjoint_direct(q_re, q_im, T_re, T_im))
    A = oracle.adjoint_direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], w["T_re"],
                              w["T_im"])
    assert eps_modes(g[0], g[1], A[0], A[1]).max() < TOL
    np.testing.assert_allclose(g[2], A[2], rtol=0, atol=TOL * np.abs(A[2]).max())
    np.testing.assert_allclose(g[3], A[3], rtol=0, atol=TOL * np.abs(A[3]).max())


def test_adjoint_fmm_matches_oracle():
    w = W.make("cfg4", ns=1200, nf=1000, n_modes=5, with_targets=True)
    pl = _plan(w, order=10, leaf=32)
    d = pl.info()["depth"]
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=d)
    q_re, q_im, T_re, T_im = to_dev(w["q_re"], w["q_im"], w["T_re"], w["T_im"])
    g = to_np(*pl.adjoint(q_re, q_im, T_re, T_im))
    A = oracle.adjoint_fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], w["T_re"], w["T_im"],
                           10, d, geom)
    assert eps_modes(g[0], g[1], A[0], A[1]).max() < TOL
    np.testing.assert_allclose(g[2], A[2], rtol=0, atol=TOL * np.abs(A[2]).max())
    np.testing.assert_allclose(g[3], A[3], rtol=0, atol=TOL * np.abs(A[3]).max())


def test_fmm_is_deterministic():
    w = W.make("cfg1")
    pl = _plan(w)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    a = to_np(*pl.eval(q_re, q_im))
    b = to_np(*pl.eval(q_re, q_im))
    np.testing.assert_array_equal(a[0], b[0])


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp64_native"])
def test_phase_timing_every_precision(precision):
    """Phase timing (CUDA events around each phase) in every precision, twice in a row, with
    and without the gradient: the FP64-native kernels fold the local expansions into the
    near-field kernel, so their L2P phase is empty and must not leave an error behind."""
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg1", ns=1500, nf=1200, n_modes=5)
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    pl = binding.Plan(sr, sz, tr, tz, 5, order=6, leaf_size=32, precision=precision)
    pl.set_timing(True)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    for f in (pl.eval, pl.grad, pl.eval):
        f(q_re, q_im)
        t = pl.timing()
        assert all(v >= 0.0 for v in t.values()), t
        assert t["near"] > 0.0 and t["total"] >= t["near"], t
    if precision == "fp64_native":  # two events back to back: microseconds apart
        assert t["l2p"] < 0.1 * t["near"], t
    pl.close()
