"""GPU parity of the mixed-precision path (AFMM_MIXED) against the FP64 oracle.

MIXED keeps the Legendre recursion, the elliptic (AGM) start values and the pair geometry
in FP64, and does the bulk accumulation in Kahan-compensated FP32 and the far field
(moments, shifts, S2L) in FP32 on box-scaled coordinates.  Its stated error, per mode
(Eq. results:error): near field and direct sums <= 2e-6, FMM <= 2e-5 on top of the FP64
FMM's own truncation error (both measured on these workloads on GB300)."""
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
