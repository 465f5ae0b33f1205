"""The FP64 path's S2L on the tensor cores (exact bf16 digit slicing, tcgen05) against the
same path on CUDA cores (FP32-pair arithmetic) and against the oracle's FMM.

Both engines evaluate the same operator (Eq. analysis:s2l) on the same tree, so they agree
to the rounding of the FP64 path; every padded width of the tensor-core kernel (KP = 16 ..
96, orders 1 .. 12) is exercised, with potential and gradient, plus the transposed
(adjoint) direction.  Order 13 exceeds the kernel's tensor memory and must fall back to the
CUDA-core engine with the same results."""
import numpy as np
import pytest

import oracle
from paper_2301_01179_gb300 import workloads as W
from tests.gpu_util import eps_modes, to_dev, to_np

pytestmark = pytest.mark.gpu


def _pair(w, M, depth, grad):
    from paper_2301_01179_gb300 import binding
    sr, sz, tr, tz, qr, qi = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    out = []
    for eng in ("auto", "cuda_cores"):
        pl = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=M, depth=depth, s2l_engine=eng)
        out.append(to_np(*(pl.grad(qr, qi) if grad else pl.eval(qr, qi))))
        pl.close()
    return out


@pytest.mark.parametrize("M", [1, 2, 4, 6, 8, 10, 12, 13])
def test_tensor_core_s2l_matches_cuda_core_s2l(M):
    w = W.make("cfg1", ns=6000, nf=5000, n_modes=7)
    tc, cc = _pair(w, M, 5, grad=True)
    for c in range(0, 6, 2):
        e = eps_modes(tc[c], tc[c + 1], cc[c], cc[c + 1])
        assert e.max() < 1e-11, (M, c, e.max())


def test_tensor_core_s2l_deep_tree_many_modes():
    # ragged units (column groups of 1..64 boxes), 33 modes, order 12 as in the benchmark
    w = W.make("cfg2", ns=40000, nf=30000, n_modes=33)
    tc, cc = _pair(w, 12, 7, grad=False)
    e = eps_modes(tc[0], tc[1], cc[0], cc[1])
    assert e.max() < 1e-11, e.max()


@pytest.mark.parametrize("M", [13, 14, 15])
def test_high_orders_match_oracle_fmm(M):
    """Orders above the FP64 tensor-core width run the S2L on CUDA cores; 15 is the highest
    order the plans accept."""
    w = W.make("cfg3", ns=3000, nf=2500, n_modes=5)
    from paper_2301_01179_gb300 import binding
    sr, sz, tr, tz, qr, qi = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    pl = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=M, depth=4)
    g = to_np(*pl.eval(qr, qi))
    pl.close()
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=4)
    F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], M, 4, geom)
    assert eps_modes(g[0], g[1], F[0], F[1]).max() < 1e-10


def test_tensor_core_s2l_adjoint_direction():
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg4", ns=5000, nf=4000, n_modes=9, with_targets=True)
    sr, sz, tr, tz, qr, qi = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    gr, gi = to_dev(w["T_re"], w["T_im"])
    res = []
    for eng in ("auto", "cuda_cores"):
        pl = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=10, depth=5, s2l_engine=eng)
        res.append(to_np(*pl.adjoint(qr, qi, gr, gi)))
        pl.close()
    for a, b in zip(res[0], res[1]):
        assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(b)), np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("M", [12, 13, 14])
def test_mixed_tensor_core_s2l_wide_tiles(M):
    """MIXED: the tensor-core S2L runs 4 digit slices, so its tiles reach 112 (order 13) and
    128 columns (order 14; the 128-wide tile keeps the expansion cube in FP32).  Against the
    MIXED CUDA-core engine and against the oracle's FP64 FMM, at the MIXED FMM bar (2e-5)."""
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg1", ns=4000, nf=3000, n_modes=5)
    sr, sz, tr, tz, qr, qi = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    out = []
    for eng in ("auto", "cuda_cores"):
        pl = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=M, depth=4, precision="mixed", s2l_engine=eng)
        out.append(to_np(*pl.grad(qr, qi)))
        pl.close()
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=4)
    F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], M, 4, geom, grad=True)
    for c in range(0, 6, 2):
        e_eng = eps_modes(out[0][c], out[0][c + 1], out[1][c], out[1][c + 1]).max()
        e_orc = eps_modes(out[0][c], out[0][c + 1], F[c], F[c + 1]).max()
        print("mixed M=%d comp %d: tc vs cuda cores %.2e, vs oracle %.2e" % (M, c, e_eng, e_orc))
        assert e_eng < 2e-5 and e_orc < 2e-5, (M, c, e_eng, e_orc)
