"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The oracle cannot run an FMM on 1e6 points, but it can compute the direct sum at a few
sampled field points one by one.  At those samples:
  - the GPU direct sum (FP64) must match the oracle to 1e-10 per mode;
  - the GPU FMM (M = 12, leaf 64, FP64, potential and gradient) must match the oracle's
    direct sum to the FMM's own truncation error (measured 1.0e-6; bound 5e-6);
  - the mixed-precision FMM must stay within its stated bound of the FP64 result.
For the adjoint configuration (2.56e5 x 2.56e5, modes 0..24, M = 10) the FMM gradient of
L = sum |Phi - T|^2 is checked against FP64 central differences (h = 1e-6) of the direct
sum at 64 sampled sources, at the FMM error level."""
import numpy as np
import pytest

import oracle
from paper_2301_01179_gb300 import workloads as W
from tests.gpu_util import eps_modes, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg2():
    return W.make("cfg2")


def test_cfg2_full_size_sampled_parity(cfg2):
    import torch
    from paper_2301_01179_gb300 import binding
    w = cfg2
    sr, sz, tr, tz, qr, qi = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    pl = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=w["order"], leaf_size=w["leaf"])
    out = to_np(*pl.grad(qr, qi))
    pl.close()
    idx = W.subset(w["tgt_r"].size, 8, seed=21)
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"][idx], w["tgt_z"][idx], w["q_re"], w["q_im"], grad=True)
    # GPU direct at the samples
    pd = binding.Plan(sr, sz, *to_dev(w["tgt_r"][idx], w["tgt_z"][idx]), w["n_modes"], order=4, leaf_size=64)
    g = to_np(*pd.direct_grad(qr, qi))
    pd.close()
    for c in range(0, 6, 2):
        assert eps_modes(g[c], g[c + 1], D[c], D[c + 1]).max() < 1e-10, c
    # FMM at the samples (truncation error of the method at M = 12)
    for c in range(0, 6, 2):
        e = eps_modes(out[c][:, idx], out[c + 1][:, idx], D[c], D[c + 1])
        assert e.max() < 5e-6, (c, e.max())


def test_cfg3_mixed_full_size_vs_fp64():
    import torch
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg3")
    sr, sz, tr, tz, qr, qi = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    res = []
    for prec in ("fp64", "mixed"):
        pl = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=w["order"], leaf_size=w["leaf"], precision=prec)
        res.append(to_np(*pl.eval(qr, qi)))
        pl.close()
    e = eps_modes(res[1][0], res[1][1], res[0][0], res[0][1])
    assert e.max() < 2e-5, e.max()


def test_cfg4_adjoint_full_size_vs_finite_differences():
    import torch
    from paper_2301_01179_gb300 import binding
    from paper_2301_01179_gb300.autograd import modal_potential
    w = W.make("cfg4", with_targets=True)
    nm = w["n_modes"]
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    q = torch.complex(*to_dev(w["q_re"], w["q_im"]))
    T = torch.complex(*to_dev(w["T_re"], w["T_im"]))
    pl = binding.Plan(sr, sz, tr, tz, nm, order=w["order"], leaf_size=w["leaf"])
    rv = sr.clone().requires_grad_(True)
    zv = sz.clone().requires_grad_(True)
    phi = modal_potential(q, pl, rv, zv)
    L = (phi - T).abs().pow(2).sum()
    L.backward()
    E = (phi.detach() - T)
    h = 1e-6
    idx = W.subset(w["src_r"].size, 64, seed=33)
    worst = 0.0
    scale = float(rv.grad.abs().max())
    for i in idx:
        for which, g in (("r", rv.grad), ("z", zv.grad)):
            dl = []
            for s in (+1, -1):
                r1 = float(w["src_r"][i]) + (s * h if which == "r" else 0.0)
                z1 = float(w["src_z"][i]) + (s * h if which == "z" else 0.0)
                G1 = binding.green(tr, torch.full_like(tr, r1), tz - z1, nm)
                G0 = binding.green(tr, torch.full_like(tr, float(w["src_r"][i])), tz - float(w["src_z"][i]), nm)
                dphi = q[:, i:i + 1] * (G1 - G0)
                dl.append(float((2 * (E.conj() * dphi).real + dphi.abs().pow(2)).sum()))
            fd = (dl[0] - dl[1]) / (2 * h)
            worst = max(worst, abs(fd - float(g[i])) / scale)
    # E is the FMM residual; the FD is of the direct sum: agreement at the FMM error level
    assert worst < 1e-4, worst
    pl.close()
