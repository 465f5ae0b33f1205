"""GPU adjoint through torch.autograd: gradients of L = sum_n,j |Phi - T|^2 with respect
to the complex amplitudes and the source positions, checked against the oracle's analytic
adjoint and against FP64 central finite differences (h = 1e-6) of the direct sum."""
import numpy as np
import pytest

import oracle
from paper_2301_01179_gb300 import workloads as W
from tests.gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def _setup(ns, nf, nm, M=10, leaf=32):
    import torch
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg4", ns=ns, nf=nf, n_modes=nm, with_targets=True)
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    pl = binding.Plan(sr, sz, tr, tz, nm, order=M, leaf_size=leaf)
    q = torch.complex(*to_dev(w["q_re"], w["q_im"]))
    T = torch.complex(*to_dev(w["T_re"], w["T_im"]))
    return w, pl, sr, sz, q, T


def _autograd(pl, sr, sz, q, T, direct):
    import torch
    from paper_2301_01179_gb300.autograd import modal_potential
    qv = q.clone().requires_grad_(True)
    rv = sr.clone().requires_grad_(True)
    zv = sz.clone().requires_grad_(True)
    phi = modal_potential(qv, pl, rv, zv, direct=direct)
    L = (phi - T).abs().pow(2).sum()
    L.backward()
    return qv.grad, rv.grad, zv.grad, phi.detach()


@pytest.mark.parametrize("direct", [True, False])
def test_autograd_matches_oracle_adjoint(direct):
    w, pl, sr, sz, q, T = _setup(1500, 1200, 9)
    gq, gr, gz, phi = _autograd(pl, sr, sz, q, T, direct)
    E = phi.cpu().numpy() - (w["T_re"] + 1j * w["T_im"])
    if direct:
        A = oracle.adjoint_direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"],
                                  2 * E.real, 2 * E.imag)
    else:
        d = pl.info()["depth"]
        _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=d)
        A = oracle.adjoint_fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], 2 * E.real,
                               2 * E.imag, 10, d, geom)
    gq = gq.cpu().numpy()
    assert np.max(np.abs(gq - (A[0] + 1j * A[1]))) < 1e-10 * np.max(np.abs(A[0] + 1j * A[1]))
    np.testing.assert_allclose(to_np(gr)[0], A[2], rtol=0, atol=1e-10 * np.abs(A[2]).max())
    np.testing.assert_allclose(to_np(gz)[0], A[3], rtol=0, atol=1e-10 * np.abs(A[3]).max())


def test_direct_adjoint_vs_central_differences():
    # FD on the direct path (reading: moving a source across a box edge changes the FMM's
    # truncation error, so FD of the FMM is meaningful only to ~eps_FMM / h)
    import torch
    from paper_2301_01179_gb300 import binding
    w, pl, sr, sz, q, T = _setup(2000, 1500, 25)
    gq, gr, gz, phi = _autograd(pl, sr, sz, q, T, True)
    E = (phi - T)
    tr, tz = to_dev(w["tgt_r"], w["tgt_z"])
    nf = tr.numel()
    h = 1e-6
    idx = W.subset(w["src_r"].size, 16, seed=9)
    for i in idx:
        for which, g in (("r", gr), ("z", gz)):
            dl = []
            for s in (+1, -1):
                r1 = float(w["src_r"][i]) + (s * h if which == "r" else 0.0)
                z1 = float(w["src_z"][i]) + (s * h if which == "z" else 0.0)
                G1 = binding.green(tr, torch.full_like(tr, r1), tz - z1, 25)
                G0 = binding.green(tr, torch.full_like(tr, float(w["src_r"][i])), tz - float(w["src_z"][i]), 25)
                dphi = q[:, i:i + 1] * (G1 - G0)
                dl.append(float((2 * (E.conj() * dphi).real + dphi.abs().pow(2)).sum()))
            fd = (dl[0] - dl[1]) / (2 * h)
            gi = float(g[i])
            assert abs(fd - gi) <= 2e-7 * max(1.0, abs(gi)), (i, which, fd, gi)
