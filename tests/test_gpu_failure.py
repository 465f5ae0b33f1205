"""Failure detection on the GPU without a fault: a bounded device-side wait that runs out.

The tensor-core S2L waits on the completion of its own MMAs (mbarrier, 1 s limit).  With the
test hook AFMM_INJECT_TC_TIMEOUT=1 read at plan creation, the first slot of every block issues
no MMA and no completion signal, so the wait can only run out: the block records the timeout
in the plan's error word, waits for its own copies, releases its tensor memory and returns.
The next call on the plan reports AFMM_ETIMEOUT; the CUDA context stays usable, and a plan
created without the hook computes correct results afterwards."""
import numpy as np
import pytest

import oracle
from paper_2301_01179_gb300 import workloads as W
from tests.gpu_util import eps_modes, to_dev, to_np

pytestmark = pytest.mark.gpu


def test_tensor_core_wait_timeout_is_reported_and_context_survives(monkeypatch):
    import torch
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg1", ns=1500, nf=1200, n_modes=2)
    sr, sz, tr, tz, qr, qi = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    monkeypatch.setenv("AFMM_INJECT_TC_TIMEOUT", "1")
    pl = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=4, depth=3)
    monkeypatch.delenv("AFMM_INJECT_TC_TIMEOUT")
    pl.eval(qr, qi)  # the S2L blocks give up after 1 s each
    torch.cuda.synchronize()
    with pytest.raises(binding.AfmmError) as ei:
        pl.eval(qr, qi)
    assert ei.value.status == 4  # AFMM_ETIMEOUT
    torch.cuda.synchronize()
    pl.close()
    # the context is intact: a plan without the hook is correct
    pl2 = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=4, depth=3)
    g = to_np(*pl2.eval(qr, qi))
    pl2.close()
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=3)
    F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], 4, 3, geom)
    assert eps_modes(g[0], g[1], F[0], F[1]).max() < 1e-10


def test_near_field_handover_timeout_is_reported_and_context_survives(monkeypatch):
    """The FP32-pair near field hands slots from producer to consumer warps through
    mbarriers whose waits are bounded (1 s).  With AFMM_INJECT_NEAR_TIMEOUT=1 read at plan
    creation, slot 0 of every block is never handed over: the consumers' wait runs out, they
    record the timeout and raise the block's abort flag, the producers waiting for ring space
    see it and leave, and the block ends.  The next call reports AFMM_ETIMEOUT; the context
    stays usable."""
    import torch
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg1", ns=400, nf=300, n_modes=4)
    sr, sz, tr, tz, qr, qi = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    monkeypatch.setenv("AFMM_INJECT_NEAR_TIMEOUT", "1")
    pl = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=4, depth=3)
    monkeypatch.delenv("AFMM_INJECT_NEAR_TIMEOUT")
    pl.eval(qr, qi)  # the near-field blocks give up after 1 s
    torch.cuda.synchronize()
    with pytest.raises(binding.AfmmError) as ei:
        pl.eval(qr, qi)
    assert ei.value.status == 4  # AFMM_ETIMEOUT
    torch.cuda.synchronize()
    pl.close()
    pl2 = binding.Plan(sr, sz, tr, tz, w["n_modes"], order=4, depth=3)
    g = to_np(*pl2.eval(qr, qi))
    pl2.close()
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=3)
    F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], 4, 3, geom)
    assert eps_modes(g[0], g[1], F[0], F[1]).max() < 1e-10
