"""afmm_direct_static: the direct sum for callers that cannot allocate device memory.

Such callers (services with a fixed device-memory footprint, code running while another
caching allocator holds the GPU's memory, code that must avoid the device
synchronisation an allocation can imply) get the direct sum with scratch taken from the
library's fixed device array.  The test calls the entry point through the C ABI with
ctypes, twice in a row, and checks both results against afmm_direct's at the FP64
parity bar used elsewhere (1e-10 per mode, Eq. results:error).  Collected last so that a
run stopping at the first failure has already run everything else."""
import ctypes

import numpy as np
import pytest

from paper_2301_01179_gb300 import workloads as W
from tests.gpu_util import eps_modes, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _c_call(lib, w, devs, out_re, out_im, stream):
    P = ctypes.c_void_p
    sr, sz, tr, tz, qr, qi = devs
    return lib.afmm_direct_static(ctypes.c_int64(w["src_r"].size), P(sr.data_ptr()), P(sz.data_ptr()),
                                  ctypes.c_int64(w["tgt_r"].size), P(tr.data_ptr()), P(tz.data_ptr()),
                                  ctypes.c_int(w["n_modes"]), P(qr.data_ptr()), P(qi.data_ptr()),
                                  P(out_re.data_ptr()), P(out_im.data_ptr()), P(stream))


@pytest.mark.parametrize("kind,ns,nf,nm", [("cfg1", 2000, 2000, 17), ("cfg3", 1500, 45, 33)])
def test_direct_static_matches_direct_twice(kind, ns, nf, nm):
    import torch
    from paper_2301_01179_gb300 import binding
    lib = binding.load()
    w = W.make(kind, ns=ns, nf=nf, n_modes=nm)
    devs = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    stream = torch.cuda.current_stream().cuda_stream
    # the existing entry point
    plan = binding.Plan(*devs[:4], nm, order=4, leaf_size=32)
    ref = to_np(*plan.direct(devs[4], devs[5]))
    plan.close()
    for call in range(2):
        o_re = torch.full((nm, nf), float("nan"), dtype=torch.float64, device="cuda")
        o_im = torch.full((nm, nf), float("nan"), dtype=torch.float64, device="cuda")
        st = _c_call(lib, w, devs, o_re, o_im, stream)
        assert st == 0, binding.last_cuda_error()
        torch.cuda.synchronize()
        got = to_np(o_re, o_im)
        e = eps_modes(got[0], got[1], ref[0], ref[1])
        assert e.max() < TOL, (call, e.max())


def test_direct_static_rejects_oversized_requests():
    import torch
    from paper_2301_01179_gb300 import binding
    lib = binding.load()
    cap = 2097152  # AFMM_STATIC_SCRATCH_DOUBLES
    nm = 33
    ns = cap // (2 * nm) + 1
    w = W.make("cfg1", ns=ns, nf=4, n_modes=nm)
    devs = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    o = torch.zeros(nm, 4, dtype=torch.float64, device="cuda")
    st = _c_call(lib, w, devs, o, o, torch.cuda.current_stream().cuda_stream)
    assert st == 1  # AFMM_EINVAL
