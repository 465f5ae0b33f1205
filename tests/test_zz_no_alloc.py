"""afmm_direct_static: the direct sum for callers that cannot allocate device memory.

Such callers (services with a fixed device-memory footprint, code running while another
caching allocator holds the GPU's memory, code that must avoid the device
synchronisation an allocation can imply) get the direct sum with scratch taken from the
library's fixed device array.  The tests call the entry point through the C ABI with
ctypes and check:
  - two calls in a row against afmm_direct's result at the FP64 parity bar used elsewhere
    (1e-10 per mode, Eq. results:error), with the device's free memory (cudaMemGetInfo)
    unchanged across them, including a case where the room left in the array, not the
    number of field-point units, limits the source split;
  - one call captured into a CUDA graph after a warm-up call, replayed, same bar;
  - the CUDA-event time of both entry points (printed: the static one runs the native
    FP64 kernel, afmm_direct the FP32-pair kernel).
Collected last so that a run stopping at the first failure has already run everything
else."""
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


def _split_count(ns, nf, nm, cap=2097152):
    """The source split afmm_direct_static chooses (restated from its documented rule:
    enough splits to give 152 x 8 units of 32 field points, at most one per 64 sources,
    at most what the rest of the array holds)."""
    need = 2 * nm * ns
    tunits, want = (nf + 31) // 32, 152 * 8
    room = (cap - need) // (2 * nm * nf)
    if tunits >= want:
        return 1, room
    return max(1, min((want + tunits - 1) // tunits, (ns + 63) // 64, room)), room


@pytest.mark.parametrize("kind,ns,nf,nm", [("cfg1", 2000, 2000, 17), ("cfg3", 1500, 45, 33), ("cfg1", 5000, 10000, 33)])
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
    nsplit, room = _split_count(ns, nf, nm)
    if ns == 5000:
        assert nsplit == room == 2  # the array's room decides the split here
    outs = [(torch.full((nm, nf), float("nan"), dtype=torch.float64, device="cuda"),
             torch.full((nm, nf), float("nan"), dtype=torch.float64, device="cuda")) for _ in range(2)]
    torch.cuda.synchronize()
    free0 = None
    for call in range(2):
        o_re, o_im = outs[call]
        st = _c_call(lib, w, devs, o_re, o_im, stream)
        assert st == 0, binding.last_cuda_error()
        torch.cuda.synchronize()
        if free0 is None:
            free0 = torch.cuda.mem_get_info()[0]  # after the first call (module loaded)
        got = to_np(o_re, o_im)
        e = eps_modes(got[0], got[1], ref[0], ref[1])
        assert e.max() < TOL, (call, e.max())
    assert torch.cuda.mem_get_info()[0] >= free0


def test_direct_static_in_a_cuda_graph_and_its_cost():
    import torch
    from paper_2301_01179_gb300 import binding
    lib = binding.load()
    nm = 17
    w = W.make("cfg1", ns=4096, nf=4096, n_modes=nm)
    devs = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    plan = binding.Plan(*devs[:4], nm, order=4, leaf_size=32)
    ref = to_np(*plan.direct(devs[4], devs[5]))
    o_re = torch.zeros(nm, 4096, dtype=torch.float64, device="cuda")
    o_im = torch.zeros_like(o_re)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        assert _c_call(lib, w, devs, o_re, o_im, s.cuda_stream) == 0  # warm-up, outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    o_re.fill_(float("nan"))
    o_im.fill_(float("nan"))
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        st = _c_call(lib, w, devs, o_re, o_im, torch.cuda.current_stream().cuda_stream)
    assert st == 0, binding.last_cuda_error()
    g.replay()
    torch.cuda.synchronize()
    got = to_np(o_re, o_im)
    assert eps_modes(got[0], got[1], ref[0], ref[1]).max() < TOL
    # cost of the two entry points (CUDA events, 5 calls each after the calls above)
    cur = torch.cuda.current_stream()
    times = {}
    for name, fn in (("afmm_direct", lambda: plan.direct(devs[4], devs[5])),
                     ("afmm_direct_static", lambda: _c_call(lib, w, devs, o_re, o_im, cur.cuda_stream))):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            fn()
        e1.record()
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / 5
    plan.close()
    print("direct-sum cost, cfg1 laws 4096 x 4096, 17 modes: %.3f ms (afmm_direct), %.3f ms (afmm_direct_static), x%.1f"
          % (times["afmm_direct"], times["afmm_direct_static"], times["afmm_direct_static"] / times["afmm_direct"]))


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
