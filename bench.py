#!/usr/bin/env python
"""Benchmark of the cylindrical-coordinate FMM (arXiv 2301.01179) on one GB300.

Metric: modal ring interactions per second, Ns * Nf * (N + 1) / step time, where a step
is one pass of the hot path over the 1e6-source / 1e6-field-point FP64 workload (r ~
U[0.05, 2], z ~ U[-2, 2], modes 0..32, order 12, leaf 64): quadtree build (plan
creation), FMM potential and field gradient.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (direct modal sum in FP64, OpenMP) on a bounded
sample of field points of the same workload, in the same unit.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "modal ring interactions/s FMM vs direct on 1 GB300 at 1e-10 rel err; fwd+bwd ms"
UNIT = "modal ring interactions/s"
WORKLOAD = "cfg2"
WORKLOAD_DESC = ("1,000,000 ring sources x 1,000,000 field points, r~U[0.05,2], z~U[-2,2], modes n=0..32, "
                 "complex N(0,1) amplitudes, FMM order 12, leaf 64, FP64")
# FP32 issue peak of the GB300 from its unit counts and clock (152 SMs x 128 FP32 lanes x
# 2.07 GHz, an FMA counting as one operation): context only; the rooflines use the peaks
# measured at run time by the FMA probes of libafmm_peaks.so.
FP32_NOMINAL_TOPS = 152 * 128 * 2.07e9 / 1e12
# Method work of the near field per (field point, source) pair, with the field gradient:
# ~80 FP64 operations of set-up (pair geometry, 2 square roots, 2 divisions, the AGM start
# values), then per mode 3 for the recursion step and 2 for the (complex) accumulation, and 6
# more for the gradient (two derivative weights, four accumulations): 80 + 11 (N + 1).
NEAR_METHOD_SETUP, NEAR_METHOD_MODE = 80, 3 + 2 + 6
# What the FP32-pair kernel issues per pair (its own arithmetic, for the issue-utilisation
# figure): ~600 FP32 operations of set-up, then per mode 22 (forward recursion step), 30 (scale
# and two compensated accumulations) and 88 (derivative weight and four compensated
# accumulations).  Miller pairs' longer sweeps are not counted.
NEAR_ISSUE_SETUP, NEAR_ISSUE_MODE = 600, 22 + 30 + 88
# S2L on the tensor cores: 21 digit-slice products per FP64-equivalent multiply-add
S2L_SLICE_PAIRS = 21


def l2p_issue_ops(M):
    """FP32 operations the local-expansion kernel issues (value and gradient, FP32 pairs) per
    field point, mode and real/imaginary part: per coefficient two pair multiply-adds (32), per
    axial degree three (48)."""
    return 32 * (M + 1) * (M + 2) // 2 + 48 * (M + 1)


def l2p_method_ops(M):
    """Method work of the local expansion with gradient per (field point, mode), complex:
    value 2 ncoef FMA plus 2 ncoef for each gradient component."""
    return 3 * 2 * (M + 1) * (M + 2) // 2


def measure_fma_peaks(dev):
    """Measured FMA throughput of this GPU (T operations/s, one FMA = one operation) from the
    probes of libafmm_peaks.so: FP32 scalar, FP32 packed f32x2, FP64; CUDA events on the
    current stream around 3 launches after one warm-up, each launch sized to ~50 ms."""
    import ctypes
    import torch
    from paper_2301_01179_gb300 import build as B
    lib = ctypes.CDLL(B.PEAKS_OUT)
    lib.afmm_peak_launch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    lib.afmm_peak_launch.restype = ctypes.c_int
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = nsm * 8
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = {}
    for kind, name, iters in ((0, "fp32", 400000), (1, "fp32x2", 200000), (2, "fp64", 6000)):
        ops = ctypes.c_double()
        rc = lib.afmm_peak_launch(kind, blocks, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops), st)
        if rc != 0:
            raise RuntimeError("afmm_peak_launch %d failed: %d" % (kind, rc))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            lib.afmm_peak_launch(kind, blocks, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops), st)
        e1.record()
        torch.cuda.synchronize()
        out[name] = 3 * ops.value / (e0.elapsed_time(e1) / 1e3) / 1e12
    out["fp32_best"] = max(out["fp32"], out["fp32x2"])
    out["probe"] = ("libafmm_peaks.so: %d blocks x 256 threads x 8 independent FMA chains, CUDA events over 3 launches"
                    % blocks)
    return out


def measured_bf16_peak():
    """Dense bf16 tensor peak (TFLOP/s) measured on the GB300s: the sustained figure
    (the S2L runs inside a long step), else the documented fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["bf16_tflops_sustained"]), "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
    except Exception:
        return 1700.0, "fallback 1.7 PFLOP/s sustained bf16 (of fallback)"


def read_traffic():
    """DRAM bytes per step of a kernel, from the ncu summaries under profiles/ (lines
    `traffic_per_step <kernel>: <bytes>`), valid only for the kernel version captured."""
    out = {}
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return out
    for f in sorted(os.listdir(d)):
        if not f.endswith(".txt"):
            continue
        for ln in open(os.path.join(d, f)):
            if ln.startswith("traffic_per_step "):
                k, v = ln[len("traffic_per_step "):].split(":")
                out[k.strip()] = float(v)
    return out


def log(*a):
    print(*a, file=sys.stderr, flush=True)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("AFMM_BENCH_GLOO") is None else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v, device):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(ws, units_per_rank_step, t_ms_local, device):
    """Whole-job throughput: each rank processes its own replica of the workload; the job's
    step time is the slowest rank's.  Returns (value, ms_per_step)."""
    t = max_over_ranks(ws, t_ms_local, device)
    return ws * units_per_rank_step / (t / 1e3), t


def cpu_baseline(w, budget_s=15.0):
    """The oracle (CPU FP64 direct sum, OpenMP on all host cores) on a bounded sample of
    field points against all sources; rate in modal interactions/s."""
    import numpy as np
    import oracle
    from paper_2301_01179_gb300 import workloads as W
    nf = w["tgt_r"].size
    cores = oracle.num_threads()
    idx = W.subset(nf, 4, seed=7)
    t0 = time.time()
    oracle.direct(w["src_r"], w["src_z"], w["tgt_r"][idx], w["tgt_z"][idx], w["q_re"], w["q_im"])
    per = (time.time() - t0) / len(idx)
    k = int(max(4, min(1024, budget_s / max(per, 1e-6))))
    idx = W.subset(nf, k, seed=8)
    t0 = time.time()
    oracle.direct(w["src_r"], w["src_z"], w["tgt_r"][idx], w["tgt_z"][idx], w["q_re"], w["q_im"])
    dt = time.time() - t0
    rate = len(idx) * w["src_r"].size * w["n_modes"] / dt
    # one core (the paper's single-core setting): 2 field points against a seeded fifth of the
    # sources
    ns1 = max(1, w["src_r"].size // 5)
    si = W.subset(w["src_r"].size, ns1, seed=9)
    ti = W.subset(nf, 2, seed=10)
    t0 = time.time()
    oracle.direct(w["src_r"][si], w["src_z"][si], w["tgt_r"][ti], w["tgt_z"][ti],
                  np.ascontiguousarray(w["q_re"][:, si]), np.ascontiguousarray(w["q_im"][:, si]), threads=1)
    dt1 = time.time() - t0
    # the thread count of the oracle's OpenMP runtime back to all cores
    oracle.direct(w["src_r"][:1], w["src_z"][:1], w["tgt_r"][:1], w["tgt_z"][:1],
                  np.ascontiguousarray(w["q_re"][:, :1]), np.ascontiguousarray(w["q_im"][:, :1]), threads=cores)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "oracle direct sum (FP64) for %d seeded field points against all %d sources, %d modes, "
                      "%.1f s" % (len(idx), w["src_r"].size, w["n_modes"], dt),
            "value_1_core": len(ti) * ns1 * w["n_modes"] / dt1,
            "sample_1_core": "one thread: %d field points against %d seeded sources, %.1f s" % (len(ti), ns1, dt1)}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from paper_2301_01179_gb300 import workloads as W
    import oracle
    w = W.make(WORKLOAD, ns=args.ns, nf=args.nf)
    nf = w["tgt_r"].size
    # size one step to about 5 s of CPU work
    idx = W.subset(nf, 4, seed=7)
    t0 = time.time()
    oracle.direct(w["src_r"], w["src_z"], w["tgt_r"][idx], w["tgt_z"][idx], w["q_re"], w["q_im"])
    per = (time.time() - t0) / 4
    k = int(max(2, min(512, 5.0 / max(per, 1e-6))))
    times = []
    for s in range(args.warmup + args.steps):
        idx = W.subset(nf, k, seed=100 + s)
        t0 = time.time()
        oracle.direct(w["src_r"], w["src_z"], w["tgt_r"][idx], w["tgt_z"][idx], w["q_re"], w["q_im"])
        if s >= args.warmup:
            times.append(time.time() - t0)
    T = sum(times)
    units = args.steps * k * w["src_r"].size * w["n_modes"]
    v = units / T
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "sample_field_points_per_step": k},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d seeded field points per step against all %d sources" % (k, w["src_r"].size)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def fwd_bwd(kind, precision, steps, warmup, dev, tree="uniform"):
    """One forward (potential) and backward (adjoint of L = sum |Phi - T|^2) step of a
    configuration, timed end to end on the device (plan creation included), plus the plan
    creation alone, on the uniform or the adaptive tree.  Returns a dict for the JSON line."""
    import numpy as np
    import torch
    from paper_2301_01179_gb300 import binding, workloads as W
    w = W.make(kind, with_targets=True)
    ns, nf, nm = w["src_r"].size, w["tgt_r"].size, w["n_modes"]

    def d(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    sr, sz, tr, tz, qr, qi, Tr, Ti = map(d, (w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"],
                                             w["T_re"], w["T_im"]))

    def step():
        pl = binding.Plan(sr, sz, tr, tz, nm, order=w["order"], leaf_size=w["leaf"], precision=precision, tree=tree)
        pr, pi = pl.eval(qr, qi)
        out = pl.adjoint(qr, qi, 2.0 * (pr - Tr), 2.0 * (pi - Ti))
        return pl, out

    for _ in range(warmup):
        pl, _o = step()
        pl.close()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        pl, _o = step()
        pl.close()
    e1.record()
    torch.cuda.synchronize()
    t_step = e0.elapsed_time(e1) / steps
    e0.record()
    for _ in range(steps):
        pl = binding.Plan(sr, sz, tr, tz, nm, order=w["order"], leaf_size=w["leaf"], precision=precision, tree=tree)
        inf = pl.info()
        pl.close()
    e1.record()
    torch.cuda.synchronize()
    t_plan = e0.elapsed_time(e1) / steps
    return {"workload": "%s: %d x %d, modes 0..%d, order %d, leaf %d" % (kind, ns, nf, nm - 1, w["order"], w["leaf"]),
            "precision": precision, "tree": tree, "depth": inf["depth"], "near_pairs": inf["near_pairs"],
            "s2l_pairs": inf["s2l_pairs"], "fwd_bwd_ms": t_step, "plan_ms": t_plan, "steps": steps,
            "modal_ring_interactions_per_s": 2.0 * ns * nf * nm / (t_step / 1e3)}


def trees_vs_direct_sampled(kind, k, precision, dev):
    """The FMM on the uniform and on the adaptive tree against the direct sum at k sampled
    field points of a configuration (all its sources): each tree's plan spans all field
    points, the direct sum (the FP64 path's FP32-pair kernel, within 1e-10 of the oracle)
    only the sample; eps^(n) = max |fmm - direct| / max |direct| per mode and component."""
    import numpy as np
    import torch
    from paper_2301_01179_gb300 import binding, workloads as W
    w = W.make(kind)
    nm = w["n_modes"]
    idx = W.subset(w["tgt_r"].size, k, seed=17)

    def d(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    sr, sz, tr, tz, qr, qi = map(d, (w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"]))
    ps = binding.Plan(sr, sz, d(w["tgt_r"][idx]), d(w["tgt_z"][idx]), nm, order=4, leaf_size=w["leaf"])
    ref = [o.cpu().numpy() for o in ps.direct_grad(qr, qi)]
    ps.close()
    ii = torch.as_tensor(idx, device=dev)
    out = {"workload": "%s: %d x %d, modes 0..%d, order %d, leaf %d, %s; %d sampled field points"
                       % (kind, w["src_r"].size, w["tgt_r"].size, nm - 1, w["order"], w["leaf"], precision, k)}
    for tree in ("uniform", "adaptive"):
        pl = binding.Plan(sr, sz, tr, tz, nm, order=w["order"], leaf_size=w["leaf"], precision=precision, tree=tree)
        res = [o[:, ii].cpu().numpy() for o in pl.grad(qr, qi)]
        pl.close()
        eps = {}
        for name, c in (("potential", 0), ("d_dr", 2), ("d_dz", 4)):
            a = res[c] + 1j * res[c + 1]
            b = ref[c] + 1j * ref[c + 1]
            den = np.max(np.abs(b), axis=1)
            eps[name] = float((np.max(np.abs(a - b), axis=1) / np.where(den > 0, den, 1.0)).max())
        out[tree] = eps
    return out


def mixed_vs_fp64(kind, steps, dev):
    """The MIXED path against the FP64 path on a configuration (the near-singular curve
    workload cfg3 by default): the FMM potential and field gradient step of each (plan
    creation included) timed on the device, and the MIXED error per mode and component,
    eps^(n) = max |mixed - fp64| / max |fp64| over the field points.  The FP64 path matches
    the oracle to 1e-10 per mode (parity tests), so this is the error against the oracle up
    to that."""
    import numpy as np
    import torch
    from paper_2301_01179_gb300 import binding, workloads as W
    w = W.make(kind)
    ns, nf, nm = w["src_r"].size, w["tgt_r"].size, w["n_modes"]

    def d(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    sr, sz, tr, tz, qr, qi = map(d, (w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"]))
    res, ms = {}, {}
    for prec in ("fp64", "mixed"):
        def step():
            pl = binding.Plan(sr, sz, tr, tz, nm, order=w["order"], leaf_size=w["leaf"], precision=prec)
            out = pl.grad(qr, qi)
            pl.close()
            return out
        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            out = step()
        e1.record()
        torch.cuda.synchronize()
        ms[prec] = e0.elapsed_time(e1) / steps
        res[prec] = [o.cpu().numpy() for o in out]
        del out
    eps = {}
    for name, c in (("potential", 0), ("d_dr", 2), ("d_dz", 4)):
        a = res["mixed"][c] + 1j * res["mixed"][c + 1]
        b = res["fp64"][c] + 1j * res["fp64"][c + 1]
        den = np.max(np.abs(b), axis=1)
        eps[name] = [float(x) for x in np.max(np.abs(a - b), axis=1) / np.where(den > 0, den, 1.0)]
    return {"workload": "%s: %d x %d, modes 0..%d, order %d, leaf %d" % (kind, ns, nf, nm - 1, w["order"], w["leaf"]),
            "step": "plan + FMM potential and field gradient", "fp64_ms": ms["fp64"], "mixed_ms": ms["mixed"],
            "speedup": ms["fp64"] / ms["mixed"], "steps": steps,
            "eps_max": {k: max(v) for k, v in eps.items()}, "eps_per_mode": eps}


def mixed_vs_fp64_sampled(kind, k, dev):
    """The MIXED path against the FP64 path at k sampled field points of a configuration
    (the 4e6-ring workload by default) against all its sources: one plan over the sources
    and the sampled points per precision (the same tree), FMM potential and gradient,
    eps^(n) = max |mixed - fp64| / max |fp64| per mode and component."""
    import numpy as np
    import torch
    from paper_2301_01179_gb300 import binding, workloads as W
    w = W.make(kind)
    nm = w["n_modes"]
    idx = W.subset(w["tgt_r"].size, k, seed=13)

    def d(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    sr, sz, tr, tz, qr, qi = map(d, (w["src_r"], w["src_z"], w["tgt_r"][idx], w["tgt_z"][idx], w["q_re"], w["q_im"]))
    res, ms = {}, {}
    for prec in ("fp64", "mixed"):
        pl = binding.Plan(sr, sz, tr, tz, nm, order=w["order"], leaf_size=w["leaf"], precision=prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = pl.grad(qr, qi)
        e1.record()
        torch.cuda.synchronize()
        ms[prec] = e0.elapsed_time(e1)
        res[prec] = [o.cpu().numpy() for o in out]
        depth = pl.info()["depth"]
        pl.close()
    eps = {}
    for name, c in (("potential", 0), ("d_dr", 2), ("d_dz", 4)):
        a = res["mixed"][c] + 1j * res["mixed"][c + 1]
        b = res["fp64"][c] + 1j * res["fp64"][c + 1]
        den = np.max(np.abs(b), axis=1)
        eps[name] = [float(x) for x in np.max(np.abs(a - b), axis=1) / np.where(den > 0, den, 1.0)]
    return {"workload": "%s: %d sources x %d sampled field points, modes 0..%d, order %d, leaf %d, depth %d"
                        % (kind, w["src_r"].size, k, nm - 1, w["order"], w["leaf"], depth),
            "fp64_grad_ms": ms["fp64"], "mixed_grad_ms": ms["mixed"],
            "eps_max": {k2: max(v) for k2, v in eps.items()}, "eps_per_mode": eps}


def native_step(w, dev):
    """The headline step (plan + FMM potential and gradient) with AFMM_FP64_NATIVE: every
    floating-point operation in native FP64 (CUDA cores), one warm-up and one timed step."""
    import numpy as np
    import torch
    from paper_2301_01179_gb300 import binding

    def d(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    sr, sz, tr, tz, qr, qi = map(d, (w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"]))
    nm = w["n_modes"]
    phases = None
    for it in range(2):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pl = binding.Plan(sr, sz, tr, tz, nm, order=w["order"], leaf_size=w["leaf"], precision="fp64_native")
        if it == 1:
            pl.set_timing(True)
        pl.grad(qr, qi)
        if it == 1:
            phases = {k: round(v, 2) for k, v in pl.timing().items()}
        pl.close()
        e1.record()
        torch.cuda.synchronize()
    return {"step_ms": e0.elapsed_time(e1), "phase_ms": phases,
            "step": "plan + FMM potential and field gradient, AFMM_FP64_NATIVE"}


def run_ours(args):
    import numpy as np
    import torch
    from paper_2301_01179_gb300 import binding, workloads as W

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.make(WORKLOAD, ns=args.ns, nf=args.nf)
    if ws > 1:  # independent replica per rank (different seed), weak scaling
        w2 = W.make(WORKLOAD, ns=args.ns, nf=args.nf)
        rng = np.random.default_rng(1000 + rank)
        perm = rng.permutation(w2["src_r"].size)
        for k in ("src_r", "src_z"):
            w[k] = np.ascontiguousarray(w2[k][perm])
        w["q_re"] = np.ascontiguousarray(w2["q_re"][:, perm])
        w["q_im"] = np.ascontiguousarray(w2["q_im"][:, perm])
    ns, nf, nm = w["src_r"].size, w["tgt_r"].size, w["n_modes"]
    M, leaf = w["order"], w["leaf"]
    units_per_step = float(ns) * nf * nm

    def d(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    sr, sz, tr, tz, qr, qi = map(d, (w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"]))
    torch.cuda.synchronize()

    def step(timing=False):
        pl = binding.Plan(sr, sz, tr, tz, nm, order=M, leaf_size=leaf)
        if timing:
            pl.set_timing(True)
        out = pl.grad(qr, qi)
        return pl, out

    info = None
    for _ in range(args.warmup):
        pl, out = step()
        info = pl.info()
        pl.close()
    torch.cuda.synchronize()

    # ---- timed region: inputs resident in HBM (528 MB of amplitudes, larger than L2)
    clk = ClockSampler(local)
    clk.start()
    barrier(ws)
    torch.cuda.synchronize()
    l0 = binding.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    phases = []
    for _ in range(args.steps):
        pl, out = step(timing=True)
        phases.append(pl.timing())
        pl.close()
    e1.record()
    torch.cuda.synchronize()
    barrier(ws)
    launches = binding.kernel_launches() - l0
    clocks = clk.stop()
    value, t_ms = aggregate(ws, units_per_step, e0.elapsed_time(e1) / args.steps, dev)

    # ---- rooflines, from the live phase split of the timed steps (CUDA events recorded by the
    # library on the plan's stream around each phase) and the FMA peaks measured on this GPU.
    # Achieved = the method's work (per-pair and per-box-pair operation counts of the method
    # itself, not the FP32-pair emulation's own instructions) / the kernel's time; the
    # emulation's issue rate is reported beside it.
    nc = (M + 1) * (M + 2) // 2
    s2l_ms = statistics.mean(p["s2l"] for p in phases)
    near_ms = statistics.mean(p["near"] for p in phases)
    traffic_of = read_traffic()
    pk = measure_fma_peaks(dev)
    near_work = NEAR_METHOD_SETUP + nm * NEAR_METHOD_MODE
    near_ach = float(info["near_pairs"]) * near_work / (near_ms / 1e3) / 1e12
    near_issue = float(info["near_pairs"]) * (NEAR_ISSUE_SETUP + nm * NEAR_ISSUE_MODE) / (near_ms / 1e3) / 1e12
    near_roof = {"bound": "alu", "kernel": "k_near_ws (near field, potential and gradient, FP32 pairs)",
                 "achieved": near_ach, "peak": pk["fp32_best"], "unit": "T operations/s (FMA = 1)",
                 "frac": near_ach / pk["fp32_best"], "traffic": traffic_of.get("k_near_ws"),
                 "work_per_unit": "%d method operations per near pair (%d + %d (N+1), FP64-class: set-up, "
                                  "recursion, accumulation, gradient) x %d pairs per launch"
                                  % (near_work, NEAR_METHOD_SETUP, NEAR_METHOD_MODE, info["near_pairs"]),
                 "peak_source": "measured FP32 FMA peak (of measured; libafmm_peaks.so, best of scalar and f32x2)",
                 "frac_of_fp64_pipe": near_ach / pk["fp64"],
                 "fp64_peak": pk["fp64"],
                 "issue_utilisation": near_issue / pk["fp32_best"],
                 "issue_work_per_unit": "%d FP32 operations per near pair issued by the FP32-pair kernel"
                                        % (NEAR_ISSUE_SETUP + nm * NEAR_ISSUE_MODE)}
    bf16_peak, bf16_src = measured_bf16_peak()
    s2l_method = float(info["s2l_pairs"]) * nm * 4.0 * nc * nc  # 2 ncoef^2 FMA per (box pair, mode)
    s2l_ach = s2l_method / (s2l_ms / 1e3) / 1e12
    s2l_roof = {"bound": "tensor", "kernel": "k_slice_moments + k_s2l_tc (tcgen05 bf16, exact 6-digit slicing; "
                                             "all levels)",
                "achieved": s2l_ach, "peak": bf16_peak, "unit": "TFLOP/s", "frac": s2l_ach / bf16_peak,
                "traffic": traffic_of.get("k_s2l_tc"),
                "work_per_unit": "2 ncoef^2 FMA (4 ncoef^2 flop, FP64-equivalent) per (box pair, mode); %d box pairs "
                                 "x %d modes" % (info["s2l_pairs"], nm),
                "peak_source": bf16_src,
                "tensor_issue_utilisation": s2l_ach * S2L_SLICE_PAIRS / bf16_peak,
                "tensor_work_per_unit": "21 digit-slice products x 4 ncoef^2 bf16 flop per (box pair, mode)"}
    l2p_ms = statistics.mean(p["l2p"] for p in phases)
    l2p_work = nm * l2p_method_ops(M)
    l2p_ach = float(nf) * l2p_work / (l2p_ms / 1e3) / 1e12
    l2p_issue = float(nf) * 2 * nm * l2p_issue_ops(M) / (l2p_ms / 1e3) / 1e12
    l2p_roof = {"bound": "alu", "kernel": "k_l2p (local expansion at the field points, value and gradient, FP32 pairs)",
                "achieved": l2p_ach, "peak": pk["fp32_best"], "unit": "T operations/s (FMA = 1)",
                "frac": l2p_ach / pk["fp32_best"], "traffic": traffic_of.get("k_l2p"),
                "work_per_unit": "%d method FMA per field point (6 ncoef per mode: value and two gradient "
                                 "components, complex) x %d points" % (l2p_work, nf),
                "peak_source": near_roof["peak_source"], "frac_of_fp64_pipe": l2p_ach / pk["fp64"],
                "issue_utilisation": l2p_issue / pk["fp32_best"]}
    roofline, secondary = (near_roof, s2l_roof) if near_ms >= s2l_ms else (s2l_roof, near_roof)
    phase_ms = {k: round(statistics.mean(p[k] for p in phases), 3) for k in phases[0]}

    if args.no_extras:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": t_ms,
                              "phase_ms": {k: round(statistics.mean(p[k] for p in phases), 3) for k in phases[0]},
                              "roofline": roofline, "roofline_secondary": secondary, "roofline_l2p": l2p_roof,
                              "fma_peaks": pk, "profiling_run": True}),
                  flush=True)
        return 0
    # ---- e2e: the public API with host buffers (H2D of inputs, D2H of results each step).
    # A serving pipeline over steps: step k + 1's inputs go up from pinned host memory on an
    # H2D stream while step k computes, and step k's six result planes come back into pinned
    # host memory on a D2H stream while step k + 1 computes (two buffer sets each way).  The
    # first upload and the last download are inside the timed region.  Events on the copy
    # streams give their busy time per step.
    hp = [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).pin_memory()
          for a in (w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])]
    hout = [[torch.empty(nm, nf, dtype=torch.float64).pin_memory() for _ in range(6)] for _ in range(2)]
    dins = [[torch.empty(t.shape, dtype=torch.float64, device=dev) for t in hp] for _ in range(2)]
    s_up, s_down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    h2d = sum(t.numel() * 8 for t in hp)
    d2h = sum(t.numel() * 8 for t in hout[0])
    ev_in = [torch.cuda.Event() for _ in range(2)]    # inputs of a slot uploaded
    ev_used = [torch.cuda.Event() for _ in range(2)]  # the step that read a slot's inputs is done

    def upload(k, evs=None):
        b = k % 2
        with torch.cuda.stream(s_up):
            s_up.wait_event(ev_used[b])
            if evs:
                evs[0].record(s_up)
            for dst, src in zip(dins[b], hp):
                dst.copy_(src, non_blocking=True)
            if evs:
                evs[1].record(s_up)
            ev_in[b].record(s_up)

    def pipeline(ke, evs=None):
        main = torch.cuda.current_stream()
        for b in range(2):
            ev_used[b].record(main)
        upload(0, evs[0] if evs else None)
        for k in range(ke):
            b = k % 2
            if k + 1 < ke:
                upload(k + 1, evs[k + 1] if evs else None)
            main.wait_event(ev_in[b])
            pl = binding.Plan(dins[b][0], dins[b][1], dins[b][2], dins[b][3], nm, order=M, leaf_size=leaf)
            out = pl.grad(dins[b][4], dins[b][5])
            ev_used[b].record(main)
            s_down.wait_stream(main)
            with torch.cuda.stream(s_down):
                if evs:
                    evs[k][2].record(s_down)
                for h, o in zip(hout[b], out):
                    h.copy_(o, non_blocking=True)
                    o.record_stream(s_down)
                if evs:
                    evs[k][3].record(s_down)
            pl.close()
        torch.cuda.synchronize()

    pipeline(2)
    barrier(ws)
    torch.cuda.synchronize()
    ke = max(5, args.steps)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(ke)]
    t0 = time.time()
    pipeline(ke, evs)
    barrier(ws)
    te = max_over_ranks(ws, (time.time() - t0) / ke, dev)
    split = {"h2d_inputs_busy": statistics.mean(e[0].elapsed_time(e[1]) for e in evs),
             "d2h_results_busy": statistics.mean(e[2].elapsed_time(e[3]) for e in evs)}
    e2e = {"value": ws * units_per_step / te, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": 1e3 * te, "steps": ke,
           "timer": "host clock over all steps; copies overlapped with the neighbouring steps' compute",
           "split_ms": {k: round(v, 3) for k, v in split.items()}}

    extra = {}
    if rank == 0:
        # FMM accuracy and direct rate on a seeded 1024-point sample of the field points
        idx = W.subset(nf, 1024, seed=3)
        pl = binding.Plan(sr, sz, d(w["tgt_r"][idx]), d(w["tgt_z"][idx]), nm, order=4, leaf_size=leaf)
        dd = pl.direct(qr, qi)
        torch.cuda.synchronize()
        t0 = time.time()
        dd = pl.direct(qr, qi)
        torch.cuda.synchronize()
        tdir = time.time() - t0
        pl.close()
        ii = torch.as_tensor(idx, device=dev)
        pl2 = binding.Plan(sr, sz, tr, tz, nm, order=M, leaf_size=leaf)
        f = pl2.eval(qr, qi)
        pl2.close()
        fa = (f[0][:, ii].cpu().numpy() + 1j * f[1][:, ii].cpu().numpy())
        da = (dd[0].cpu().numpy() + 1j * dd[1].cpu().numpy())
        eps = np.max(np.abs(fa - da), axis=1) / np.max(np.abs(da), axis=1)
        extra = {"fmm_eps_vs_direct_max": float(eps.max()), "fmm_eps_vs_direct_n0": float(eps[0]),
                 "direct_gpu_rate": len(idx) * ns * nm / tdir, "direct_sample_points": len(idx)}
        # plan creation (quadtree build and allocation) alone, part of every timed step above
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            binding.Plan(sr, sz, tr, tz, nm, order=M, leaf_size=leaf).close()
        e1.record()
        torch.cuda.synchronize()
        extra["plan_ms"] = e0.elapsed_time(e1) / 3
        # forward + backward (adjoint) steps of the gradient configurations (not the headline)
        fb = {}
        kinds = [("cfg4", "fp64", "uniform")] + ([] if args.no_cfg5 else [("cfg5", "mixed", "adaptive"),
                                                                          ("cfg5", "mixed", "uniform")])
        for kind, prec, tree in kinds:
            key = kind + ("_adaptive" if tree == "adaptive" else "")
            try:
                fb[key] = fwd_bwd(kind, prec, 2 if kind == "cfg5" else 3, 1, dev, tree=tree)
            except Exception as exc:  # an extra must not cost the headline line
                fb[key] = {"error": str(exc)[:200]}
        extra["fwd_bwd"] = fb
        if not args.no_cfg5:
            try:  # the 4e6-ring workload's FMM error on both trees (MIXED) at sampled points
                extra["cfg5_trees_vs_direct"] = trees_vs_direct_sampled("cfg5", 512, "mixed", dev)
            except Exception as exc:
                extra["cfg5_trees_vs_direct"] = {"error": str(exc)[:200]}
        # the mixed-precision path on the near-singular curve workload, and on the 4e6-ring
        # workload at sampled field points (not the headline)
        try:
            extra["mixed_vs_fp64"] = mixed_vs_fp64("cfg3", 2, dev)
        except Exception as exc:
            extra["mixed_vs_fp64"] = {"error": str(exc)[:200]}
        if not args.no_cfg5:
            try:
                extra["mixed_vs_fp64_cfg5"] = mixed_vs_fp64_sampled("cfg5", 1024, dev)
            except Exception as exc:
                extra["mixed_vs_fp64_cfg5"] = {"error": str(exc)[:200]}
        # the same headline step with every operation in native FP64 (what the FP32-pair and
        # tensor-core design buys on this chip)
        try:
            extra["fp64_native_step"] = native_step(w, dev)
        except Exception as exc:
            extra["fp64_native_step"] = {"error": str(exc)[:200]}

    line = None
    if rank == 0:
        cb = cpu_baseline(w) if ws == 1 and not args.no_cpu_baseline else None
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64-class (fp32-pair, bf16-digit tensor, f64)", "data": "synthetic",
                "config": {"workload": WORKLOAD_DESC, "ns": ns, "nf": nf, "n_modes": nm, "order": M, "leaf": leaf,
                           "depth": info["depth"], "step": "quadtree build + FMM potential and field gradient",
                           "l2": "inputs larger than L2 (amplitudes 528 MB per step)",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "roofline_secondary": secondary,
                "roofline_l2p": l2p_roof, "fma_peaks": pk,
                "cpu_baseline": cb,
                "clocks": clocks, "phase_ms": phase_ms,
                "near_pairs": info["near_pairs"], "s2l_pairs": info["s2l_pairs"]}
        line.update(extra)
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ns", type=int, default=None, help="profiling captures: fewer sources (same laws)")
    ap.add_argument("--nf", type=int, default=None, help="profiling captures: fewer field points")
    ap.add_argument("--no-extras", action="store_true", help="profiling captures: skip e2e and accuracy legs")
    ap.add_argument("--no-cfg5", action="store_true",
                    help="skip the 4e6-ring MIXED forward+adjoint step and its sampled error (about 40 s)")
    ap.add_argument("--peaks", action="store_true",
                    help="print only the measured FMA peaks (FP32, f32x2, FP64) with the clocks seen, and exit")
    ap.add_argument("--fwd-bwd-only", default=None, metavar="KIND:PREC:TREE",
                    help="profiling captures: time only one forward + backward step of a configuration "
                         "(e.g. cfg5:mixed:adaptive) over --steps steps after --warmup, print it, and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    from paper_2301_01179_gb300 import build as B
    B.build()
    if args.peaks:
        return run_peaks()
    if args.fwd_bwd_only:
        import torch
        kind, prec, tree = (args.fwd_bwd_only.split(":") + ["fp64", "uniform"])[:3]
        torch.cuda.set_device(0)
        out = fwd_bwd(kind, prec, args.steps, args.warmup, torch.device("cuda", 0), tree=tree)
        print(json.dumps({"fwd_bwd": out}), flush=True)
        return 0
    return run_ours(args)


def run_peaks():
    """The FMA peak probes alone, three times in a row, with the clocks sampled meanwhile."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    clk = ClockSampler(0)
    clk.start()
    runs = [measure_fma_peaks(dev) for _ in range(3)]
    clocks = clk.stop()
    out = {"fma_peaks_tops": {k: [round(r[k], 4) for r in runs] for k in ("fp32", "fp32x2", "fp64")},
           "unit": "T FMA/s (one FMA = one operation)", "probe": runs[0]["probe"],
           "device": torch.cuda.get_device_name(dev), "clocks": clocks}
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
