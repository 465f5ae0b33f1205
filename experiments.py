"""The paper's numerical study (Sec. 4) re-run on the GPU.

Carley (arXiv 2301.01179) measures its FMM on a synthetic case: sources and field points
uniform on the unit square 0 <= r, z <= 1, real amplitudes S^(n) in (0, 1), modes
n = 0..17, Ns = Nf = 2^10 .. 2^16, expansion orders M = 6..16 and tree depths d = 4..7, with
the per-mode error eps^(n) = max|Phi_FMM - Phi_D| / max|Phi_D| (Eq. results:error) against
the direct sum.  Its figures are not reproduced as numbers in the text, so this script
produces the same curves for this implementation:

  E1  eps^(n) against n            (Ns = 2^16, d = 6, several M)
  E2  eps against M for n = 0, 8   (Ns = 2^14, 2^16; d = 5, 6, 7) with the fitted slope
      of log10 eps against M (the paper reports eps ~ C^(-0.4 M))
  E3  time against Ns, direct and FMM (M = 6 and the paper's highest order, 16)
  E4  FMM time per phase (tree and set-up, upward pass, expansion coefficients, S2L,
      downward pass, near field and local evaluation)
  E5  error against FMM time over (M, d) at Ns = 2^16

The direct reference is the GPU direct sum of the FP64 path (parity with the CPU oracle is
1e-10, far below the FMM errors measured here).  Times are CUDA-event times of the
potential evaluation (plan creation timed separately), after one warm-up.  One JSON object
per line on stdout.

    python experiments.py [E1 E2 E3 E4 E5] [--quick]
"""
import argparse
import json
import sys

import numpy as np


def _dev(a, torch, dev):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def _eps(a, b):
    """Eq. results:error per mode (complex modulus)."""
    a = np.asarray(a[0]) + 1j * np.asarray(a[1])
    b = np.asarray(b[0]) + 1j * np.asarray(b[1])
    den = np.max(np.abs(b), axis=-1)
    return np.max(np.abs(a - b), axis=-1) / np.where(den > 0, den, 1.0)


class Case:
    """One point set of the paper's test case on the device, with its direct reference."""

    def __init__(self, n, seed=11):
        import torch
        from paper_2301_01179_gb300 import workloads as W
        self.torch = torch
        self.dev = torch.device("cuda", 0)
        w = W.make("paper", ns=n, nf=n)
        self.w = w
        d = lambda a: _dev(a, torch, self.dev)
        self.sr, self.sz, self.tr, self.tz = map(d, (w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"]))
        self.qr, self.qi = d(w["q_re"]), d(w["q_im"])
        self.nm = w["n_modes"]
        self._ref = None
        self.direct_ms = None

    def plan(self, M, depth=0, leaf=32):
        from paper_2301_01179_gb300 import binding
        return binding.Plan(self.sr, self.sz, self.tr, self.tz, self.nm, order=M, depth=depth, leaf_size=leaf)

    def timed(self, fn, reps=1):
        torch = self.torch
        out = fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / reps

    def reference(self):
        if self._ref is None:
            pl = self.plan(6, depth=2)
            out, ms = self.timed(lambda: pl.direct(self.qr, self.qi))
            self._ref = [o.cpu().numpy() for o in out]
            self.direct_ms = ms
            pl.close()
        return self._ref

    def fmm(self, M, depth):
        pl = self.plan(M, depth=depth)
        pl.set_timing(True)
        out, ms = self.timed(lambda: pl.eval(self.qr, self.qi))
        phases = pl.timing()
        res = [o.cpu().numpy() for o in out]
        pl.close()
        return res, ms, phases


def e1(quick):
    n = 2 ** 14 if quick else 2 ** 16
    c = Case(n)
    ref = c.reference()
    for M in (6, 8, 10, 12, 14, 16):
        res, ms, _ = c.fmm(M, 6)
        yield {"exp": "E1", "Ns": n, "d": 6, "M": M, "eps_per_mode": [float(x) for x in _eps(res, ref)]}


def e2(quick):
    sizes = (2 ** 12, 2 ** 14) if quick else (2 ** 14, 2 ** 16)
    for n in sizes:
        c = Case(n)
        ref = c.reference()
        for d in (5, 6, 7):
            eps0, eps8, Ms = [], [], list(range(6, 17))
            for M in Ms:
                res, ms, _ = c.fmm(M, d)
                e = _eps(res, ref)
                eps0.append(float(e[0]))
                eps8.append(float(e[8]))
            # slope of log10 eps against M (the paper: eps ~ C^(-0.4 M))
            s0 = float(np.polyfit(Ms, np.log10(eps0), 1)[0])
            s8 = float(np.polyfit(Ms, np.log10(eps8), 1)[0])
            yield {"exp": "E2", "Ns": n, "d": d, "M": Ms, "eps_n0": eps0, "eps_n8": eps8,
                   "slope_log10_eps_per_M_n0": s0, "slope_log10_eps_per_M_n8": s8}


def e3(quick):
    top = 16 if quick else 20
    for k in range(10, top + 1, 2):
        n = 2 ** k
        c = Case(n)
        c.reference() if k <= 18 else None
        row = {"exp": "E3", "Ns": n, "direct_ms": c.direct_ms}
        for M in (6, 16):
            pl = c.plan(M, leaf=32)
            out, ms = c.timed(lambda: pl.eval(c.qr, c.qi))
            info = pl.info()
            row["fmm_ms_M%d" % M] = ms
            row["depth_M%d" % M] = info["depth"]
            pl.close()
        _, plan_ms = c.timed(lambda: c.plan(6, leaf=32).close())
        row["plan_ms"] = plan_ms
        yield row


def e4(quick):
    n = 2 ** 14 if quick else 2 ** 16
    c = Case(n)
    for M in (6, 12, 16):
        res, ms, ph = c.fmm(M, 6)
        yield {"exp": "E4", "Ns": n, "d": 6, "M": M, "total_ms": ms, "phase_ms": {k: round(v, 4) for k, v in ph.items()}}


def e5(quick):
    n = 2 ** 14 if quick else 2 ** 16
    c = Case(n)
    ref = c.reference()
    for d in (4, 5, 6, 7):
        for M in (6, 8, 10, 12, 14, 16):
            res, ms, _ = c.fmm(M, d)
            e = _eps(res, ref)
            yield {"exp": "E5", "Ns": n, "d": d, "M": M, "fmm_ms": ms, "direct_ms": c.direct_ms,
                   "eps_max_over_modes": float(e.max()), "eps_n0": float(e[0])}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("which", nargs="*", default=["E1", "E2", "E3", "E4", "E5"])
    ap.add_argument("--quick", action="store_true", help="smaller sizes (a minute)")
    args = ap.parse_args(argv)
    runs = {"E1": e1, "E2": e2, "E3": e3, "E4": e4, "E5": e5}
    for k in args.which:
        for row in runs[k](args.quick):
            print(json.dumps(row), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
