"""Seeded synthetic inputs for the modal ring-source problem.

This module holds input generators only (no arithmetic of the method), so that the CUDA
path, the CPU oracle, the tests and the benchmark all see identical inputs.

Each workload draws four independent streams from one ``numpy.random.SeedSequence``:
source positions, field-point positions, source amplitudes S_i^(n) and (for the adjoint
loss) target values T_j^(n).  Amplitudes are mode-major float64 planes ``[n_modes, n]``.

Workloads (sizes and laws of the benchmark configurations; the paper's own test case,
Sec. 4, is ``paper``: uniform points on the unit square, real amplitudes in (0, 1),
modes 0..17):

* ``cfg1``  2,000 / 2,000 rings, r ~ U[0.1, 1], z ~ U[-1, 1], modes 0..16, complex
  N(0,1) amplitudes, order M = 8, leaf 32.
* ``cfg2``  1e6 / 1e6, r ~ U[0.05, 2], z ~ U[-2, 2], modes 0..32, M = 12, leaf 64.
* ``cfg3``  1e6 / 1e6 on the curve r = 0.5 + 0.2 cos t, z = 0.3 sin t, t ~ U[0, 2 pi),
  plus N(0, 5e-3) jitter per coordinate; modes 0..32, M = 12, leaf 64.
* ``cfg4``  2.56e5 / 2.56e5 with the cfg1 law, modes 0..24, M = 10, leaf 64, plus
  complex N(0,1) targets T for the loss sum |Phi - T|^2.
* ``cfg5``  4e6 / 4e6, r ~ Exponential(mean 0.5) truncated to [0.01, 3] by redrawing,
  z ~ N(0, 1); |S^(n)| = max(n, 1)^-2 with uniform phase; modes 0..64, M = 14, leaf 64.
"""
import numpy as np

CONFIGS = {
    "cfg1": dict(ns=2000, nf=2000, n_modes=17, order=8, leaf=32, seed=1),
    "cfg2": dict(ns=1_000_000, nf=1_000_000, n_modes=33, order=12, leaf=64, seed=2),
    "cfg3": dict(ns=1_000_000, nf=1_000_000, n_modes=33, order=12, leaf=64, seed=3),
    "cfg4": dict(ns=256_000, nf=256_000, n_modes=25, order=10, leaf=64, seed=4),
    "cfg5": dict(ns=4_000_000, nf=4_000_000, n_modes=65, order=14, leaf=64, seed=5),
    "paper": dict(ns=4096, nf=4096, n_modes=18, order=12, leaf=32, seed=11),
}


def _streams(seed):
    ss = np.random.SeedSequence(seed)
    return [np.random.default_rng(s) for s in ss.spawn(4)]


def _points(kind, rng, n):
    if kind in ("cfg1", "cfg4"):
        return rng.uniform(0.1, 1.0, n), rng.uniform(-1.0, 1.0, n)
    if kind == "cfg2":
        return rng.uniform(0.05, 2.0, n), rng.uniform(-2.0, 2.0, n)
    if kind == "cfg3":
        t = rng.uniform(0.0, 2.0 * np.pi, n)
        r = 0.5 + 0.2 * np.cos(t) + rng.normal(0.0, 5e-3, n)
        z = 0.3 * np.sin(t) + rng.normal(0.0, 5e-3, n)
        return r, z
    if kind == "cfg5":
        r = rng.exponential(0.5, n)
        bad = (r < 0.01) | (r > 3.0)
        while bad.any():
            r[bad] = rng.exponential(0.5, int(bad.sum()))
            bad = (r < 0.01) | (r > 3.0)
        return r, rng.normal(0.0, 1.0, n)
    if kind == "paper":
        # uniform on 0 < r <= 1, 0 <= z <= 1 (r = 0 is the axis, excluded)
        return 1.0 - rng.uniform(0.0, 1.0, n), rng.uniform(0.0, 1.0, n)
    raise ValueError(kind)


def _amplitudes(kind, rng, n_modes, n):
    if kind == "paper":
        return rng.uniform(0.0, 1.0, (n_modes, n)), np.zeros((n_modes, n))
    if kind == "cfg5":
        mag = 1.0 / np.maximum(np.arange(n_modes), 1.0) ** 2
        ph = rng.uniform(0.0, 2.0 * np.pi, (n_modes, n))
        return mag[:, None] * np.cos(ph), mag[:, None] * np.sin(ph)
    return rng.standard_normal((n_modes, n)), rng.standard_normal((n_modes, n))


def make(kind, ns=None, nf=None, n_modes=None, with_targets=False):
    """Return a dict with src_r, src_z, tgt_r, tgt_z, q_re, q_im (and T_re, T_im when
    ``with_targets``), plus the workload's order, leaf and n_modes.  ``ns``, ``nf`` and
    ``n_modes`` override the configuration's sizes (same laws, same seed)."""
    c = dict(CONFIGS[kind])
    ns = c["ns"] if ns is None else int(ns)
    nf = c["nf"] if nf is None else int(nf)
    nm = c["n_modes"] if n_modes is None else int(n_modes)
    rs, rt, rq, rT = _streams(c["seed"])
    sr, sz = _points(kind, rs, ns)
    tr, tz = _points(kind, rt, nf)
    qr, qi = _amplitudes(kind, rq, nm, ns)
    out = dict(src_r=np.ascontiguousarray(sr), src_z=np.ascontiguousarray(sz),
               tgt_r=np.ascontiguousarray(tr), tgt_z=np.ascontiguousarray(tz),
               q_re=np.ascontiguousarray(qr), q_im=np.ascontiguousarray(qi),
               order=c["order"], leaf=c["leaf"], n_modes=nm, kind=kind)
    if with_targets:
        out["T_re"] = rT.standard_normal((nm, nf))
        out["T_im"] = rT.standard_normal((nm, nf))
    return out


def subset(n, k, seed=0):
    """A seeded sorted subset of k indices out of n (for sampled checks at full size)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, n, k]))
    return np.sort(rng.choice(n, size=min(k, n), replace=False))
