"""GPU parity of the all-pairs direct sum (afmm_direct, afmm_direct_grad) and of the
quadtree set-up against the oracle, element by element, through the C ABI.
Bar: Eq. results:error per mode <= 1e-10 (FP64 path)."""
import numpy as np
import pytest

import oracle
from paper_2301_01179_gb300 import workloads as W
from tests.gpu_util import eps_modes, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _plan(w, **kw):
    from paper_2301_01179_gb300 import binding
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    return binding.Plan(sr, sz, tr, tz, w["n_modes"], order=kw.pop("order", w["order"]),
                        leaf_size=kw.pop("leaf", w["leaf"]), **kw)


def test_tree_matches_oracle():
    for kind, ns, nf in (("cfg1", None, None), ("cfg2", 20000, 15000), ("cfg3", 20000, 20000), ("cfg5", 30000, 9000)):
        w = W.make(kind, ns=ns, nf=nf)
        pl = _plan(w)
        info = pl.info()
        d, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["leaf"])
        assert info["depth"] == d, kind
        assert (info["r0"], info["z0"], info["side"]) == tuple(geom), kind


def test_direct_cfg1_matches_oracle():
    w = W.make("cfg1")
    pl = _plan(w)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.direct(q_re, q_im))
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    e = eps_modes(g[0], g[1], D[0], D[1])
    assert e.max() < TOL, e
    # element by element as well
    np.testing.assert_allclose(g[0], D[0], rtol=0, atol=TOL * np.abs(D[0]).max())


def test_direct_grad_cfg1_matches_oracle():
    w = W.make("cfg1", ns=1200, nf=800)
    pl = _plan(w)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.direct_grad(q_re, q_im))
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], grad=True)
    for c in range(0, 6, 2):
        e = eps_modes(g[c], g[c + 1], D[c], D[c + 1])
        assert e.max() < TOL, (c, e)


@pytest.mark.parametrize("ns,nf,n_modes", [(1, 1, 1), (1, 33, 2), (37, 1, 5), (100, 257, 17), (513, 31, 65)])
def test_direct_ragged_sizes(ns, nf, n_modes):
    w = W.make("cfg3", ns=ns, nf=nf, n_modes=n_modes)
    pl = _plan(w, order=4, leaf=8)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.direct_grad(q_re, q_im))
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], grad=True)
    for c in range(0, 6, 2):
        assert eps_modes(g[c], g[c + 1], D[c], D[c + 1]).max() < TOL


def test_direct_coincident_points_contribute_zero():
    w = W.make("cfg1", ns=300, nf=300)
    w["tgt_r"][:100] = w["src_r"][:100]
    w["tgt_z"][:100] = w["src_z"][:100]
    pl = _plan(w)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.direct(q_re, q_im))
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    assert np.all(np.isfinite(g[0]))
    assert eps_modes(g[0], g[1], D[0], D[1]).max() < TOL


def test_plan_rejects_bad_coordinates():
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg1", ns=50, nf=40)
    for bad in (0.0, -1.0, np.nan, np.inf):
        sr = w["src_r"].copy()
        sr[7] = bad
        a, b, c, d = to_dev(sr, w["src_z"], w["tgt_r"], w["tgt_z"])
        with pytest.raises(binding.AfmmError) as ei:
            binding.Plan(a, b, c, d, 3)
        assert ei.value.status == 1
    a, b, c, d = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    for kw in (dict(order=-1), dict(leaf_size=0), dict(depth=1), dict(depth=17)):
        with pytest.raises(binding.AfmmError):
            binding.Plan(a, b, c, d, 3, **kw)
    with pytest.raises(binding.AfmmError):
        binding.Plan(a, b, c, d, 0)


def test_direct_is_deterministic():
    w = W.make("cfg1", ns=700, nf=500)
    pl = _plan(w)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    a = to_np(*pl.direct(q_re, q_im))
    b = to_np(*pl.direct(q_re, q_im))
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("n_modes", [89, 129])
def test_direct_mode_ranges_match_oracle(n_modes):
    """More modes than one launch of the FP32-pair near-field kernel holds (72 with the
    gradient): the kernel runs over mode ranges, each recomputing the pair sequences (89:
    72 + 17; 129, the highest order the plans accept: 72 + 57).  Both sweeps (forward and
    Miller) occur at these orders."""
    w = W.make("cfg1", ns=400, nf=300, n_modes=n_modes)
    pl = _plan(w)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.direct_grad(q_re, q_im))
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], grad=True)
    for c in range(0, 6, 2):
        e = eps_modes(g[c], g[c + 1], D[c], D[c + 1])
        assert e.max() < TOL, (c, e.max())


@pytest.mark.parametrize("nf", [1, 5, 16, 17, 33])
def test_fmm_near_lane_packing_matches_oracle_fmm(nf):
    """Near-field units of 1..33 field points: the kernel packs 32 / 2^ceil(log2 c) sources
    into each slot for small units and sums the lane groups at the end."""
    w = W.make("cfg1", ns=2000, nf=nf, n_modes=6)
    pl = _plan(w, order=4, depth=3)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.grad(q_re, q_im))
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=3)
    F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], 4, 3, geom, grad=True)
    for c in range(0, 6, 2):
        e = eps_modes(g[c], g[c + 1], F[c], F[c + 1])
        assert e.max() < TOL, (c, e.max())


def test_direct_near_the_axis_matches_oracle():
    """Rings within 1e-6..1e-4 of the axis against rings at distance ~0.1-1: chi - 1 reaches
    ~1e9, so the backward sweep's values grow by ~1e9 per step and must be rescaled before
    they leave the FP32 range; nearly coincident pairs near the axis as well."""
    rng = np.random.default_rng(5)
    w = W.make("paper", ns=300, nf=200, n_modes=18)
    w["src_r"][:60] = 10.0 ** rng.uniform(-6, -4, 60)
    w["tgt_r"][:40] = 10.0 ** rng.uniform(-6, -4, 40)
    w["tgt_z"][:10] = w["src_z"][:10] + 1e-7
    pl = _plan(w, order=6, leaf=32)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.direct_grad(q_re, q_im))
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], grad=True)
    assert all(np.all(np.isfinite(x)) for x in g)
    for c in range(0, 6, 2):
        e = eps_modes(g[c], g[c + 1], D[c], D[c + 1])
        assert e.max() < TOL, (c, e.max())
