"""GPU parity of the adaptive-tree FMM (afmm_options.tree = AFMM_TREE_ADAPTIVE) against the
adaptive oracle (oracle.adaptive, the variant that sums the W and X pairs directly) through
the C ABI.

Both sides build the same tree from the same square (every box of levels 0..1 split, a box
of level >= 2 split while it holds more than leaf_size sources or field points, or, with the
balance factor K, while a same-level neighbour holds more than K leaf_size of either, up to
the maximum level) and apply the same expansions (Sec. 2: moments, shifts, the S2L of
Eq. analysis:s2l over the V lists, local expansions), so they agree to rounding: bar 1e-10
per mode (Eq. results:error) on the FP64 path, 2e-5 for MIXED (its stated FMM bound).  The
tree itself is compared box for box: boxes and leaves per level, the directly summed pairs
and the pairs covered by the S2L lists (together every pair once)."""
import numpy as np
import pytest

import oracle
from oracle import adaptive as A
from paper_2301_01179_gb300 import workloads as W
from tests.gpu_util import eps_modes, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-10
TOL_MIXED = 2e-5


def _plan(w, M, leaf, maxlev, precision="fp64", K=4):
    """GPU plan on the adaptive tree; K: balance factor (0: the rule off)."""
    from paper_2301_01179_gb300 import binding
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    return binding.Plan(sr, sz, tr, tz, w["n_modes"], order=M, leaf_size=leaf, depth=maxlev, precision=precision,
                        tree="adaptive", balance=K if K > 0 else -1)


def _tree(w, leaf, maxlev, K=4):
    return A.AdaptiveTree(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], leaf, max_level=maxlev, refine_to=2,
                          balance=K)


@pytest.mark.parametrize("kind,ns,nf,leaf,maxlev,K", [("cfg5", 6000, 5000, 32, 12, 4), ("cfg5", 6000, 5000, 32, 12, 0),
                                                      ("cfg5", 5000, 6000, 20, 5, 2), ("cfg3", 4000, 4000, 16, 12, 4),
                                                      ("cfg1", 3000, 2000, 40, 12, 4)])
def test_adaptive_tree_matches_oracle_tree(kind, ns, nf, leaf, maxlev, K):
    w = W.make(kind, ns=ns, nf=nf, n_modes=1)
    T = _tree(w, leaf, maxlev, K)
    info = _plan(w, 4, leaf, maxlev, K=K).info()
    assert info["tree"] == "adaptive"
    levels = sorted({b[0] for b in T.boxes})
    assert info["depth"] == max(levels)
    for l in range(2, max(levels) + 1):
        assert info["n_boxes"][l] == sum(1 for b in T.boxes if b[0] == l), l
        assert info["n_leaves"][l] == sum(1 for b in T.leaves if b[0] == l), l
    near = sum(len(T.tgt[B]) * len(A.direct_sources(T, B)) for B in T.leaves)
    s2l = sum(len(T.V[b]) for b in T.boxes if b[0] >= 2)
    assert info["near_pairs"] == near
    assert info["s2l_pairs"] == s2l
    assert info["near_pairs"] + info["s2l_point_pairs"] == ns * nf
    if maxlev == 5:  # the maximum level binds: leaves there hold more than leaf_size points
        assert any(max(len(T.src[b]), len(T.tgt[b])) > leaf for b in T.leaves if b[0] == 5)


@pytest.mark.parametrize("kind,ns,nf,nm,M,leaf,maxlev,K", [
    ("cfg5", 6000, 5000, 9, 8, 32, 12, 4),
    ("cfg5", 6000, 5000, 9, 8, 32, 12, 0),      # without the balance rule
    ("cfg5", 12000, 10000, 33, 12, 64, 12, 4),  # the headline shape: modes 0..32, order 12, leaf 64
    ("cfg5", 5000, 6000, 5, 6, 20, 5, 2),       # leaves held at the maximum level
    ("cfg3", 5000, 4000, 9, 10, 24, 12, 4),     # points on a curve
])
def test_adaptive_fmm_grad_matches_oracle(kind, ns, nf, nm, M, leaf, maxlev, K):
    w = W.make(kind, ns=ns, nf=nf, n_modes=nm)
    T = _tree(w, leaf, maxlev, K)
    assert len({b[0] for b in T.leaves}) >= 3
    pl = _plan(w, M, leaf, maxlev, K=K)
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.grad(q_re, q_im))
    F = A.adaptive_fmm(T, w["q_re"], w["q_im"], M, grad=True, wx="direct")
    for c in (0, 2, 4):
        e = eps_modes(g[c], g[c + 1], F[c], F[c + 1])
        assert e.max() < TOL, (c, e)
    p = to_np(*pl.eval(q_re, q_im))  # the potential-only kernel
    assert eps_modes(p[0], p[1], F[0], F[1]).max() < TOL


def test_adaptive_mixed_matches_oracle():
    w = W.make("cfg5", ns=8000, nf=7000, n_modes=17)
    T = _tree(w, 48, 12)
    pl = _plan(w, 10, 48, 12, precision="mixed")
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.grad(q_re, q_im))
    F = A.adaptive_fmm(T, w["q_re"], w["q_im"], 10, grad=True, wx="direct")
    for c in (0, 2, 4):
        assert eps_modes(g[c], g[c + 1], F[c], F[c + 1]).max() < TOL_MIXED


def test_adaptive_adjoint_matches_oracle():
    w = W.make("cfg5", ns=5000, nf=4000, n_modes=9, with_targets=True)
    T = _tree(w, 24, 12)
    pl = _plan(w, 8, 24, 12)
    rng = np.random.default_rng(11)
    g_re, g_im = rng.standard_normal((2, 9, 4000))
    q_re, q_im, gr, gi = to_dev(w["q_re"], w["q_im"], g_re, g_im)
    a = to_np(*pl.adjoint(q_re, q_im, gr, gi))
    o = A.adaptive_adjoint(T, w["q_re"], w["q_im"], g_re, g_im, 8)
    assert eps_modes(a[0], a[1], o[0], o[1]).max() < TOL
    for k in (2, 3):
        assert np.max(np.abs(a[k] - o[k])) < TOL * np.max(np.abs(o[k]))


def test_adaptive_fewer_near_pairs_than_uniform_on_clustered_points():
    """On cfg5's clustered laws the adaptive tree sums far fewer pairs directly than the
    uniform tree of the occupancy rule, and both cover every pair once."""
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg5", ns=200000, nf=200000, n_modes=1)
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    u = binding.Plan(sr, sz, tr, tz, 1, order=4, leaf_size=64).info()
    a = binding.Plan(sr, sz, tr, tz, 1, order=4, leaf_size=64, tree="adaptive").info()
    for i in (u, a):
        assert i["near_pairs"] + i["s2l_point_pairs"] == 200000 * 200000
    assert a["near_pairs"] < 0.6 * u["near_pairs"], (a["near_pairs"], u["near_pairs"])


def test_adaptive_balance_bounds_near_lists_at_full_size():
    """The 4e6-ring workload's laws at full size: with the balance rule the largest direct
    sum of a leaf stays within (9 K + 8 (d - 2)) leaf_size sources (afmm_plan_info reports
    the largest near list), without it a sparse coarse leaf sums a dense subtree."""
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg5", n_modes=1)
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    n = w["src_r"].size
    for K in (4, 2):
        i = binding.Plan(sr, sz, tr, tz, 1, order=4, leaf_size=64, tree="adaptive", balance=K).info()
        assert i["near_pairs"] + i["s2l_point_pairs"] == n * n
        assert 0 < i["near_max_sources"] <= (9 * K + 8 * (i["depth"] - 2)) * 64, i["near_max_sources"]
    f = binding.Plan(sr, sz, tr, tz, 1, order=4, leaf_size=64, tree="adaptive", balance=-1).info()
    assert f["near_max_sources"] > 10 * (9 * 4 + 8 * (f["depth"] - 2)) * 64


@pytest.mark.parametrize("ns,nf", [(1, 1), (5, 3), (70, 2)])
def test_adaptive_tiny_sets_match_oracle(ns, nf):
    """Few points: the tree stops at level 2 (or a little below)."""
    w = W.make("cfg5", ns=ns, nf=nf, n_modes=5)
    T = _tree(w, 8, 12)
    pl = _plan(w, 6, 8, 12)
    info = pl.info()
    assert info["depth"] == max(b[0] for b in T.boxes)
    assert info["near_pairs"] + info["s2l_point_pairs"] == ns * nf
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.grad(q_re, q_im))
    F = A.adaptive_fmm(T, w["q_re"], w["q_im"], 6, grad=True, wx="direct")
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], grad=True)
    for c in (0, 2, 4):
        assert eps_modes(g[c], g[c + 1], F[c], F[c + 1]).max() < TOL
        if info["s2l_point_pairs"] == 0:  # every pair is direct: the FMM is the direct sum
            assert eps_modes(g[c], g[c + 1], D[c], D[c + 1]).max() < TOL


def test_adaptive_long_near_lists_and_coincident_points():
    """Leaves of up to 200 points with the balance rule give near lists of several thousand
    sources over many ranges (past the kernel's staged source list, so each producer finds
    its source by a binary search over the ranges); a cluster of coincident points holds
    leaves at the maximum level with more than leaf_size points."""
    w = W.make("cfg5", ns=9000, nf=7000, n_modes=9)
    for k in ("src", "tgt"):  # 400 points of each role on one spot
        w[k + "_r"][:400] = 0.3
        w[k + "_z"][:400] = 0.1
    leaf, maxlev = 200, 9
    T = _tree(w, leaf, maxlev)
    assert any(len(T.src[b]) > leaf for b in T.leaves if b[0] == maxlev)
    pl = _plan(w, 8, leaf, maxlev)
    info = pl.info()
    assert info["near_max_sources"] > 1024
    assert info["near_pairs"] + info["s2l_point_pairs"] == 9000 * 7000
    q_re, q_im = to_dev(w["q_re"], w["q_im"])
    g = to_np(*pl.grad(q_re, q_im))
    F = A.adaptive_fmm(T, w["q_re"], w["q_im"], 8, grad=True, wx="direct")
    for c in (0, 2, 4):
        assert eps_modes(g[c], g[c + 1], F[c], F[c + 1]).max() < TOL
