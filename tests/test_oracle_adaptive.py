"""The adaptive-quadtree FMM of the oracle (oracle.adaptive), pinned on the CPU:

- on a tree refined uniformly to depth d its lists reduce to the uniform method's (U: the
  3 x 3 neighbour leaves, V: the S2L list, W = X = {}), so it must reproduce the uniform
  oracle FMM (Algorithm 1) to rounding;
- the four lists must account for every (field leaf, source leaf) pair exactly once (a
  combinatorial check, independent of the expansions);
- on clustered points (leaves on several levels, W and X lists in use) it must converge
  to the direct sum as the order M grows, potential and field gradient;
- the variant that sums the point pairs of W and X directly (wx="direct", the form the GPU
  plans take) must sum, at every field point, each source exactly once: directly or through
  the V lists of the boxes that contain the point's leaf; it converges to the direct sum
  like the expansion variant, and the two agree within their truncation errors."""
import numpy as np
import pytest

import oracle
from oracle import adaptive as A
from paper_2301_01179_gb300 import workloads as W


def _eps(F, D, c):
    a = F[c] + 1j * F[c + 1]
    b = D[c] + 1j * D[c + 1]
    return float((np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)).max())


def test_uniform_refinement_reproduces_uniform_fmm():
    w = W.make("cfg1", ns=900, nf=700, n_modes=4)
    sr, sz, tr, tz = w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"]
    d, geom = oracle.tree_setup(sr, sz, tr, tz, 32, depth_override=4)
    tree = A.AdaptiveTree(sr, sz, tr, tz, 10 ** 9, refine_to=d, geom=geom)
    assert {b[0] for b in tree.leaves} == {d}
    assert not any(tree.W.values()) and not any(tree.X.values())
    F = A.adaptive_fmm(tree, w["q_re"], w["q_im"], 6, grad=True)
    U = oracle.fmm(sr, sz, tr, tz, w["q_re"], w["q_im"], 6, d, geom, grad=True)
    for c in (0, 2, 4):
        assert _eps(F, U, c) < 1e-12


def _ancestors(tree, b):
    out = []
    while b is not None:
        out.append(b)
        b = tree.parent[b]
    return out


def test_lists_cover_every_leaf_pair_once():
    w = W.make("cfg5", ns=1500, nf=1100, n_modes=1)
    tree = A.AdaptiveTree(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 20)
    assert len({b[0] for b in tree.leaves}) >= 3
    assert sum(len(v) for v in tree.W.values()) > 0
    for B in tree.leaves:
        upB = _ancestors(tree, B)
        for C in tree.leaves:
            upC = set(_ancestors(tree, C))
            n = int(C in tree.U[B])
            n += sum(1 for Wc in tree.W[B] if Wc in upC)
            n += sum(1 for D in upB for Vc in tree.V[D] if Vc in upC)
            n += sum(1 for D in upB if C in tree.X[D])
            assert n == 1, (B, C, n)


def test_converges_to_direct_on_clustered_points():
    w = W.make("cfg5", ns=1200, nf=900, n_modes=4)
    sr, sz, tr, tz = w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"]
    tree = A.AdaptiveTree(sr, sz, tr, tz, 24)
    assert len({b[0] for b in tree.leaves}) >= 3
    assert sum(len(v) for v in tree.W.values()) > 0 and sum(len(v) for v in tree.X.values()) > 0
    D = oracle.direct(sr, sz, tr, tz, w["q_re"], w["q_im"], grad=True)
    errs = []
    for M in (4, 7, 10):
        F = A.adaptive_fmm(tree, w["q_re"], w["q_im"], M, grad=True)
        errs.append([_eps(F, D, c) for c in (0, 2, 4)])
    errs = np.array(errs)
    assert np.all(errs[1:] < 0.2 * errs[:-1]), errs  # geometric in M
    assert errs[-1].max() < 1e-5, errs


def test_fast_lists_match_their_definitions():
    w = W.make("cfg5", ns=2000, nf=1500, n_modes=1)
    tree = A.AdaptiveTree(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 16)
    U, V, Wl, X = tree.lists_brute()
    assert {b: sorted(v) for b, v in tree.U.items()} == U
    assert {b: sorted(v) for b, v in tree.V.items()} == {b: sorted(v) for b, v in V.items()}
    assert {b: sorted(v) for b, v in tree.W.items()} == Wl
    assert {b: sorted(v) for b, v in tree.X.items()} == {b: sorted(v) for b, v in X.items()}


def test_wx_direct_sources_and_v_lists_partition_the_sources():
    w = W.make("cfg5", ns=1800, nf=1300, n_modes=1)
    tree = A.AdaptiveTree(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 20, refine_to=2)
    assert len({b[0] for b in tree.leaves}) >= 3
    assert sum(len(v) for v in tree.W.values()) > 0 and sum(len(v) for v in tree.X.values()) > 0
    ns = w["src_r"].size
    for B in tree.leaves:
        if len(tree.tgt[B]) == 0:
            continue
        cnt = np.bincount(A.direct_sources(tree, B), minlength=ns)
        for D in _ancestors(tree, B):
            for c in tree.V[D]:
                cnt += np.bincount(tree.src[c], minlength=ns)
        assert cnt.min() == 1 and cnt.max() == 1, (B, cnt.min(), cnt.max())


def test_wx_direct_converges_and_agrees_with_expansions():
    w = W.make("cfg5", ns=1200, nf=900, n_modes=4)
    sr, sz, tr, tz = w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"]
    tree = A.AdaptiveTree(sr, sz, tr, tz, 24, refine_to=2)
    assert sum(len(v) for v in tree.W.values()) > 0 and sum(len(v) for v in tree.X.values()) > 0
    D = oracle.direct(sr, sz, tr, tz, w["q_re"], w["q_im"], grad=True)
    errs = []
    for M in (4, 7, 10):
        F = A.adaptive_fmm(tree, w["q_re"], w["q_im"], M, grad=True, wx="direct")
        E = A.adaptive_fmm(tree, w["q_re"], w["q_im"], M, grad=True)
        e_d = [_eps(F, D, c) for c in (0, 2, 4)]
        e_e = [_eps(E, D, c) for c in (0, 2, 4)]
        errs.append(e_d)
        for c, k in zip((0, 2, 4), range(3)):
            assert _eps(F, E, c) <= 1.01 * (e_d[k] + e_e[k]) + 1e-14
    errs = np.array(errs)
    assert np.all(errs[1:] < 0.2 * errs[:-1]), errs
    assert errs[-1].max() < 1e-5, errs


def test_wx_direct_on_a_uniform_tree_is_the_uniform_fmm():
    w = W.make("cfg1", ns=700, nf=600, n_modes=3)
    sr, sz, tr, tz = w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"]
    d, geom = oracle.tree_setup(sr, sz, tr, tz, 32, depth_override=4)
    tree = A.AdaptiveTree(sr, sz, tr, tz, 10 ** 9, refine_to=d, geom=geom)
    F = A.adaptive_fmm(tree, w["q_re"], w["q_im"], 6, grad=True, wx="direct")
    U = oracle.fmm(sr, sz, tr, tz, w["q_re"], w["q_im"], 6, d, geom, grad=True)
    for c in (0, 2, 4):
        assert _eps(F, U, c) < 1e-12


def test_adaptive_adjoint_on_a_uniform_tree_is_the_uniform_adjoint():
    w = W.make("cfg4", ns=600, nf=500, n_modes=3, with_targets=True)
    sr, sz, tr, tz = w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"]
    d, geom = oracle.tree_setup(sr, sz, tr, tz, 32, depth_override=4)
    tree = A.AdaptiveTree(sr, sz, tr, tz, 10 ** 9, refine_to=d, geom=geom)
    rng = np.random.default_rng(5)
    g_re, g_im = rng.standard_normal((2, 3, tr.size))
    a = A.adaptive_adjoint(tree, w["q_re"], w["q_im"], g_re, g_im, 6)
    u = oracle.adjoint_fmm(sr, sz, tr, tz, w["q_re"], w["q_im"], g_re, g_im, 6, d, geom)
    assert _eps(a, u, 0) < 1e-12
    for k in (2, 3):
        assert np.max(np.abs(a[k] - u[k])) < 1e-12 * np.max(np.abs(u[k]))


def test_adaptive_adjoint_matches_the_direct_adjoint():
    w = W.make("cfg5", ns=900, nf=700, n_modes=3)
    sr, sz, tr, tz = w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"]
    tree = A.AdaptiveTree(sr, sz, tr, tz, 20, refine_to=2)
    assert len({b[0] for b in tree.leaves}) >= 3
    rng = np.random.default_rng(6)
    g_re, g_im = rng.standard_normal((2, 3, tr.size))
    a = A.adaptive_adjoint(tree, w["q_re"], w["q_im"], g_re, g_im, 10)
    u = oracle.adjoint_direct(sr, sz, tr, tz, w["q_re"], w["q_im"], g_re, g_im)
    assert _eps(a, u, 0) < 1e-5
    for k in (2, 3):
        assert np.max(np.abs(a[k] - u[k])) < 1e-5 * np.max(np.abs(u[k]))


@pytest.mark.parametrize("K", [2, 4])
def test_balanced_tree_lists_partition_and_bound_the_direct_sums(K):
    """With the balance rule every leaf's directly summed sources are bounded by
    (9 K + 8 (l - 2)) leaf_size, and the lists still cover every pair exactly once."""
    w = W.make("cfg5", ns=2500, nf=2000, n_modes=1)
    leaf = 12
    tree = A.AdaptiveTree(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], leaf, refine_to=2, balance=K)
    free = A.AdaptiveTree(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], leaf, refine_to=2)
    assert len(tree.boxes) > len(free.boxes)
    ns = w["src_r"].size
    worst_free = max(len(A.direct_sources(free, B)) for B in free.leaves)
    for B in tree.leaves:
        s = A.direct_sources(tree, B)
        assert len(s) <= (9 * K + 8 * (B[0] - 2)) * leaf, (B, len(s))
        cnt = np.bincount(s, minlength=ns)
        for D in _ancestors(tree, B):
            for c in tree.V[D]:
                cnt += np.bincount(tree.src[c], minlength=ns)
        assert cnt.min() == 1 and cnt.max() == 1
    worst = max(len(A.direct_sources(tree, B)) for B in tree.leaves)
    assert worst_free > 5 * worst  # the rule is what bounds them
    T = A.transposed(tree)
    assert T.boxes == tree.boxes and all(T.V[b] == tree.V[b] for b in tree.boxes)


def test_balanced_tree_converges_to_direct():
    w = W.make("cfg5", ns=1200, nf=900, n_modes=3)
    sr, sz, tr, tz = w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"]
    tree = A.AdaptiveTree(sr, sz, tr, tz, 16, refine_to=2, balance=4)
    D = oracle.direct(sr, sz, tr, tz, w["q_re"], w["q_im"], grad=True)
    errs = []
    for M in (4, 7, 10):
        F = A.adaptive_fmm(tree, w["q_re"], w["q_im"], M, grad=True, wx="direct")
        errs.append([_eps(F, D, c) for c in (0, 2, 4)])
    errs = np.array(errs)
    assert np.all(errs[1:] < 0.2 * errs[:-1]), errs
    assert errs[-1].max() < 1e-5, errs
