"""Pins for the oracle's direct sum, tree, FMM (Algorithm 1) and adjoints.

The FMM has no printed numbers to match, so it is pinned by convergence to the direct
sum as the order M grows (Sec. 4: error falling roughly like C^(-0.4 M)), by the paper's
accuracy statement on its own test case (ten digits at the highest orders), and by
identities: the S2L lists are complete exactly when the error vanishes with M.
The adjoint is pinned by finite differences of the direct sum.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2301_01179_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _eps(a_re, a_im, b_re, b_im):
    """Eq. results:error per mode, complex modulus."""
    a = a_re + 1j * a_im
    b = b_re + 1j * b_im
    return np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)


def test_direct_matches_pairwise_green():
    w = W.make("cfg1", ns=40, nf=30)
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    N = w["n_modes"] - 1
    ref_re = np.zeros((N + 1, 30))
    ref_im = np.zeros((N + 1, 30))
    for j in range(30):
        for i in range(40):
            G = oracle.green(w["tgt_r"][j], w["src_r"][i], w["tgt_z"][j] - w["src_z"][i], N)
            ref_re[:, j] += w["q_re"][:, i] * G
            ref_im[:, j] += w["q_im"][:, i] * G
    np.testing.assert_allclose(D[0], ref_re, rtol=1e-12, atol=1e-14 * np.abs(ref_re).max())
    np.testing.assert_allclose(D[1], ref_im, rtol=1e-12, atol=1e-14 * np.abs(ref_im).max())


def test_direct_is_linear_and_threads_agree():
    w = W.make("cfg1", ns=300, nf=200)
    a = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], threads=1)
    b = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], threads=4)
    np.testing.assert_array_equal(a[0], b[0])
    c = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 2 * w["q_re"] - w["q_im"],
                      w["q_im"] + w["q_re"])
    np.testing.assert_allclose(c[0], 2 * a[0] - a[1], rtol=1e-12, atol=1e-13 * np.abs(a[0]).max())


def test_tree_depth_rule():
    # 4 x 4 grid of sources at cell centres of the unit square: depth 2 has 16 non-empty
    # leaves with one source each; leaf size 1 must give d = 2, leaf size 0.5 forces deeper.
    g = (np.arange(4) + 0.5) / 4
    r, z = np.meshgrid(g + 1.0, g, indexing="ij")
    r = r.ravel()
    z = z.ravel()
    d, geom = oracle.tree_setup(r, z, r, z, 1)
    assert d == 2
    np.testing.assert_allclose(geom, [1.125, 0.125, 0.75])
    # 8 coincident copies per site can never be split below 8 per leaf: the rule runs to
    # its cap of 16 levels
    d8, _ = oracle.tree_setup(np.repeat(r, 8), np.repeat(z, 8), r, z, 4)
    assert d8 == 16
    d8, _ = oracle.tree_setup(np.repeat(r, 8), np.repeat(z, 8), r, z, 8)
    assert d8 == 2
    # uniform random: mean occupancy rule
    w = W.make("cfg1")
    d, _ = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["leaf"])
    assert d == 4


def test_fmm_converges_to_direct_cfg1():
    w = W.make("cfg1")
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    d, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["leaf"])
    errs = []
    for M in (4, 6, 8):
        F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], M, d, geom)
        errs.append(_eps(F[0], F[1], D[0], D[1]).max())
    # roughly geometric decay in M (Sec. 4); a missing or doubled S2L pair would stall it
    assert errs[0] < 5e-3 and errs[2] < 5e-5
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3


def test_fmm_paper_workload_ten_digits():
    # the paper's test case (Sec. 4): uniform unit square, real 0 < S < 1, modes 0..17;
    # ten-digit accuracy for n = 0 at the highest order M = 16
    digits = GOLD["fmm_accuracy_digits"]["value"]
    M = max(GOLD["test_orders"]["value"])
    w = W.make("paper", ns=2048, nf=2048)
    assert w["n_modes"] - 1 == GOLD["test_modes_max"]["value"]
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    d, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["leaf"])
    F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], M, d, geom)
    e = _eps(F[0], F[1], D[0], D[1])
    assert e[0] < 10.0 ** (-digits + 0.5)
    assert e.max() < 1e-7


def test_fmm_gradient_converges():
    w = W.make("cfg1", ns=1500, nf=700)
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], grad=True)
    d, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 32)
    F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], 8, d, geom, grad=True)
    assert _eps(F[0], F[1], D[0], D[1]).max() < 1e-4
    assert _eps(F[2], F[3], D[2], D[3]).max() < 1e-3
    assert _eps(F[4], F[5], D[4], D[5]).max() < 1e-3


def test_direct_gradient_vs_finite_difference():
    w = W.make("cfg1", ns=50, nf=5)
    h = 1e-6
    D = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], grad=True)
    P = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"] + h, w["tgt_z"], w["q_re"], w["q_im"])
    Mn = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"] - h, w["tgt_z"], w["q_re"], w["q_im"])
    np.testing.assert_allclose((P[0] - Mn[0]) / (2 * h), D[2], rtol=1e-6, atol=1e-6 * np.abs(D[2]).max())
    P = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"] + h, w["q_re"], w["q_im"])
    Mn = oracle.direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"] - h, w["q_re"], w["q_im"])
    np.testing.assert_allclose((P[1] - Mn[1]) / (2 * h), D[5], rtol=1e-6, atol=1e-6 * np.abs(D[5]).max())


def _loss_terms(w, sr, sz):
    D = oracle.direct(sr, sz, w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"])
    return D[0] - w["T_re"], D[1] - w["T_im"]


def test_adjoint_direct_vs_finite_difference():
    # L = sum_n,j |Phi - T|^2; gradient w.r.t. q (complex), r_i, z_i by central differences
    # (h = 1e-6) on a few sources, evaluated incrementally to avoid cancellation
    w = W.make("cfg4", ns=120, nf=90, n_modes=7, with_targets=True)
    Er, Ei = _loss_terms(w, w["src_r"], w["src_z"])
    gq_re, gq_im, g_r, g_z = oracle.adjoint_direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"],
                                                   w["q_re"], w["q_im"], 2 * Er, 2 * Ei)
    N = w["n_modes"] - 1
    h = 1e-6
    for i in (0, 17, 63, 119):
        for which, g in (("r", g_r), ("z", g_z)):
            dl = []
            for s in (+1, -1):
                r = w["src_r"][i] + (s * h if which == "r" else 0.0)
                z = w["src_z"][i] + (s * h if which == "z" else 0.0)
                dphi_re = np.zeros_like(Er)
                dphi_im = np.zeros_like(Er)
                for j in range(len(w["tgt_r"])):
                    G1 = oracle.green(w["tgt_r"][j], r, w["tgt_z"][j] - z, N)
                    G0 = oracle.green(w["tgt_r"][j], w["src_r"][i], w["tgt_z"][j] - w["src_z"][i], N)
                    dphi_re[:, j] = w["q_re"][:, i] * (G1 - G0)
                    dphi_im[:, j] = w["q_im"][:, i] * (G1 - G0)
                dl.append(np.sum(2 * (Er * dphi_re + Ei * dphi_im) + dphi_re ** 2 + dphi_im ** 2))
            fd = (dl[0] - dl[1]) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, which, fd, g[i])
        # q: L is quadratic in q, so the central difference is exact up to rounding
        for n in (0, N):
            G = np.array([oracle.green(w["tgt_r"][j], w["src_r"][i], w["tgt_z"][j] - w["src_z"][i], N)[n]
                          for j in range(len(w["tgt_r"]))])
            fd_re = np.sum(2 * Er[n] * G)
            fd_im = np.sum(2 * Ei[n] * G)
            assert abs(fd_re - gq_re[n, i]) < 1e-12 * max(1, abs(fd_re))
            assert abs(fd_im - gq_im[n, i]) < 1e-12 * max(1, abs(fd_im))


def test_adjoint_fmm_matches_adjoint_direct():
    w = W.make("cfg4", ns=1200, nf=1000, n_modes=5, with_targets=True)
    d, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 32)
    gp_re, gp_im = w["T_re"], w["T_im"]
    A = oracle.adjoint_direct(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], gp_re, gp_im)
    B = oracle.adjoint_fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], gp_re, gp_im,
                           10, d, geom)
    assert _eps(B[0], B[1], A[0], A[1]).max() < 1e-5
    assert np.max(np.abs(B[2] - A[2])) / np.max(np.abs(A[2])) < 1e-4
    assert np.max(np.abs(B[3] - A[3])) / np.max(np.abs(A[3])) < 1e-4


@pytest.mark.parametrize("kind,ns,nf,nm,M,d", [("cfg1", 2000, 1500, 17, 8, 4), ("cfg3", 4000, 3000, 9, 6, 5),
                                                ("cfg5", 3000, 2500, 9, 6, 6), ("cfg2", 6000, 6000, 5, 12, 5)])
def test_fmm_sampled_equals_full_fmm(kind, ns, nf, nm, M, d):
    """The sampled oracle (each level's S2L evaluated at the point, shifts skipped as exact
    re-expansions) must give the full Algorithm-1 oracle's field and gradient at the
    sampled points to rounding; a dropped level, a wrong orientation or a list slot
    missing would show at 1e-3..1e-8, far above this bar."""
    w = W.make(kind, ns=ns, nf=nf, n_modes=nm)
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=d)
    F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], M, d, geom, grad=True)
    idx = W.subset(nf, 37, seed=9)
    S = oracle.fmm_sampled(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], M, d, geom, idx,
                           grad=True)
    for c in range(0, 6, 2):
        assert _eps(S[c], S[c + 1], F[c][:, idx], F[c + 1][:, idx]).max() < 1e-12, c
    P = oracle.fmm_sampled(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], M, d, geom, idx)
    np.testing.assert_array_equal(P[0], S[0])


def test_adjoint_fmm_sampled_equals_full_adjoint():
    w = W.make("cfg4", ns=1500, nf=1200, n_modes=7, with_targets=True)
    d = 5
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=d)
    A = oracle.adjoint_fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], w["T_re"], w["T_im"],
                           8, d, geom)
    idx = W.subset(1500, 29, seed=4)
    S = oracle.adjoint_fmm_sampled(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], w["q_re"], w["q_im"], w["T_re"],
                                   w["T_im"], 8, d, geom, idx)
    assert _eps(S[0], S[1], A[0][:, idx], A[1][:, idx]).max() < 1e-12
    for c in (2, 3):
        np.testing.assert_allclose(S[c], A[c][idx], rtol=0, atol=1e-12 * np.abs(A[c]).max())


def _box(v, v0, L, l):
    return np.clip(np.floor((v - v0) * (2 ** l) / L), 0, 2 ** l - 1).astype(np.int64)


@pytest.mark.parametrize("kind,n,d", [("cfg1", 300, 4), ("cfg5", 400, 5), ("cfg3", 350, 5)])
def test_tree_counts_by_brute_force(kind, n, d):
    """Tree counts against a pair-by-pair classification from the definitions of Sec. 2.2:
    a pair is near when its leaves are 3x3 neighbours, else it belongs to the one level l
    where its boxes are not neighbours but their parents are; box pairs count each
    (field box, source box) of a list once when both boxes hold a point."""
    w = W.make(kind, ns=n, nf=n - 50, n_modes=1)
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=d)
    near, box_pairs, far = oracle.tree_counts(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], d, geom)
    r0, z0, L = geom
    near_bf = 0
    levels_hit = np.zeros(d + 1, dtype=np.int64)
    for j in range(w["tgt_r"].size):
        for i in range(n):
            hit = 0
            for l in range(2, d + 1):
                a = [_box(w["tgt_r"][j], r0, L, l), _box(w["tgt_z"][j], z0, L, l)]
                b = [_box(w["src_r"][i], r0, L, l), _box(w["src_z"][i], z0, L, l)]
                nbr = max(abs(a[0] - b[0]), abs(a[1] - b[1])) <= 1
                pnbr = max(abs(a[0] // 2 - b[0] // 2), abs(a[1] // 2 - b[1] // 2)) <= 1
                if not nbr and pnbr:
                    hit += 1
                    levels_hit[l] += 1
                if l == d and nbr:
                    near_bf += 1
                    hit += 1
            assert hit == 1
    assert near == near_bf
    assert near + far == n * (n - 50)
    assert far == int(levels_hit.sum())
    # box pairs: occupied boxes per level, list membership by the same rule
    bp = 0
    for l in range(2, d + 1):
        occ = set(zip(_box(w["src_r"], r0, L, l), _box(w["src_z"], z0, L, l))) | \
            set(zip(_box(w["tgt_r"], r0, L, l), _box(w["tgt_z"], z0, L, l)))
        for (ti, tj) in occ:
            for (ui, uj) in occ:
                nbr = max(abs(ti - ui), abs(tj - uj)) <= 1
                pnbr = max(abs(ti // 2 - ui // 2), abs(tj // 2 - uj // 2)) <= 1
                bp += (not nbr) and pnbr
    assert box_pairs == bp
