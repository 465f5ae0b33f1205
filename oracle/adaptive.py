"""Adaptive-quadtree FMM in FP64: the uniform method's expansions (Sec. 2) on a tree refined
only where the points are dense.

TEST INFRASTRUCTURE ONLY (as the rest of ``oracle``): imported by the test suite.  It shares
no code with the CUDA library.

The paper's tree is uniform (Sec. 4).  On strongly clustered points a uniform depth either
leaves dense leaves (many near pairs) or creates many boxes elsewhere (many S2L pairs).  This
module keeps every expansion of the uniform method and changes only the tree and the
bookkeeping, in the standard adaptive-FMM form: boxes are split while they hold more than
``leaf_size`` sources or field points, and for a leaf B

  U(B)  leaves adjacent to B (B included):                 direct sums (Eq. analysis:sum);
  V(B)  same-level boxes not adjacent to B whose parent is adjacent to B's parent:
        source-to-local of their moments (Eq. analysis:s2l), for every box B;
  W(B)  finer boxes not adjacent to B whose parent is adjacent to B: their moments
        evaluated at B's field points (the source-to-local with a field "box" of one point);
  X(B)  coarser leaves C with B in W(C): C's sources into B's local expansion (the
        source-to-local with a source "box" of one point), for every box B.

Every interaction is one generalised source-to-local between a source centre (r1, z1) with
moments S_ij (Eq. analysis:moments, no factorials) and a field centre (r, z):

  F_kl = sum_ij s(j, l) C(j + l, j) gbar_{k, i, j + l} S_ij,

with gbar the Taylor coefficients of G about (max(r, r1), min(r, r1), |z - z1|) (Appendix A),
the radial indices swapped when the field centre has the smaller radius (G(r, r1, x) =
G(r1, r, x)), s(j, l) = (-1)^j for z >= z1 and (-1)^l below (G is even in x).  The moments
and locals shift between parent and child as in Eqs. analysis:shift and analysis:l2l.
"""
import numpy as np

from . import _f64, direct, gbar, tree_setup


def _box_coord(v, v0, L, level):
    """Box index of coordinate v at a level, clamped to the square (as the uniform tree)."""
    s = float(1 << level) / L
    i = np.floor((v - v0) * s).astype(np.int64)
    return np.clip(i, 0, (1 << level) - 1)


def _cidx(M):
    """(i, j) of the coefficients i + j <= M in storage order (row i holds M + 1 - i)."""
    I, J = [], []
    for i in range(M + 1):
        for j in range(M + 1 - i):
            I.append(i)
            J.append(j)
    return np.array(I), np.array(J)


def _binom(n, k):
    from math import comb
    return float(comb(n, k))


class AdaptiveTree:
    """Boxes keyed by (level, ir, iz); each box holds the indices of its sources and field
    points.  ``refine_to`` forces every non-empty box to split down to that level (with a
    large ``leaf_size`` this reproduces the uniform tree of that depth).

    ``balance`` = K > 0 also splits a box (below the maximum level) when one of its
    same-level neighbours holds more than K leaf_size sources or field points.  A leaf then
    sums directly at most the points of 9 boxes of its level, each holding at most
    K leaf_size, plus at most 8 coarser leaves per level: without it a sparse coarse leaf
    touching a dense box would sum that box's whole subtree directly.  The tree is built
    level by level, since the rule looks at a box's neighbours."""

    def __init__(self, src_r, src_z, tgt_r, tgt_z, leaf_size, max_level=12, refine_to=0, geom=None, balance=0):
        self.sr, self.sz, self.tr, self.tz = map(_f64, (src_r, src_z, tgt_r, tgt_z))
        if geom is None:
            geom = tree_setup(self.sr, self.sz, self.tr, self.tz, max(1, int(leaf_size)))[1]
        self.r0, self.z0, self.L = (float(g) for g in geom)
        self.leaf_size = int(leaf_size)
        self.max_level = int(max_level)
        self.refine_to = int(refine_to)
        self.balance = int(balance)
        self.src, self.tgt, self.children, self.parent = {}, {}, {}, {}
        root = (0, 0, 0)
        self.src[root] = np.arange(self.sr.shape[0])
        self.tgt[root] = np.arange(self.tr.shape[0])
        self.parent[root] = None
        level = [root]
        while level:
            nxt = []
            for b in level:
                lvl = b[0]
                s, t = self.src[b], self.tgt[b]
                split = lvl < self.refine_to or len(s) > self.leaf_size or len(t) > self.leaf_size
                if not split and self.balance > 0:
                    lim = self.balance * self.leaf_size
                    for di in (-1, 0, 1):
                        for dj in (-1, 0, 1):
                            c = (lvl, b[1] + di, b[2] + dj)
                            if c != b and c in self.src and (len(self.src[c]) > lim or len(self.tgt[c]) > lim):
                                split = True
                if not split or lvl >= self.max_level:
                    self.children[b] = []
                    continue
                kids = []
                si = _box_coord(self.sr[s], self.r0, self.L, lvl + 1)
                sj = _box_coord(self.sz[s], self.z0, self.L, lvl + 1)
                ti = _box_coord(self.tr[t], self.r0, self.L, lvl + 1)
                tj = _box_coord(self.tz[t], self.z0, self.L, lvl + 1)
                for a in (0, 1):
                    for c in (0, 1):
                        ir, iz = 2 * b[1] + a, 2 * b[2] + c
                        cs = s[(si == ir) & (sj == iz)]
                        ct = t[(ti == ir) & (tj == iz)]
                        if len(cs) == 0 and len(ct) == 0:
                            continue
                        k = (lvl + 1, ir, iz)
                        self.src[k], self.tgt[k], self.parent[k] = cs, ct, b
                        kids.append(k)
                        nxt.append(k)
                self.children[b] = kids
            level = nxt
        self.boxes = sorted(self.src)
        self.leaves = [b for b in self.boxes if not self.children[b]]
        self._lists()

    def centre(self, b):
        h = self.L / (1 << b[0])
        return self.r0 + (b[1] + 0.5) * h, self.z0 + (b[2] + 0.5) * h

    @staticmethod
    def adjacent(a, b):
        """Closed squares touch or overlap (tree boxes are nested or disjoint)."""
        lf = max(a[0], b[0])
        sa, sb = 1 << (lf - a[0]), 1 << (lf - b[0])
        a0i, a1i, a0j, a1j = a[1] * sa, (a[1] + 1) * sa, a[2] * sa, (a[2] + 1) * sa
        b0i, b1i, b0j, b1j = b[1] * sb, (b[1] + 1) * sb, b[2] * sb, (b[2] + 1) * sb
        return a0i <= b1i and b0i <= a1i and a0j <= b1j and b0j <= a1j

    def _lists(self):
        """U, V, W, X from each box's colleagues (same-level adjacent boxes), O(boxes)."""
        adj, box = self.adjacent, self.src
        self.V, self.U, self.W = {}, {}, {}
        self.X = {b: [] for b in self.boxes}

        def colleagues(b):
            out = []
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    c = (b[0], b[1] + di, b[2] + dj)
                    if c in box:
                        out.append(c)
            return out

        for b in self.boxes:
            pb = self.parent[b]
            if b[0] < 2 or pb is None:
                self.V[b] = []
                continue
            self.V[b] = [d for c in colleagues(pb) for d in self.children[c] if not adj(d, b)]
        for b in self.leaves:
            U, W = set(), []
            stack = list(colleagues(b))
            while stack:  # same level and finer: descend while adjacent
                c = stack.pop()
                if not self.children[c]:
                    U.add(c)
                    continue
                for d in self.children[c]:
                    if adj(d, b):
                        stack.append(d)
                    else:
                        W.append(d)
            for lc in range(b[0] - 1, -1, -1):  # coarser adjacent leaves
                sh = b[0] - lc
                for di in (-1, 0, 1):
                    for dj in (-1, 0, 1):
                        c = (lc, (b[1] + di) >> sh, (b[2] + dj) >> sh)
                        if c in box and not self.children[c] and adj(c, b):
                            U.add(c)
            self.U[b] = sorted(U)
            self.W[b] = sorted(W)
            for c in self.W[b]:
                self.X[c].append(b)

    def lists_brute(self):
        """The same lists from their definitions by exhaustive search (for checking)."""
        adj = self.adjacent
        V = {b: ([c for c in self.boxes if c[0] == b[0] and c != b and not adj(c, b)
                  and adj(self.parent[c], self.parent[b])] if b[0] >= 2 else []) for b in self.boxes}
        U = {b: sorted(c for c in self.leaves if adj(c, b)) for b in self.leaves}
        W = {b: sorted(c for c in self.boxes if c[0] > b[0] and not adj(c, b) and adj(self.parent[c], b))
             for b in self.leaves}
        X = {b: [] for b in self.boxes}
        for b in self.leaves:
            for c in W[b]:
                X[c].append(b)
        return U, V, W, X


_S2L_TABLES = {}


def _s2l_tables(Mf, Ms):
    """Index and weight tables of the generalised source-to-local (cached per orders)."""
    key = (Mf, Ms)
    if key not in _S2L_TABLES:
        K, Lf = _cidx(Mf)
        I, J = _cidx(Ms)
        jl = J[None, :] + Lf[:, None]
        binom = np.array([[_binom(jl[a, b], J[b]) for b in range(len(J))] for a in range(len(K))])
        s_up = np.where(J[None, :] % 2 == 1, -1.0, 1.0) * np.ones_like(binom)    # z >= z1: (-1)^j
        s_down = np.where(Lf[:, None] % 2 == 1, -1.0, 1.0) * np.ones_like(binom)  # z < z1: (-1)^l
        _S2L_TABLES[key] = (K, Lf, I, jl, binom * s_up, binom * s_down)
    return _S2L_TABLES[key]


def _s2l_matrix(rf, zf, rs, zs, N, Mf, Ms):
    """The generalised source-to-local from moments of total degree <= Ms about (rs, zs) to
    local coefficients of total degree <= Mf about (rf, zf): T[n, kl, ij]."""
    K, Lf, I, jl, w_up, w_down = _s2l_tables(Mf, Ms)
    x = zf - zs
    E = gbar(max(rf, rs), min(rf, rs), abs(x), N, Mf + Ms)
    if rf < rs:  # field centre at the smaller radius: the radial indices swap
        g = E[:, I[None, :], K[:, None], jl]
    else:
        g = E[:, K[:, None], I[None, :], jl]
    return g * (w_down if x < 0 else w_up)[None, :, :]


def _moments(sr, sz, q, rc, zc, M):
    """S_ij = sum q (r' - rc)^i (z' - zc)^j (Eq. analysis:moments): [nmodes, nc]."""
    I, J = _cidx(M)
    w = (sr[:, None] - rc) ** I[None, :] * (sz[:, None] - zc) ** J[None, :]
    return q @ w


def _shift_up(S, D, M):
    """Moments about a child centre -> about the parent centre (Eq. analysis:shift);
    D = parent centre - child centre."""
    I, J = _cidx(M)
    idx = {(i, j): c for c, (i, j) in enumerate(zip(I, J))}
    A = np.zeros((len(I), len(I)))
    for p, (i, j) in enumerate(zip(I, J)):
        for qq in range(i + 1):
            for u in range(j + 1):
                A[p, idx[(i - qq, j - u)]] += _binom(i, qq) * _binom(j, u) * (-D[0]) ** qq * (-D[1]) ** u
    return S @ A.T


def _shift_down(F, D, M):
    """Locals about a parent centre -> about a child centre (Eq. analysis:l2l);
    D = parent centre - child centre."""
    I, J = _cidx(M)
    idx = {(i, j): c for c, (i, j) in enumerate(zip(I, J))}
    A = np.zeros((len(I), len(I)))
    for p, (i, j) in enumerate(zip(I, J)):
        for qq in range(M + 1 - i):
            for u in range(M + 1 - i - j - qq):
                A[p, idx[(i + qq, j + u)]] += _binom(i + qq, qq) * _binom(j + u, u) * (-D[0]) ** qq * (-D[1]) ** u
    return F @ A.T


def direct_sources(tree, B):
    """Sources that the W / X-as-direct variant of :func:`adaptive_fmm` sums directly at the
    field points of leaf B: the sources of U(B), of the subtrees of W(B), and of the leaves
    in X(b) for every b that contains B (B itself included).  These are exactly the pairs
    that the expansion variant takes through W and X, so the far field (V lists and the
    shifts) is the same in both variants."""
    boxes = list(tree.U[B]) + list(tree.W[B])
    b = B
    while b is not None:
        boxes += tree.X[b]
        b = tree.parent[b]
    if not boxes:
        return np.zeros(0, np.int64)
    return np.concatenate([tree.src[c] for c in boxes])


def adaptive_fmm(tree, q_re, q_im, M, grad=False, wx="expansion"):
    """The FMM on an :class:`AdaptiveTree`.  Returns (phi_re, phi_im[, dr_re, dr_im, dz_re,
    dz_im]), each [nmodes, nf], in the caller's point order.

    wx = "expansion": W and X through the generalised source-to-local (the standard
    adaptive FMM).  wx = "direct": the point pairs of W and X summed directly (Eq.
    analysis:sum) with the U list, as :func:`direct_sources` lists them; exact for those
    pairs, and no expansion about a single point is needed."""
    if wx not in ("expansion", "direct"):
        raise ValueError("wx must be 'expansion' or 'direct'")
    wxd = wx == "direct"
    q = _f64(q_re) + 1j * _f64(q_im)
    nm = q.shape[0]
    N = nm - 1
    nf = tree.tr.shape[0]
    ncomp = 3 if grad else 1
    out = np.zeros((ncomp, nm, nf), dtype=complex)
    nc = (M + 1) * (M + 2) // 2
    # upward pass: leaf moments, then children into parents (deepest level first)
    mom = {}
    for b in sorted(tree.boxes, key=lambda k: -k[0]):
        rc, zc = tree.centre(b)
        if not tree.children[b]:
            s = tree.src[b]
            mom[b] = _moments(tree.sr[s], tree.sz[s], q[:, s], rc, zc, M) if len(s) else np.zeros((nm, nc), complex)
        else:
            acc = np.zeros((nm, nc), complex)
            for c in tree.children[b]:
                cr, cz = tree.centre(c)
                acc += _shift_up(mom[c], (rc - cr, zc - cz), M)
            mom[b] = acc
    # downward pass: parent locals, V list (moments), X list (sources).  A V-list operator
    # depends only on the level, the two radial stations and the axial box offset (Sec. 2.2:
    # the operators are shared along z), so it is built once per such key
    loc, vop = {}, {}
    for b in sorted(tree.boxes, key=lambda k: k[0]):
        rc, zc = tree.centre(b)
        F = np.zeros((nm, nc), complex)
        pb = tree.parent[b]
        if pb is not None and pb in loc:
            pr, pz = tree.centre(pb)
            F += _shift_down(loc[pb], (pr - rc, pz - zc), M)
        for c in tree.V[b]:
            key = (b[0], b[1], c[1], b[2] - c[2])
            if key not in vop:
                cr, cz = tree.centre(c)
                vop[key] = _s2l_matrix(rc, zc, cr, cz, N, M, M)
            F += np.einsum('nab,nb->na', vop[key], mom[c])
        for c in ([] if wxd else tree.X[b]):
            for s in tree.src[c]:
                T = _s2l_matrix(rc, zc, tree.sr[s], tree.sz[s], N, M, 0)
                F += T[:, :, 0] * q[:, s][:, None]
        loc[b] = F
    # leaves: local expansion, W list (moments at the points), U list (direct)
    K, Lf = _cidx(M)
    for b in tree.leaves:
        t = tree.tgt[b]
        if len(t) == 0:
            continue
        rc, zc = tree.centre(b)
        du, dv = tree.tr[t] - rc, tree.tz[t] - zc
        pw = du[:, None] ** K[None, :] * dv[:, None] ** Lf[None, :]
        out[0][:, t] += loc[b] @ pw.T
        if grad:
            pr_ = np.where(K > 0, K, 0)[None, :] * du[:, None] ** np.maximum(K - 1, 0)[None, :] * dv[:, None] ** Lf[None, :]
            pz_ = np.where(Lf > 0, Lf, 0)[None, :] * du[:, None] ** K[None, :] * dv[:, None] ** np.maximum(Lf - 1, 0)[None, :]
            out[1][:, t] += loc[b] @ pr_.T
            out[2][:, t] += loc[b] @ pz_.T
        for c in ([] if wxd else tree.W[b]):
            cr, cz = tree.centre(c)
            for jj, j in enumerate(t):
                T = _s2l_matrix(tree.tr[j], tree.tz[j], cr, cz, N, 1 if grad else 0, M)
                v = np.einsum('nab,nb->na', T, mom[c])  # coefficients (0,0), (0,1), (1,0)
                out[0][:, j] += v[:, 0]
                if grad:
                    out[1][:, j] += v[:, 2]  # (k, l) = (1, 0)
                    out[2][:, j] += v[:, 1]  # (k, l) = (0, 1)
        if wxd:
            s = direct_sources(tree, b)
        else:
            s = np.concatenate([tree.src[c] for c in tree.U[b]]) if tree.U[b] else np.zeros(0, np.int64)
        if len(s):
            d = direct(tree.sr[s], tree.sz[s], tree.tr[t], tree.tz[t], q.real[:, s], q.imag[:, s], grad=grad)
            out[0][:, t] += d[0] + 1j * d[1]
            if grad:
                out[1][:, t] += d[2] + 1j * d[3]
                out[2][:, t] += d[4] + 1j * d[5]
    res = []
    for c in range(ncomp):
        res += [np.ascontiguousarray(out[c].real), np.ascontiguousarray(out[c].imag)]
    return tuple(res)


def transposed(tree):
    """The same tree with the roles of sources and field points exchanged.  The split rule
    (more than leaf_size sources or field points) and the square are symmetric in the two
    roles, so the boxes and the V lists are the same; the lists of each role follow."""
    return AdaptiveTree(tree.tr, tree.tz, tree.sr, tree.sz, tree.leaf_size, max_level=tree.max_level,
                        refine_to=tree.refine_to, geom=(tree.r0, tree.z0, tree.L), balance=tree.balance)


def adaptive_adjoint(tree, q_re, q_im, gphi_re, gphi_im, M, wx="direct"):
    """Adjoint of :func:`adaptive_fmm` for a real loss with dL/dPhi = gphi (the FMM with the
    roles exchanged, evaluated with its gradient at the sources; G is symmetric in r <-> r1
    and even in x, Sec. 2.2).  Returns (gq_re, gq_im [nmodes, ns], g_r, g_z [ns]) with
    g_r = sum_n Re(S) dPsi_re/dr + Im(S) dPsi_im/dr (the same for z), Psi the transposed
    field at the sources."""
    T = transposed(tree)
    P = adaptive_fmm(T, gphi_re, gphi_im, M, grad=True, wx=wx)
    q_re, q_im = _f64(q_re), _f64(q_im)
    g_r = np.sum(q_re * P[2] + q_im * P[3], axis=0)
    g_z = np.sum(q_re * P[4] + q_im * P[5], axis=0)
    return P[0], P[1], g_r, g_z
