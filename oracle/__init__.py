"""CPU FP64 oracle for the cylindrical-coordinate FMM (arXiv 2301.01179).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``, never by the product package.  It shares
no code with the CUDA library; the C source ``afmm_oracle.c`` states which passage of
the paper each routine follows.

Layouts: amplitudes and results are mode-major planes, ``q[n, i]`` for mode ``n`` of
source ``i`` and ``phi[n, j]`` for field point ``j`` (numpy float64, C order).

``oracle.adaptive`` holds the FMM on an adaptive quadtree, built on this module's Taylor
coefficients and direct sum.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "afmm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

RULE_SAFE = 0
RULE_PAPER = 1


def build(force=False):
    """Compile liboracle.so with gcc (plain -O2, no fast-math, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    D = ctypes.c_double
    I = ctypes.c_int
    I64 = ctypes.c_int64
    P = ctypes.POINTER(ctypes.c_double)
    lib.orc_carlson_rf.argtypes = [D, D, D]
    lib.orc_carlson_rf.restype = D
    lib.orc_carlson_rd.argtypes = [D, D, D]
    lib.orc_carlson_rd.restype = D
    lib.orc_ellip_ke.argtypes = [D, D, P, P]
    lib.orc_ellip_ke.restype = None
    lib.orc_legendre_q.argtypes = [D, D, D, I, I, P]
    lib.orc_legendre_q.restype = I
    lib.orc_set_rule.argtypes = [I]
    lib.orc_set_rule.restype = None
    lib.orc_green.argtypes = [D, D, D, I, P]
    lib.orc_green.restype = None
    lib.orc_green_grad.argtypes = [D, D, D, I, P, P, P, P]
    lib.orc_green_grad.restype = None
    lib.orc_gbar.argtypes = [D, D, D, I, I, P]
    lib.orc_gbar.restype = I
    lib.orc_direct.argtypes = [I64, P, P, I64, P, P, I, P, P, P, P, P, P, P, P, I]
    lib.orc_direct.restype = None
    lib.orc_adjoint_direct.argtypes = [I64, P, P, I64, P, P, I, P, P, P, P, P, P, P, P, I]
    lib.orc_adjoint_direct.restype = None
    lib.orc_tree_setup.argtypes = [I64, P, P, I64, P, P, I, I, ctypes.POINTER(I), P]
    lib.orc_tree_setup.restype = I
    lib.orc_fmm.argtypes = [I64, P, P, I64, P, P, I, P, P, I, I, P, P, P, P, P, P, P]
    lib.orc_fmm.restype = I
    lib.orc_adjoint_fmm.argtypes = [I64, P, P, I64, P, P, I, P, P, P, P, I, I, P, P, P, P, P]
    lib.orc_adjoint_fmm.restype = I
    PI64 = ctypes.POINTER(ctypes.c_int64)
    lib.orc_fmm_sampled.argtypes = [I64, P, P, I64, P, P, I, P, P, I, I, P, I64, PI64, P, P, P, P, P, P]
    lib.orc_fmm_sampled.restype = I
    lib.orc_adjoint_fmm_sampled.argtypes = [I64, P, P, I64, P, P, I, P, P, P, P, I, I, P, I64, PI64, P, P, P, P]
    lib.orc_adjoint_fmm_sampled.restype = I
    lib.orc_tree_counts.argtypes = [I64, P, P, I64, P, P, I, P, PI64]
    lib.orc_tree_counts.restype = I
    lib.orc_num_threads.argtypes = []
    lib.orc_num_threads.restype = I
    lib.orc_fourier_analysis.argtypes = [I64, I, P, I, P, P]
    lib.orc_fourier_analysis.restype = None
    lib.orc_fourier_synthesis.argtypes = [I64, I, P, P, I, P]
    lib.orc_fourier_synthesis.restype = None
    _lib = lib
    return lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads():
    return _load().orc_num_threads()


def set_rule(rule):
    """Select the Legendre-recursion rule: RULE_SAFE (default) or RULE_PAPER."""
    _load().orc_set_rule(int(rule))


def carlson_rf(x, y, z):
    return _load().orc_carlson_rf(float(x), float(y), float(z))


def carlson_rd(x, y, z):
    return _load().orc_carlson_rd(float(x), float(y), float(z))


def ellip_ke(k2, kp2=None):
    """Complete elliptic integrals K(k), E(k) of modulus k, given k^2 (and optionally
    k'^2 = 1 - k^2 computed without cancellation)."""
    if kp2 is None:
        kp2 = 1.0 - k2
    K = ctypes.c_double()
    E = ctypes.c_double()
    _load().orc_ellip_ke(float(k2), float(kp2), ctypes.byref(K), ctypes.byref(E))
    return K.value, E.value


def legendre_q(t, N, rule=RULE_SAFE):
    """Q_{n-1/2}(1 + t) for n = 0..N; returns (array, used_miller)."""
    t = float(t)
    chi = 1.0 + t
    k2 = 2.0 / (chi + 1.0)
    kp2 = t / (chi + 1.0)
    out = np.zeros(N + 1)
    m = _load().orc_legendre_q(t, k2, kp2, int(N), int(rule), _p(out))
    return out, bool(m)


def green(r, r1, x, N):
    """G^(n)(r, r1, x), n = 0..N (Eq. analysis:gfunc)."""
    out = np.zeros(N + 1)
    _load().orc_green(float(r), float(r1), float(x), int(N), _p(out))
    return out


def green_grad(r, r1, x, N):
    """(G, dG/dr, dG/dx) for n = 0..N."""
    G = np.zeros(N + 1)
    Gr = np.zeros(N + 1)
    Gx = np.zeros(N + 1)
    Gw = np.zeros(max(N, 1) + 1)
    _load().orc_green_grad(float(r), float(r1), float(x), int(N), _p(G), _p(Gr), _p(Gx), _p(Gw))
    return G, Gr, Gx


def gbar(r, r1, x, N, P):
    """Taylor coefficients gbar^(n)_{i,j,k}(r, r1, x) for i+j+k <= P as a dense array
    g[n, i, j, k] (zeros where i+j+k > P)."""
    out = np.zeros((N + 1, P + 1, P + 1, P + 1))
    rc = _load().orc_gbar(float(r), float(r1), float(x), int(N), int(P), _p(out))
    if rc != 0:
        raise MemoryError("orc_gbar")
    return out


def direct(src_r, src_z, tgt_r, tgt_z, q_re, q_im, grad=False, threads=0):
    """Direct modal sum (Eq. analysis:sum).  Returns (phi_re, phi_im) or, with grad,
    (phi_re, phi_im, dr_re, dr_im, dz_re, dz_im), each [nmodes, nf]."""
    sr, sz, tr, tz = map(_f64, (src_r, src_z, tgt_r, tgt_z))
    q_re = _f64(q_re)
    q_im = _f64(q_im)
    nmodes, ns = q_re.shape
    nf = tr.shape[0]
    outs = [np.zeros((nmodes, nf)) for _ in range(6 if grad else 2)]
    g = outs[2:] if grad else [None] * 4
    _load().orc_direct(ns, _p(sr), _p(sz), nf, _p(tr), _p(tz), nmodes, _p(q_re), _p(q_im),
                       _p(outs[0]), _p(outs[1]), _p(g[0]), _p(g[1]), _p(g[2]), _p(g[3]), int(threads))
    return tuple(outs)


def adjoint_direct(src_r, src_z, tgt_r, tgt_z, q_re, q_im, gphi_re, gphi_im, threads=0):
    """Adjoint of the direct sum: returns (gq_re, gq_im, g_r, g_z)."""
    sr, sz, tr, tz = map(_f64, (src_r, src_z, tgt_r, tgt_z))
    q_re, q_im, gphi_re, gphi_im = map(_f64, (q_re, q_im, gphi_re, gphi_im))
    nmodes, ns = q_re.shape
    nf = tr.shape[0]
    gq_re = np.zeros((nmodes, ns))
    gq_im = np.zeros((nmodes, ns))
    g_r = np.zeros(ns)
    g_z = np.zeros(ns)
    _load().orc_adjoint_direct(ns, _p(sr), _p(sz), nf, _p(tr), _p(tz), nmodes, _p(q_re), _p(q_im),
                               _p(gphi_re), _p(gphi_im), _p(gq_re), _p(gq_im), _p(g_r), _p(g_z),
                               int(threads))
    return gq_re, gq_im, g_r, g_z


def tree_setup(src_r, src_z, tgt_r, tgt_z, leaf_size, depth_override=0):
    """Depth d and square domain (r0, z0, L) of the uniform quadtree."""
    sr, sz, tr, tz = map(_f64, (src_r, src_z, tgt_r, tgt_z))
    d = ctypes.c_int()
    geom = np.zeros(3)
    _load().orc_tree_setup(sr.shape[0], _p(sr), _p(sz), tr.shape[0], _p(tr), _p(tz),
                           int(leaf_size), int(depth_override), ctypes.byref(d), _p(geom))
    return d.value, geom


def fmm(src_r, src_z, tgt_r, tgt_z, q_re, q_im, M, d, geom, grad=False):
    """Algorithm 1 (FP64).  Returns (phi_re, phi_im[, dr_re, dr_im, dz_re, dz_im])."""
    sr, sz, tr, tz = map(_f64, (src_r, src_z, tgt_r, tgt_z))
    q_re = _f64(q_re)
    q_im = _f64(q_im)
    geom = _f64(geom)
    nmodes, ns = q_re.shape
    nf = tr.shape[0]
    outs = [np.zeros((nmodes, nf)) for _ in range(6 if grad else 2)]
    g = outs[2:] if grad else [None] * 4
    rc = _load().orc_fmm(ns, _p(sr), _p(sz), nf, _p(tr), _p(tz), nmodes, _p(q_re), _p(q_im), int(M),
                         int(d), _p(geom), _p(outs[0]), _p(outs[1]), _p(g[0]), _p(g[1]), _p(g[2]),
                         _p(g[3]))
    if rc != 0:
        raise RuntimeError("orc_fmm failed: %d" % rc)
    return tuple(outs)


def adjoint_fmm(src_r, src_z, tgt_r, tgt_z, q_re, q_im, gphi_re, gphi_im, M, d, geom):
    """Adjoint of the FMM on the same tree: returns (gq_re, gq_im, g_r, g_z)."""
    sr, sz, tr, tz = map(_f64, (src_r, src_z, tgt_r, tgt_z))
    q_re, q_im, gphi_re, gphi_im = map(_f64, (q_re, q_im, gphi_re, gphi_im))
    geom = _f64(geom)
    nmodes, ns = q_re.shape
    nf = tr.shape[0]
    gq_re = np.zeros((nmodes, ns))
    gq_im = np.zeros((nmodes, ns))
    g_r = np.zeros(ns)
    g_z = np.zeros(ns)
    rc = _load().orc_adjoint_fmm(ns, _p(sr), _p(sz), nf, _p(tr), _p(tz), nmodes, _p(q_re), _p(q_im),
                                 _p(gphi_re), _p(gphi_im), int(M), int(d), _p(geom), _p(gq_re),
                                 _p(gq_im), _p(g_r), _p(g_z))
    if rc != 0:
        raise RuntimeError("orc_adjoint_fmm failed: %d" % rc)
    return gq_re, gq_im, g_r, g_z


def _idx(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def fmm_sampled(src_r, src_z, tgt_r, tgt_z, q_re, q_im, M, d, geom, samples, grad=False):
    """Algorithm 1 (FP64) evaluated only at the field points ``samples`` (indices), for
    checks at full size: each level's S2L into the sample's ancestor box is evaluated at
    the point directly (the shifts are exact re-expansions).  Returns arrays
    [nmodes, len(samples)] as ``fmm``."""
    sr, sz, tr, tz = map(_f64, (src_r, src_z, tgt_r, tgt_z))
    q_re = _f64(q_re)
    q_im = _f64(q_im)
    geom = _f64(geom)
    idx, pidx = _idx(samples)
    nmodes, ns = q_re.shape
    k = idx.shape[0]
    outs = [np.zeros((nmodes, k)) for _ in range(6 if grad else 2)]
    g = outs[2:] if grad else [None] * 4
    rc = _load().orc_fmm_sampled(ns, _p(sr), _p(sz), tr.shape[0], _p(tr), _p(tz), nmodes, _p(q_re), _p(q_im),
                                 int(M), int(d), _p(geom), k, pidx, _p(outs[0]), _p(outs[1]), _p(g[0]),
                                 _p(g[1]), _p(g[2]), _p(g[3]))
    if rc != 0:
        raise RuntimeError("orc_fmm_sampled failed: %d" % rc)
    return tuple(outs)


def adjoint_fmm_sampled(src_r, src_z, tgt_r, tgt_z, q_re, q_im, gphi_re, gphi_im, M, d, geom, samples):
    """The FMM adjoint at the sources ``samples`` only: (gq_re, gq_im) [nmodes, k] and
    (g_r, g_z) [k]."""
    sr, sz, tr, tz = map(_f64, (src_r, src_z, tgt_r, tgt_z))
    q_re, q_im, gphi_re, gphi_im = map(_f64, (q_re, q_im, gphi_re, gphi_im))
    geom = _f64(geom)
    idx, pidx = _idx(samples)
    nmodes, ns = q_re.shape
    k = idx.shape[0]
    gq_re = np.zeros((nmodes, k))
    gq_im = np.zeros((nmodes, k))
    g_r = np.zeros(k)
    g_z = np.zeros(k)
    rc = _load().orc_adjoint_fmm_sampled(ns, _p(sr), _p(sz), tr.shape[0], _p(tr), _p(tz), nmodes, _p(q_re),
                                         _p(q_im), _p(gphi_re), _p(gphi_im), int(M), int(d), _p(geom), k, pidx,
                                         _p(gq_re), _p(gq_im), _p(g_r), _p(g_z))
    if rc != 0:
        raise RuntimeError("orc_adjoint_fmm_sampled failed: %d" % rc)
    return gq_re, gq_im, g_r, g_z


def tree_counts(src_r, src_z, tgt_r, tgt_z, d, geom):
    """(near pairs, S2L box pairs, point pairs under those box pairs) of the uniform tree
    of depth d on the square ``geom``, from the list definitions of Sec. 2.2."""
    sr, sz, tr, tz = map(_f64, (src_r, src_z, tgt_r, tgt_z))
    geom = _f64(geom)
    out, pout = _idx(np.zeros(3, dtype=np.int64))
    rc = _load().orc_tree_counts(sr.shape[0], _p(sr), _p(sz), tr.shape[0], _p(tr), _p(tz), int(d), _p(geom), pout)
    if rc != 0:
        raise RuntimeError("orc_tree_counts failed: %d" % rc)
    return int(out[0]), int(out[1]), int(out[2])


def fourier_analysis(samples, n_modes):
    """Azimuthal Fourier coefficients (Eq. analysis:source) S^(n), n = 0..n_modes-1, of real
    ring densities sampled at K equispaced angles: samples [K, npts] -> (S_re, S_im)
    [n_modes, npts]."""
    smp = _f64(samples)
    K, npts = smp.shape
    S_re = np.zeros((n_modes, npts))
    S_im = np.zeros((n_modes, npts))
    _load().orc_fourier_analysis(npts, K, _p(smp), int(n_modes), _p(S_re), _p(S_im))
    return S_re, S_im


def fourier_synthesis(P_re, P_im, K):
    """phi(theta_k) = Re Phi^(0) + 2 sum_{n>=1} Re(Phi^(n) e^{i n theta_k}) (Eq. analysis:phi)
    at theta_k = 2 pi k / K: [n_modes, npts] -> [K, npts]."""
    P_re = _f64(P_re)
    P_im = _f64(P_im)
    n_modes, npts = P_re.shape
    phi = np.zeros((int(K), npts))
    _load().orc_fourier_synthesis(npts, n_modes, _p(P_re), _p(P_im), int(K), _p(phi))
    return phi
