"""Thin Python binding of libafmm (include/afmm.h): argument marshalling only.

Every computation runs in the CUDA kernels of libafmm.so; torch provides device memory and
the current stream.  Arrays are torch float64 CUDA tensors; amplitudes and results are
mode-major ``[n_modes, n]`` planes with separate real and imaginary parts, in the caller's
point order.  A missing library or a non-CUDA tensor raises; there is no CPU fallback.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libafmm.so")

AFMM_FP64 = 0
AFMM_MIXED = 1
AFMM_FP64_NATIVE = 2
_PREC = {"fp64": AFMM_FP64, "mixed": AFMM_MIXED, "fp64_native": AFMM_FP64_NATIVE}
_STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
           4: "device wait timed out", 5: "unsupported request"}
EXPORTS = ["afmm_options_default", "afmm_plan_create", "afmm_plan_destroy", "afmm_plan_info", "afmm_eval",
           "afmm_grad", "afmm_direct", "afmm_direct_grad", "afmm_adjoint", "afmm_adjoint_direct", "afmm_green",
           "afmm_green_expansion", "afmm_status_string", "afmm_last_cuda_error", "afmm_set_timing",
           "afmm_get_timing", "afmm_kernel_launches", "afmm_direct_static", "afmm_fourier_analysis",
           "afmm_fourier_synthesis"]


class AfmmError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s (%s)" % (what, _STATUS.get(status, "?"), last_cuda_error()))


class Options(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("leaf_size", ctypes.c_int), ("depth_override", ctypes.c_int),
                ("precision", ctypes.c_int), ("fwd_switch", ctypes.c_double), ("miller_extra", ctypes.c_int),
                ("s2l_engine", ctypes.c_int), ("tree", ctypes.c_int), ("balance", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int), ("n_modes", ctypes.c_int), ("order", ctypes.c_int),
                ("precision", ctypes.c_int), ("r0", ctypes.c_double), ("z0", ctypes.c_double),
                ("side", ctypes.c_double), ("ns", ctypes.c_int64), ("nf", ctypes.c_int64),
                ("n_boxes", ctypes.c_int64 * 17), ("near_pairs", ctypes.c_int64),
                ("s2l_pairs", ctypes.c_int64), ("expansions", ctypes.c_int64),
                ("s2l_point_pairs", ctypes.c_int64), ("s2l_tensor_cores", ctypes.c_int), ("tree", ctypes.c_int),
                ("n_leaves", ctypes.c_int64 * 17), ("near_max_sources", ctypes.c_int64)]


_lib = None


def load():
    """Load libafmm.so (built by paper_2301_01179_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libafmm.so not built: run `python -m paper_2301_01179_gb300.build` "
                           "(no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    lib.afmm_options_default.argtypes = [ctypes.POINTER(Options)]
    lib.afmm_options_default.restype = None
    lib.afmm_plan_create.argtypes = [ctypes.POINTER(P), I64, P, P, I64, P, P, I, ctypes.POINTER(Options), P]
    lib.afmm_plan_create.restype = I
    lib.afmm_plan_destroy.argtypes = [P]
    lib.afmm_plan_destroy.restype = None
    lib.afmm_plan_info.argtypes = [P, ctypes.POINTER(PlanInfo)]
    lib.afmm_plan_info.restype = I
    for name in ("afmm_eval", "afmm_direct"):
        getattr(lib, name).argtypes = [P, P, P, P, P]
        getattr(lib, name).restype = I
    for name in ("afmm_grad", "afmm_direct_grad", "afmm_adjoint", "afmm_adjoint_direct"):
        getattr(lib, name).argtypes = [P] * 9
        getattr(lib, name).restype = I
    lib.afmm_green.argtypes = [I64, P, P, P, I, P, P, P, P]
    lib.afmm_green.restype = I
    lib.afmm_green_expansion.argtypes = [I64, P, P, P, I, I, P, P]
    lib.afmm_green_expansion.restype = I
    lib.afmm_status_string.argtypes = [I]
    lib.afmm_status_string.restype = ctypes.c_char_p
    lib.afmm_last_cuda_error.argtypes = []
    lib.afmm_last_cuda_error.restype = ctypes.c_char_p
    lib.afmm_set_timing.argtypes = [P, I]
    lib.afmm_set_timing.restype = I
    lib.afmm_get_timing.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)]
    lib.afmm_get_timing.restype = I
    lib.afmm_direct_static.argtypes = [I64, P, P, I64, P, P, I, P, P, P, P, P]
    lib.afmm_direct_static.restype = I
    lib.afmm_kernel_launches.argtypes = []
    lib.afmm_kernel_launches.restype = ctypes.c_longlong
    lib.afmm_fourier_analysis.argtypes = [I64, I, P, I, P, P, P]
    lib.afmm_fourier_analysis.restype = I
    lib.afmm_fourier_synthesis.argtypes = [I64, I, P, P, I, P, P]
    lib.afmm_fourier_synthesis.restype = I
    _lib = lib
    return lib


def kernel_launches():
    """Kernel launches made by libafmm in this process so far."""
    return int(load().afmm_kernel_launches())


def last_cuda_error():
    if _lib is None:
        return "library not loaded"
    return _lib.afmm_last_cuda_error().decode()


def _check(status, what):
    if status != 0:
        raise AfmmError(status, what)


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _empty(*shape, like):
    return torch.empty(*shape, dtype=torch.float64, device=like.device)


class Plan:
    """A quadtree plan over sources and field points (afmm_plan_create).

    Parameters mirror ``afmm_options``: ``order`` (M), ``leaf_size``, ``depth`` (0 = rule),
    ``precision`` ("fp64", "mixed" or "fp64_native"), ``fwd_switch``, ``miller_extra``,
    ``s2l_engine`` ("auto": tensor cores where supported, "cuda_cores"), ``tree`` ("uniform":
    the paper's uniform quadtree; "adaptive": boxes split while they hold more than
    ``leaf_size`` sources or field points, ``depth`` then the maximum level) and ``balance``
    (adaptive tree: also split boxes whose neighbour holds more than balance x leaf_size
    points; 0: 4, negative: off).  The plan is bound to the current torch stream at creation.
    """

    def __init__(self, src_r, src_z, tgt_r, tgt_z, n_modes, order=8, leaf_size=32, depth=0, precision="fp64",
                 fwd_switch=0.0, miller_extra=0, s2l_engine="auto", tree="uniform", balance=0):
        lib = load()
        self._lib = lib
        self.ns = int(src_r.numel())
        self.nf = int(tgt_r.numel())
        self.n_modes = int(n_modes)
        self.device = src_r.device
        opt = Options()
        lib.afmm_options_default(ctypes.byref(opt))
        opt.order = int(order)
        opt.leaf_size = int(leaf_size)
        opt.depth_override = int(depth)
        opt.precision = _PREC[precision]
        opt.fwd_switch = float(fwd_switch)
        opt.miller_extra = int(miller_extra)
        opt.s2l_engine = {"auto": 0, "cuda_cores": 1}[s2l_engine]
        opt.tree = {"uniform": 0, "adaptive": 1}[tree]
        opt.balance = int(balance)
        h = ctypes.c_void_p()
        st = lib.afmm_plan_create(ctypes.byref(h), self.ns, _ptr(src_r), _ptr(src_z), self.nf, _ptr(tgt_r),
                                  _ptr(tgt_z), self.n_modes, ctypes.byref(opt), _stream())
        _check(st, "afmm_plan_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.afmm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        inf = PlanInfo()
        _check(self._lib.afmm_plan_info(self._h, ctypes.byref(inf)), "afmm_plan_info")
        return dict(depth=inf.depth, n_modes=inf.n_modes, order=inf.order, precision=inf.precision, r0=inf.r0,
                    z0=inf.z0, side=inf.side, ns=inf.ns, nf=inf.nf, n_boxes=list(inf.n_boxes),
                    near_pairs=inf.near_pairs, s2l_pairs=inf.s2l_pairs, expansions=inf.expansions,
                    s2l_point_pairs=inf.s2l_point_pairs, s2l_tensor_cores=bool(inf.s2l_tensor_cores),
                    tree=("uniform", "adaptive")[inf.tree], n_leaves=list(inf.n_leaves),
                    near_max_sources=inf.near_max_sources)

    def set_timing(self, enable=True):
        _check(self._lib.afmm_set_timing(self._h, 1 if enable else 0), "afmm_set_timing")

    def timing(self):
        out = {}
        for name in ("perm", "p2m", "m2m", "gexp", "s2l", "l2l", "l2p", "near", "total"):
            v = ctypes.c_double()
            _check(self._lib.afmm_get_timing(self._h, name.encode(), ctypes.byref(v)), "afmm_get_timing")
            out[name] = v.value
        return out

    def _out(self, n):
        return _empty(self.n_modes, n, like=self._dev_tensor())

    def _dev_tensor(self):
        return torch.empty(0, dtype=torch.float64, device=self.device)

    def eval(self, q_re, q_im):
        """FMM potentials (afmm_eval): returns (phi_re, phi_im), each [n_modes, nf]."""
        o_re, o_im = self._out(self.nf), self._out(self.nf)
        _check(self._lib.afmm_eval(self._h, _ptr(q_re), _ptr(q_im), _ptr(o_re), _ptr(o_im)), "afmm_eval")
        return o_re, o_im

    def direct(self, q_re, q_im):
        """All-pairs potentials (afmm_direct)."""
        o_re, o_im = self._out(self.nf), self._out(self.nf)
        _check(self._lib.afmm_direct(self._h, _ptr(q_re), _ptr(q_im), _ptr(o_re), _ptr(o_im)), "afmm_direct")
        return o_re, o_im

    def _grad(self, fn, q_re, q_im):
        outs = [self._out(self.nf) for _ in range(6)]
        _check(fn(self._h, _ptr(q_re), _ptr(q_im), *[_ptr(o) for o in outs]), "grad")
        return tuple(outs)

    def grad(self, q_re, q_im):
        """FMM potentials and field gradient: (phi_re, phi_im, dr_re, dr_im, dz_re, dz_im)."""
        return self._grad(self._lib.afmm_grad, q_re, q_im)

    def direct_grad(self, q_re, q_im):
        return self._grad(self._lib.afmm_direct_grad, q_re, q_im)

    def _adj(self, fn, q_re, q_im, gphi_re, gphi_im):
        gq_re, gq_im = self._out(self.ns), self._out(self.ns)
        g_r = torch.empty(self.ns, dtype=torch.float64, device=self.device)
        g_z = torch.empty(self.ns, dtype=torch.float64, device=self.device)
        _check(fn(self._h, _ptr(q_re), _ptr(q_im), _ptr(gphi_re), _ptr(gphi_im), _ptr(gq_re), _ptr(gq_im),
                  _ptr(g_r), _ptr(g_z)), "adjoint")
        return gq_re, gq_im, g_r, g_z

    def adjoint(self, q_re, q_im, gphi_re, gphi_im):
        """Adjoint of eval: (dL/dq re, im, dL/dr_src, dL/dz_src) for upstream dL/dPhi."""
        return self._adj(self._lib.afmm_adjoint, q_re, q_im, gphi_re, gphi_im)

    def adjoint_direct(self, q_re, q_im, gphi_re, gphi_im):
        return self._adj(self._lib.afmm_adjoint_direct, q_re, q_im, gphi_re, gphi_im)


def green(r, r1, x, n_modes, grad=False):
    """G^(n)(r[p], r1[p], x[p]) [n_modes, npairs] (afmm_green); with grad also dG/dr, dG/dx."""
    lib = load()
    n = int(r.numel())
    G = _empty(n_modes, n, like=r)
    Gr = _empty(n_modes, n, like=r) if grad else None
    Gx = _empty(n_modes, n, like=r) if grad else None
    _check(lib.afmm_green(n, _ptr(r), _ptr(r1), _ptr(x), int(n_modes), _ptr(G), _ptr(Gr), _ptr(Gx), _stream()),
           "afmm_green")
    return (G, Gr, Gx) if grad else G


def green_expansion(r, r1, x, n_modes, P):
    """Taylor coefficients gbar^(n)_{i,j,k} [npts, n_modes, P+1, P+1, P+1] (afmm_green_expansion)."""
    lib = load()
    n = int(r.numel())
    out = torch.empty(n, n_modes, P + 1, P + 1, P + 1, dtype=torch.float64, device=r.device)
    _check(lib.afmm_green_expansion(n, _ptr(r), _ptr(r1), _ptr(x), int(n_modes), int(P), _ptr(out), _stream()),
           "afmm_green_expansion")
    return out


def direct_static(src_r, src_z, tgt_r, tgt_z, q_re, q_im):
    """All-pairs potentials without any device allocation inside the library
    (afmm_direct_static): scratch comes from the library's fixed device array."""
    lib = load()
    ns, nf = int(src_r.numel()), int(tgt_r.numel())
    nm = int(q_re.shape[0])
    o_re = _empty(nm, nf, like=src_r)
    o_im = _empty(nm, nf, like=src_r)
    _check(lib.afmm_direct_static(ns, _ptr(src_r), _ptr(src_z), nf, _ptr(tgt_r), _ptr(tgt_z), nm, _ptr(q_re),
                                  _ptr(q_im), _ptr(o_re), _ptr(o_im), _stream()), "afmm_direct_static")
    return o_re, o_im


def fourier_analysis(samples, n_modes):
    """Azimuthal Fourier coefficients S^(n), n = 0..n_modes-1, of real ring densities sampled at
    K equispaced angles (afmm_fourier_analysis): samples [K, npts] -> (S_re, S_im) [n_modes, npts]."""
    lib = load()
    K, npts = samples.shape
    S_re = _empty(n_modes, npts, like=samples)
    S_im = _empty(n_modes, npts, like=samples)
    _check(lib.afmm_fourier_analysis(npts, K, _ptr(samples), int(n_modes), _ptr(S_re), _ptr(S_im), _stream()),
           "afmm_fourier_analysis")
    return S_re, S_im


def fourier_synthesis(phi_re, phi_im, K):
    """The field at K equispaced angles from its modes (afmm_fourier_synthesis):
    [n_modes, npts] -> [K, npts]."""
    lib = load()
    n_modes, npts = phi_re.shape
    out = _empty(int(K), npts, like=phi_re)
    _check(lib.afmm_fourier_synthesis(npts, int(n_modes), _ptr(phi_re), _ptr(phi_im), int(K), _ptr(out), _stream()),
           "afmm_fourier_synthesis")
    return out
