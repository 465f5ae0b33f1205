"""torch.autograd.Function over the FMM and its adjoint.

``modal_potential(q, plan, src_r, src_z)`` returns the complex modal potentials
Phi^(n)_j = sum_i q_i^(n) G^(n)(r_j, r_i, z_j - z_i) (Eq. analysis:sum) as a complex128
tensor [n_modes, nf]; its backward calls ``afmm_adjoint`` (or ``afmm_adjoint_direct``),
which runs the transposed FMM on the plan's tree and recomputes every Legendre recursion
instead of storing them.  Gradients flow to the complex amplitudes ``q`` and to the
source positions ``src_r``, ``src_z`` (at a fixed tree; the plan is not rebuilt, so the
gradient is that of the FMM evaluated on this tree).

The positions passed here must be those the plan was built on; they only carry the
gradient.  All arithmetic runs in libafmm's kernels.
"""
import torch

from . import binding


class _ModalPotential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, src_r, src_z, plan, direct):
        q_re = q.real.contiguous()
        q_im = q.imag.contiguous()
        if direct:
            phi_re, phi_im = plan.direct(q_re, q_im)
        else:
            phi_re, phi_im = plan.eval(q_re, q_im)
        ctx.plan = plan
        ctx.direct = direct
        ctx.save_for_backward(q_re, q_im)
        return torch.complex(phi_re, phi_im)

    @staticmethod
    def backward(ctx, gphi):
        q_re, q_im = ctx.saved_tensors
        # torch's convention for a real loss: gphi = dL/dRe(Phi) + i dL/dIm(Phi)
        g_re = gphi.real.contiguous()
        g_im = gphi.imag.contiguous()
        fn = ctx.plan.adjoint_direct if ctx.direct else ctx.plan.adjoint
        gq_re, gq_im, g_r, g_z = fn(q_re, q_im, g_re, g_im)
        return torch.complex(gq_re, gq_im), g_r, g_z, None, None


def modal_potential(q, plan, src_r, src_z, direct=False):
    """Differentiable modal potentials at the plan's field points.

    q: complex128 CUDA tensor [n_modes, ns] of source amplitudes S_i^(n).
    plan: a binding.Plan built on (src_r, src_z) and the field points.
    direct: use the all-pairs sum instead of the FMM (forward and adjoint).
    """
    if not q.is_complex():
        raise TypeError("q must be complex (S^(n) for n >= 0)")
    return _ModalPotential.apply(q, src_r, src_z, plan, bool(direct))
