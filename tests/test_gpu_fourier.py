"""GPU azimuthal Fourier analysis and synthesis (Sec. 2, Eqs. analysis:source and
analysis:phi) against the oracle, alone and in the whole pipeline: sampled ring densities ->
modes -> FMM modal potentials -> field at equispaced angles."""
import numpy as np
import pytest

import oracle
from paper_2301_01179_gb300 import workloads as W
from tests.gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K,nm,npts", [(1, 1, 7), (17, 9, 1000), (64, 33, 4099), (96, 33, 257), (8, 12, 300)])
def test_analysis_matches_oracle(K, nm, npts):
    from paper_2301_01179_gb300 import binding
    rng = np.random.default_rng(K + nm)
    s = rng.standard_normal((K, npts))
    Sr, Si = binding.fourier_analysis(*to_dev(s), nm)
    Or, Oi = oracle.fourier_analysis(s, nm)
    g = to_np(Sr, Si)
    assert np.max(np.abs(g[0] + 1j * g[1] - (Or + 1j * Oi))) < 1e-13 * np.abs(s).max()


@pytest.mark.parametrize("K,nm,npts", [(1, 1, 5), (33, 17, 1000), (128, 33, 3001), (7, 12, 64)])
def test_synthesis_matches_oracle(K, nm, npts):
    from paper_2301_01179_gb300 import binding
    rng = np.random.default_rng(3 * K + nm)
    Pr, Pi = rng.standard_normal((nm, npts)), rng.standard_normal((nm, npts))
    g = to_np(binding.fourier_synthesis(*to_dev(Pr, Pi), K))[0]
    o = oracle.fourier_synthesis(Pr, Pi, K)
    assert np.max(np.abs(g - o)) < 1e-13 * max(1.0, np.abs(o).max())


def test_limits():
    from paper_2301_01179_gb300 import binding
    s = to_dev(np.zeros((4097, 3)))[0]
    with pytest.raises(binding.AfmmError) as ei:
        binding.fourier_analysis(s, 2)
    assert ei.value.status == 1


def test_pipeline_densities_to_field():
    """Ring densities s_i(theta) -> S^(n) -> Phi^(n) by the FMM -> phi(r_j, theta_k, z_j),
    against the same chain in the oracle (same tree) at the FP64 bar."""
    from paper_2301_01179_gb300 import binding
    w = W.make("cfg1", ns=2500, nf=1500, n_modes=9)
    K, nm = 17, 9
    rng = np.random.default_rng(21)
    s = rng.standard_normal((K, 2500))  # sampled real densities, band-limited to 8 by K = 17
    sr, sz, tr, tz = to_dev(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"])
    Sr, Si = binding.fourier_analysis(to_dev(s)[0], nm)
    pl = binding.Plan(sr, sz, tr, tz, nm, order=8, depth=4)
    Pr, Pi = pl.eval(Sr, Si)
    pl.close()
    phi = to_np(binding.fourier_synthesis(Pr, Pi, K))[0]
    Or, Oi = oracle.fourier_analysis(s, nm)
    _, geom = oracle.tree_setup(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], 1, depth_override=4)
    F = oracle.fmm(w["src_r"], w["src_z"], w["tgt_r"], w["tgt_z"], Or, Oi, 8, 4, geom)
    ref = oracle.fourier_synthesis(F[0], F[1], K)
    assert np.max(np.abs(phi - ref)) < 1e-10 * np.abs(ref).max()
