"""Pins of the oracle's azimuthal Fourier analysis and synthesis (Sec. 2: Eq. analysis:source
for s(theta) = sum_n S^(n) e^{i n theta}, Eq. analysis:phi for phi = sum_n Phi^(n) e^{i n theta}).

- exact coefficients of band-limited densities with known coefficients;
- the library FFT: S^(n) = rfft(s)[n] / K;
- round trip synthesis(analysis(s)) = s when K >= 2N + 1;
- the convention end to end: analysis -> direct modal sum (Eq. analysis:sum) -> synthesis
  equals a brute-force periodic quadrature of phi(r, theta, z) = int s(theta_1) / (4 pi R)
  dtheta_1 over a ring (Sec. 2), at angles where the sign of the sine terms matters."""
import numpy as np
import pytest

import oracle


def _trig_poly(rng, npts, N, K):
    """Real densities with known coefficients: s = sum_{n=-N..N} S^(n) e^{i n theta}."""
    S = rng.standard_normal((N + 1, npts)) + 1j * rng.standard_normal((N + 1, npts))
    S[0] = S[0].real
    th = 2 * np.pi * np.arange(K) / K
    s = np.real(S[0][None, :] + 2 * sum(S[n][None, :] * np.exp(1j * n * th)[:, None] for n in range(1, N + 1)))
    return S, s


@pytest.mark.parametrize("N,K", [(0, 1), (3, 7), (8, 17), (16, 64), (32, 65)])
def test_analysis_recovers_known_coefficients(N, K):
    rng = np.random.default_rng(N + K)
    S, s = _trig_poly(rng, 5, N, K)
    Sr, Si = oracle.fourier_analysis(s, N + 1)
    assert np.max(np.abs(Sr + 1j * Si - S)) < 1e-13 * max(1.0, np.abs(S).max())


def test_analysis_matches_library_fft():
    rng = np.random.default_rng(3)
    K = 48
    s = rng.standard_normal((K, 7))
    Sr, Si = oracle.fourier_analysis(s, K // 2 + 1)
    F = np.fft.rfft(s, axis=0) / K
    assert np.max(np.abs(Sr + 1j * Si - F)) < 1e-14


@pytest.mark.parametrize("N,K", [(4, 9), (12, 32), (32, 96)])
def test_round_trip(N, K):
    rng = np.random.default_rng(7)
    _, s = _trig_poly(rng, 4, N, K)
    Sr, Si = oracle.fourier_analysis(s, N + 1)
    back = oracle.fourier_synthesis(Sr, Si, K)
    assert np.max(np.abs(back - s)) < 1e-13 * np.abs(s).max()


def test_aliasing_folds_higher_modes():
    # with K < 2N + 1 the mode N + j lands on mode K - N - j: the analysis is the DFT
    K = 8
    th = 2 * np.pi * np.arange(K) / K
    s = np.cos(6 * th)[:, None]  # mode 6 aliases to mode 2 for K = 8
    Sr, Si = oracle.fourier_analysis(s, 3)
    assert abs(Sr[2, 0] - 0.5) < 1e-14 and abs(Sr[1, 0]) < 1e-14


def test_synthesis_of_modal_potentials_is_the_ring_integral():
    # one ring at (r1, z1) with density s(theta_1); field points off the ring
    N, K = 6, 16
    r1, z1 = 0.7, 0.1
    rng = np.random.default_rng(11)
    S, s = _trig_poly(rng, 1, N, K)
    tr = np.array([0.35, 1.2, 0.9, 0.05])
    tz = np.array([0.4, -0.3, 0.1, 0.9])
    Sr, Si = oracle.fourier_analysis(s, N + 1)
    Pr, Pi = oracle.direct(np.array([r1]), np.array([z1]), tr, tz, Sr, Si)
    phi = oracle.fourier_synthesis(Pr, Pi, K)  # [K, nf]
    # brute force: periodic trapezoid rule over theta_1 (spectral for a smooth periodic integrand)
    Q = 4096
    t1 = 2 * np.pi * np.arange(Q) / Q
    dens = np.real(S[0, 0] + 2 * sum(S[n, 0] * np.exp(1j * n * t1) for n in range(1, N + 1)))
    th = 2 * np.pi * np.arange(K) / K
    ref = np.zeros((K, tr.size))
    for j in range(tr.size):
        for k in range(K):
            R = np.sqrt(tr[j] ** 2 + r1 ** 2 - 2 * tr[j] * r1 * np.cos(th[k] - t1) + (tz[j] - z1) ** 2)
            ref[k, j] = np.sum(dens / (4 * np.pi * R)) * (2 * np.pi / Q)
    assert np.max(np.abs(phi - ref)) < 1e-12 * np.abs(ref).max()
