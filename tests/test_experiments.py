"""Host-side checks of experiments.py (the paper's numerical study re-run on the GPU): the
error measure and the command line.  The runs themselves need the GPU."""
import numpy as np

import experiments


def test_error_measure_is_max_normalised_per_mode():
    # Eq. results:error: max_j |a - b| / max_j |b| per mode, complex modulus
    b = (np.array([[3.0, 4.0], [0.0, 0.0]]), np.array([[4.0, 0.0], [0.0, 2.0]]))
    a = (b[0] + np.array([[0.5, 0.0], [0.0, 0.0]]), b[1].copy())
    e = experiments._eps(a, b)
    assert np.allclose(e, [0.5 / 5.0, 0.0])


def test_unknown_experiment_is_rejected():
    try:
        experiments.main(["E9"])
    except KeyError:
        return
    raise AssertionError("E9 accepted")
