"""The paper's numerical study (Sec. 4) re-run on the GPU by experiments.py, in its quick
form, checked for the trends the paper reports (no numbers are printed in the paper):
  - E1: the axisymmetric mode is the most accurate, the error larger at larger n (relative
    measure, Sec. 4);
  - E2: log10 eps falls roughly linearly with the order M (the paper's eps ~ C^(-0.4 M)),
    with a weak dependence on the depth, and the axisymmetric mode reaches ten digits at
    M = 16 (Fig. results:error)."""
import contextlib
import io
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rows(which):
    import experiments
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert experiments.main(which + ["--quick"]) == 0
    return [json.loads(l) for l in buf.getvalue().splitlines() if l.strip()]


def test_e1_error_grows_with_mode():
    rows = _rows(["E1"])
    assert [r["M"] for r in rows] == [6, 8, 10, 12, 14, 16]
    for r in rows:
        e = np.array(r["eps_per_mode"])
        assert e.shape == (18,)
        assert e[0] < np.median(e[9:]) / 2, r["M"]
    # and falls with the order at every mode
    e6, e16 = np.array(rows[0]["eps_per_mode"]), np.array(rows[-1]["eps_per_mode"])
    assert np.all(e16 < e6 / 100)


def test_e2_error_against_order():
    rows = _rows(["E2"])
    assert {r["d"] for r in rows} == {5, 6, 7}
    for r in rows:
        assert r["M"][-1] == 16
        assert -0.8 < r["slope_log10_eps_per_M_n0"] < -0.25, r
        assert -0.8 < r["slope_log10_eps_per_M_n8"] < -0.25, r
    big = [r for r in rows if r["Ns"] == max(x["Ns"] for x in rows)]
    assert min(r["eps_n0"][-1] for r in big) < 10 ** -9.5
    # weak dependence on the depth: the slopes of the three depths agree to 25 %
    s = [r["slope_log10_eps_per_M_n0"] for r in big]
    assert (max(s) - min(s)) < 0.25 * abs(np.mean(s)), s
