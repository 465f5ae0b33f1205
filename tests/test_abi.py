"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/afmm.h declares (no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "afmm.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(afmm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("afmm_plan_create", "afmm_eval", "afmm_direct", "afmm_grad", "afmm_adjoint",
                     "afmm_plan_destroy", "afmm_status_string"):
        assert required in names


def test_library_builds_and_exports_every_symbol():
    from paper_2301_01179_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_peak_probe_library_exports_its_header():
    from paper_2301_01179_gb300 import build as B
    B.build()
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "afmm_peaks.h")).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(afmm_[a-z_]+)\s*\(", src)))
    assert names == ["afmm_peak_launch"]
    lib = ctypes.CDLL(B.PEAKS_OUT)
    assert all(hasattr(lib, n) for n in names)
    # bad arguments are rejected on the host, before any launch
    lib.afmm_peak_launch.restype = ctypes.c_int
    ops = ctypes.c_double()
    assert lib.afmm_peak_launch(7, 1, 1, None, ctypes.byref(ops), None) == -1


def test_binding_covers_header():
    torch = pytest.importorskip("torch")  # noqa: F841
    from paper_2301_01179_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_status_strings_and_defaults_without_gpu():
    from paper_2301_01179_gb300 import build as B
    lib = ctypes.CDLL(B.build())
    lib.afmm_status_string.restype = ctypes.c_char_p
    assert lib.afmm_status_string(0) == b"ok"
    assert lib.afmm_status_string(1) == b"invalid argument"
    # plan creation rejects bad sizes on the host before touching the device
    lib.afmm_plan_create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    st = lib.afmm_plan_create(ctypes.byref(h), ctypes.c_int64(0), None, None, ctypes.c_int64(0), None, None, 1,
                              None, None)
    assert st == 1 and not h.value


def test_oracle_builds_and_is_independent():
    import oracle
    path = oracle.build()
    assert os.path.exists(path)
    # the oracle shares no source with the CUDA library
    csrc = os.path.join(ROOT, "paper_2301_01179_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower()
    for f in ("binding.py", "build.py", "workloads.py", "__init__.py"):
        text = open(os.path.join(ROOT, "paper_2301_01179_gb300", f)).read()
        assert "import oracle" not in text and "from oracle" not in text


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of afmm_options and afmm_plan_info_t have the C layout: every
    field at the offset the C compiler gives it, and the same total size."""
    import shutil
    import subprocess
    from paper_2301_01179_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"afmm_options": binding.Options, "afmm_plan_info_t": binding.PlanInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "afmm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _t in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = {}
    for ln in subprocess.check_output([str(exe)]).decode().split("\n"):
        if ln:
            s, f, v = ln.split()
            out[(s, f)] = int(v)
    for cname, py in structs.items():
        assert out[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f, _t in py._fields_:
            assert out[(cname, f)] == getattr(py, f).offset, (cname, f)
