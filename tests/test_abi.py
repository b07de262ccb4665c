"""The C-ABI library builds, loads and exports every entry point that
include/rpim.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes as C
import os
import re

import paper_1802_04256_gb300 as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = ""
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            with open(os.path.join(ROOT, "include", h)) as fh:
                src += fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rpim_\w+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    R.build()
    L = R.lib()
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(R.EXPORTED)


def test_host_side_argument_checks_without_gpu():
    L = R.lib()
    assert R.rpim_version().startswith("rpim-gb300")
    h = C.c_void_p()
    prm = R.Params(2.5, 4.0, 1.03, 0.2, 2)
    assert L.rpim_build_pattern(0, None, None, None, C.byref(prm), None, C.byref(h), None) == 1
    assert b"node count" in L.rpim_last_error()
    info = R.PatternInfo()
    assert L.rpim_pattern_get_info(None, C.byref(info)) == 1
    assert L.rpim_pattern_free(None) == 0


def test_kernel_series_accuracy_host_only():
    """The series that stands for the multiquadric minus its chord agrees
    with the closed form to 5e-17 (absolute; the values are O(0.1)) over the
    whole range of s for the support radii of the workloads."""
    for als in (2.0, 2.5, 3.0, 3.5):
        pieces, degree, n64, err = R.rpim_kernel_series_info(4.0, als, 1.03)
        assert 2 <= pieces <= 16 and degree <= 24 and n64 <= degree + 1
        assert err < 5e-17, (als, err)
