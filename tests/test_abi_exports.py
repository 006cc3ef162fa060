"""The C ABI library builds, loads without a GPU, and exports every entry
point that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        for m in re.finditer(r"SCD_API\s+[\w\s\*]+?\b(scd_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["scd_scene_create", "scd_build_boxes", "scd_find_pairs", "scd_find_pairs_device",
                 "scd_get_boxes", "scd_batch_find_pairs", "scd_last_metrics", "scd_scene_destroy",
                 "scd_status_string", "scd_set_allocator", "scd_propagate"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1901_10475_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_1901_10475_gb300 import _binding as B
    assert B.status_string(0) == "ok"
    assert "too small" in B.status_string(B.SCD_ERR_BUFFER_TOO_SMALL)


def test_host_side_argument_checks_without_gpu():
    """Invalid elements and horizons are refused before any device work."""
    import numpy as np
    from paper_1901_10475_gb300 import _binding as B
    pol = B.make_step_policy(B.SCD_STEP_FIXED, fixed_ticks=10)
    good = np.array([[7000.0, 0.01, 0.5, 0.1, 0.2, 0.3, 1.0]])
    for bad_el, hz, tk in [(np.array([[7000.0, 1.0, 0, 0, 0, 0, 1.0]]), 600.0, 1.0),
                           (np.array([[-1.0, 0.0, 0, 0, 0, 0, 1.0]]), 600.0, 1.0),
                           (np.array([[np.nan, 0.0, 0, 0, 0, 0, 1.0]]), 600.0, 1.0),
                           (np.array([[7000.0, 0.0, 0, 0, 0, 0, -1.0]]), 600.0, 1.0),
                           (good, 600.5, 1.0), (good, -5.0, 1.0), (good, 600.0, 0.0)]:
        try:
            B.scd_scene_create(bad_el, hz, tk, pol)
        except B.ScdError as e:
            assert e.status == B.SCD_ERR_INVALID_ARG
        else:
            raise AssertionError("accepted invalid input")


def test_narrow_and_refinement_refuse_missing_arguments_without_gpu():
    """The narrow phase and the refinement entry points check their host
    arguments first (no scene, no output count, eps <= 0): no device work."""
    import ctypes
    from paper_1901_10475_gb300 import _binding as B
    L = B.lib()
    n = ctypes.c_int64(0)
    assert L.scd_narrow_phase(None, None, 0, None, None, None) == B.SCD_ERR_INVALID_ARG
    assert L.scd_narrow_phase(None, None, -1, None, None, None) == B.SCD_ERR_INVALID_ARG
    assert L.scd_refine_witnesses(None, None, 0, ctypes.byref(n), None, None) == \
        B.SCD_ERR_INVALID_ARG
    assert L.scd_refine_continuous(None, 1.0, None, 0, ctypes.byref(n), None, None) == \
        B.SCD_ERR_INVALID_ARG
