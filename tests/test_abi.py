"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, and exports every entry point include/sw.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "sw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(sw_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1202_0635_gb300 import build
    build.build()
    import paper_1202_0635_gb300 as sw
    return sw.lib()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("sw_create", "sw_sweep", "sw_measure", "sw_destroy", "sw_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    import paper_1202_0635_gb300 as sw
    bound = {n for n, _, _ in sw.EXPORTS}
    assert bound == set(header_functions())
    for name in header_functions():
        assert callable(getattr(sw, name)), name


def test_host_only_entry_points(lib):
    import paper_1202_0635_gb300 as sw
    assert sw.sw_ncounters(2, sw.SW_ISING) == 6
    assert sw.sw_ncounters(6, sw.SW_CLOCK) == 6 + 3 * 4 + 2   # + correlation classes at L/4, L/2
    assert sw.sw_ncounters(3, sw.SW_POTTS) == 3 + 2 + 2
    assert lib.sw_destroy(None) == 0
    assert lib.sw_sweep(None, 1) == sw.SW_ERR_ARG
    assert "null" in sw.sw_last_error()


def test_invalid_arguments_rejected_before_any_device_work(lib):
    import paper_1202_0635_gb300 as sw
    for args in ((6, 2, sw.SW_POTTS, 1.0), (2, 2, sw.SW_POTTS, 1.0), (64, 1, sw.SW_POTTS, 1.0),
                 (64, 3, sw.SW_ISING, 1.0), (64, 2, sw.SW_POTTS, 0.0), (64, 2, sw.SW_POTTS, float("inf")),
                 (64, 65, sw.SW_CLOCK, 1.0), (64, 128, sw.SW_POTTS, 1.0), (64, 2, 7, 1.0),
                 (46344, 2, sw.SW_POTTS, 1.0)):
        h = lib.sw_create(*args[:3], args[3], 1)
        assert not h, args
        assert sw.sw_last_error()
