"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a,
loads, and exports every entry point declared in include/ww.h; the binding
rejects malformed arguments before any device call."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_1210_5672_gb300 import build as B
    B.build()
    import paper_1210_5672_gb300 as ww
    return ww.lib()


def test_header_declares_the_paper_entry_points():
    names = declared_functions()
    for want in ("dtn_setup", "dtn_apply", "shoot", "shoot_jacobian", "objective_and_grad",
                 "ww_create", "ww_destroy", "ww_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(built):
    for name in declared_functions():
        assert hasattr(built, name), name


def test_binding_lists_match_header():
    import paper_1210_5672_gb300 as ww
    assert sorted(ww.EXPORTS) == declared_functions()


def test_library_targets_sm103a(built):
    from paper_1210_5672_gb300 import build as B
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)


def test_binding_rejects_bad_host_arrays():
    import paper_1210_5672_gb300 as ww
    with pytest.raises(TypeError):
        ww._hptr(np.zeros(4, dtype=np.float32), 4, "x")
    with pytest.raises(ValueError):
        ww._hptr(np.zeros(3), 4, "x")
