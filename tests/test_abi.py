"""The C-ABI library loads on a machine without a GPU and exports every
entry point include/gfors.h declares (no compute calls here)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gfors.h")).read()
    return sorted(set(re.findall(r"^GFORS_API[^(]*?\b(gfors_\w+)\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2510_27117_b300 import gfors as G
    names = _declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(G._lib, n), n


def test_host_only_entry_points():
    from paper_2510_27117_b300 import gfors as G
    assert "sm_103a" in G.version()
    p = G.default_params()
    assert abs(p.sigma - 0.99) < 1e-15 and p.k_int == 50 and p.k_b == 1024
    assert G.mlp_nparams(8, 128) == 128 * 8 + 128 + 128 * 128 + 128 + 128 + 1
