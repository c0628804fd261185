"""The C-ABI library loads (no GPU needed) and exports every function that
include/vklb.h declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "vklb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vklb_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("vklb_create", "vklb_step", "vklb_moments", "vklb_conservation_totals", "vklb_step_to",
              "vklb_batch_create", "vklb_batch_step"):
        assert n in names


def test_library_exports_all_declared_symbols():
    from paper_2608_04283_b300 import build
    build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_errors_without_gpu():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    assert vklb.lib().vklb_strerror(vklb.ERR_CFL).decode().startswith("fixed lattice speed")
    # argument checks run before any device call
    import pytest
    with pytest.raises(vklb.VKLBError) as e:
        vklb.Sim("euler", (16, 16), (0, 0), (1, 1), omega=2.5)
    assert e.value.status == vklb.ERR_ARG
    with pytest.raises(vklb.VKLBError) as e:
        vklb.Sim("euler", (16, 8), (0, 0), (1, 1))          # dx != dy (Sec. 3.4)
    assert e.value.status == vklb.ERR_ARG
    with pytest.raises(vklb.VKLBError) as e:
        vklb.Sim("mhd_glm", (16,), (0,), (1,))               # MHD-GLM is built for D2Q5 only
    assert e.value.status == vklb.ERR_UNSUPPORTED
