"""Argument checks of the C ABI that run before any CUDA call, so they are
tested here on the CPU: empty and too-small grids, the parameter ranges the
paper fixes (omega in (0, 2], Sec. 2.3; 0 < nu <= 1, Eq. 28; dx == dy on D2Q5,
Sec. 3.4), combinations that are not built, and null handles."""
import ctypes as C

import pytest


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    return vklb


def _status(vk, fn):
    with pytest.raises(vk.VKLBError) as e:
        fn()
    return e.value.status


@pytest.mark.parametrize("kw,status", [
    (dict(n=(0, 32)), "ERR_ARG"),                              # empty grid
    (dict(n=(32, 0)), "ERR_ARG"),
    (dict(n=(2,), lo=(0.0,), hi=(1.0,)), "ERR_ARG"),           # D1Q3 needs 3 cells
    (dict(omega=0.0), "ERR_ARG"), (dict(omega=2.5), "ERR_ARG"),
    (dict(cfl=0.0), "ERR_ARG"), (dict(cfl=1.5), "ERR_ARG"),
    (dict(set_kind="centered", eta=1.0), "ERR_ARG"),          # subcharacteristic: eta < 1 (Sec. 2.3)
    (dict(set_kind="centered", eta=-0.5), "ERR_ARG"),
    (dict(k=-1.0), "ERR_ARG"),
    (dict(n=(32, 16), hi=(1.0, 1.0)), "ERR_ARG"),            # dx != dy
    (dict(hi=(0.0, 1.0)), "ERR_ARG"),                          # empty domain
    (dict(bc="characteristic", n=(2, 2)), "ERR_ARG"),          # a characteristic axis needs 3 cells
    (dict(gamma=1.0), "ERR_ARG"),                              # ideal gas needs gamma > 1
])
def test_create_rejects(vk, kw, status):
    args = dict(system="euler", n=(32, 32), lo=(0.0, 0.0), hi=(1.0, 1.0), precision="fp32")
    args.update(kw)
    system, n, lo, hi = args.pop("system"), args.pop("n"), args.pop("lo"), args.pop("hi")
    assert _status(vk, lambda: vk.Sim(system, n, lo, hi, **args)) == getattr(vk, status)


def test_create_rejects_system_parameters(vk):
    assert _status(vk, lambda: vk.Sim("swe", (32, 32), (0, 0), (1, 1), g=0.0)) == vk.ERR_ARG
    assert _status(vk, lambda: vk.Sim("mhd_glm", (32, 32), (0, 0), (1, 1), ch_factor=0.0)) == vk.ERR_ARG
    assert _status(vk, lambda: vk.Sim("mhd_glm", (32,), (0.0,), (1.0,))) == vk.ERR_UNSUPPORTED   # MHD-GLM is 2D
    # non-periodic 2D faces need 3 or more cells across (checked before any device call)
    assert _status(vk, lambda: vk.Sim("mhd_glm", (2, 32), (0, 0), (2 / 32, 1), bc="characteristic")) == vk.ERR_ARG


def test_null_handles(vk):
    lib = vk._lib
    assert lib.vklb_step(None, 1) == vk.ERR_ARG
    assert lib.vklb_sync(None) == vk.ERR_ARG
    assert lib.vklb_destroy(None) == vk.ERR_ARG
    assert lib.vklb_set_form(None, 1) == vk.ERR_ARG
    assert lib.vklb_set_tiling(None, 128, 8) == vk.ERR_ARG
    assert lib.vklb_batch_step(None, 1, 0) == vk.ERR_ARG
    info = vk.Info()
    assert lib.vklb_info(None, C.byref(info)) == vk.ERR_ARG
    assert lib.vklb_create(None, vk.D2Q5, None, None, None, 0.0, 1, None, None) == vk.ERR_ARG
    for st in (vk.OK, vk.ERR_ARG, vk.ERR_TIMEOUT, vk.ERR_LIMIT):
        assert lib.vklb_strerror(st)


def test_create_rejects_unknown_alpha_norm(vk):
    """vklb_weight.alpha_norm must be VKLB_ALPHA_LOCAL or VKLB_ALPHA_GLOBAL."""
    s = vk.System(vk.EULER, 1.4, 9.81, 6.0, (C.c_double * 2)(1.0, 0.0))
    g = vk.Grid(2, (C.c_int64 * 2)(32, 32), (C.c_double * 2)(0.0, 0.0), (C.c_double * 2)(1.0, 1.0))
    b = vk.BC((C.c_int32 * 2)(0, 0), (C.c_int32 * 2)(0, 0))
    h = vk._P()
    for bad in (2, -1):
        w = vk.Weight(vk.SET_WEIGHTED, 0.05, 2.0, 1.0, 0.9, 0.0, bad)
        assert vk._lib.vklb_create(C.byref(s), vk.D2Q5, C.byref(g), C.byref(b), C.byref(w), 0.0, vk.FP32, None,
                                   C.byref(h)) == vk.ERR_ARG


class _FakeCuda:
    """Stands in for a torch CUDA tensor (attributes only, no device memory)."""

    def __init__(self, shape, dtype="torch.float64", contiguous=True):
        self.is_cuda = True
        self.shape = shape
        self.dtype = dtype
        self._c = contiguous

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        raise AssertionError("the library was reached with an unchecked device buffer")


@pytest.mark.parametrize("bad", [dict(shape=(4, 32, 31)), dict(shape=(4, 32, 32), dtype="torch.float32"),
                                 dict(shape=(4, 32, 32), contiguous=False)])
def test_device_buffers_checked_before_the_library(vk, bad):
    """moments(out=...) and set_state(...) with a CUDA tensor hand the library a
    bare device pointer it cannot bound-check: a wrong shape, dtype or layout is
    rejected in the binding, before any call into the library."""
    stub = vk.Sim.__new__(vk.Sim)
    stub.shape = (4, 32, 32)
    stub._h = vk._P()
    with pytest.raises(ValueError):
        vk.Sim.moments(stub, out=_FakeCuda(**bad))
    with pytest.raises(ValueError):
        vk.Sim.set_state(stub, _FakeCuda(**bad))


class _FakeTensor:
    """Stands in for a CUDA tensor: only a pointer and a size (the library
    checks these before any device call)."""

    is_cuda = True

    def __init__(self, ptr, nbytes):
        self._ptr, self._n = ptr, nbytes

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return self._ptr

    def numel(self):
        return self._n

    def element_size(self):
        return 1


def test_buffer_bytes(vk):
    assert vk.buffer_bytes("euler", (100, 37), "fp32") == 5 * 4 * 128 * 37 * 4   # rows padded to bricks
    assert vk.buffer_bytes("mhd_glm", (64, 64), "bf16") == 5 * 9 * 64 * 64 * 2
    assert vk.buffer_bytes("swe", (400,), "fp64") == 3 * 2 * 400 * 8


@pytest.mark.parametrize("case", ["misaligned", "overlap", "null"])
def test_borrowed_buffers_rejected_before_device_calls(vk, case):
    need = vk.buffer_bytes("euler", (64, 64), "fp32")
    base = 1 << 40
    bufs = {"misaligned": (_FakeTensor(base + 16, need), _FakeTensor(base + 2 * need, need)),
            "overlap": (_FakeTensor(base, need), _FakeTensor(base + need // 2, need)),
            "null": (_FakeTensor(0, need), _FakeTensor(base, need))}[case]
    assert _status(vk, lambda: vk.Sim("euler", (64, 64), (0, 0), (1, 1), buffers=bufs)) == vk.ERR_ARG


def test_borrowed_buffers_too_short(vk):
    need = vk.buffer_bytes("euler", (64, 64), "fp32")
    base = 1 << 40
    with pytest.raises(ValueError):     # the binding's check
        vk.Sim("euler", (64, 64), (0, 0), (1, 1), buffers=(_FakeTensor(base, need), _FakeTensor(base + need, 64)))
    # and the library's own, called directly with a short size
    s = vk.System(vk.EULER, 1.4, 9.81, 6.0, (C.c_double * 2)(1.0, 0.0))
    grid = vk.Grid(2, (C.c_int64 * 2)(64, 64), (C.c_double * 2)(0, 0), (C.c_double * 2)(1, 1))
    b = vk.BC((C.c_int32 * 2)(0, 0), (C.c_int32 * 2)(0, 0))
    w = vk.Weight(0, 0.05, 2.0, 1.0, 0.9, 0.0, 0)
    ptrs = (C.c_void_p * 2)(base, base + 2 * need)
    h = C.c_void_p()
    st = vk.lib().vklb_create_borrowed(C.byref(s), vk.D2Q5, C.byref(grid), C.byref(b), C.byref(w), 0.0, vk.FP32,
                                        None, ptrs, need - 1, C.byref(h))
    assert st == vk.ERR_ARG and not h.value


@pytest.mark.parametrize("bc,status", [
    (("transmissive", "characteristic"), "ERR_ARG"),        # the open axes take one kind
    (("characteristic", "transmissive"), "ERR_ARG"),
    ("nonsense", None),
])
def test_boundary_kinds(vk, bc, status):
    if status is None:
        with pytest.raises(KeyError):
            vk.Sim("euler", (16, 16), (0, 0), (1, 1), bc=bc)
        return
    assert _status(vk, lambda: vk.Sim("euler", (16, 16), (0, 0), (1, 1), bc=bc)) == getattr(vk, status)


def test_transmissive_refusals(vk):
    assert _status(vk, lambda: vk.Sim("mhd_glm", (16, 2), (0, 0), (1, 2 / 16), bc="transmissive")) == vk.ERR_ARG
    assert _status(vk, lambda: vk.Sim("euler", (2, 16), (0, 0), (1, 8), bc=("transmissive", "periodic"))) == \
        vk.ERR_ARG
