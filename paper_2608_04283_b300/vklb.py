"""Thin ctypes binding of libvklb.so (C ABI in include/vklb.h).

Argument marshalling only: every step of the method runs in the CUDA kernels of
the library.  Importing this module raises if the library has not been built
(``python -m paper_2608_04283_b300.build``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvklb.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libvklb.so is not built: run `python -m paper_2608_04283_b300.build`")
_lib = C.CDLL(LIB_PATH)

# ------------------------------------------------------------------ constants
OK, ERR_ARG, ERR_NOMEM, ERR_CUDA, ERR_NONPHYSICAL, ERR_CFL, ERR_TIMEOUT, ERR_STATE, ERR_UNSUPPORTED, ERR_LIMIT = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9
ADVECT, SWE, EULER, MHD_GLM = 0, 1, 2, 3
D1Q3, D2Q5 = 13, 25
BC_PERIODIC, BC_CHARACTERISTIC, BC_TRANSMISSIVE = 0, 1, 2
BC_KIND = {"periodic": BC_PERIODIC, "characteristic": BC_CHARACTERISTIC, "transmissive": BC_TRANSMISSIVE}
SET_WEIGHTED, SET_CENTERED, SET_DISCONTINUOUS = 0, 1, 2
FP64, FP32, BF16_STORE = 0, 1, 2

SYSTEM_KIND = {"advection": ADVECT, "swe": SWE, "euler": EULER, "mhd_glm": MHD_GLM}
SET_KIND = {"weighted": SET_WEIGHTED, "centered": SET_CENTERED, "discontinuous": SET_DISCONTINUOUS}
ALPHA_NORM = {"global": 0, "local": 1}   # vklb_alpha_norm
PRECISION = {"fp64": FP64, "fp32": FP32, "bf16": BF16_STORE}


class System(C.Structure):
    _fields_ = [("kind", C.c_int32), ("gamma", C.c_double), ("g", C.c_double),
                ("ch_factor", C.c_double), ("adv_speed", C.c_double * 2)]


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int64 * 2), ("lo", C.c_double * 2), ("hi", C.c_double * 2)]


class BC(C.Structure):
    _fields_ = [("lo", C.c_int32 * 2), ("hi", C.c_int32 * 2)]


class Weight(C.Structure):
    _fields_ = [("set", C.c_int32), ("c", C.c_double), ("k", C.c_double), ("omega", C.c_double),
                ("cfl", C.c_double), ("eta", C.c_double), ("alpha_norm", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("p", C.c_int32), ("q", C.c_int32), ("precision", C.c_int32), ("store_bytes", C.c_int32),
                ("cells", C.c_int64), ("bytes_per_lup", C.c_int64), ("state_bytes", C.c_int64),
                ("dx", C.c_double), ("tile_x", C.c_int32), ("tile_y", C.c_int32),
                ("kernels_per_step", C.c_int32), ("variant", C.c_int32), ("pitch", C.c_int64),
                ("blocks_per_sm", C.c_int32), ("sms", C.c_int32), ("form", C.c_int32)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIGS = {
    "vklb_create": (C.c_int, [C.POINTER(System), C.c_int32, C.POINTER(Grid), C.POINTER(BC), C.POINTER(Weight),
                              C.c_double, C.c_int32, _P, C.POINTER(_P)]),
    "vklb_create_borrowed": (C.c_int, [C.POINTER(System), C.c_int32, C.POINTER(Grid), C.POINTER(BC),
                                       C.POINTER(Weight), C.c_double, C.c_int32, _P, C.POINTER(_P), C.c_size_t,
                                       C.POINTER(_P)]),
    "vklb_buffer_bytes": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(Grid), C.c_int32, C.POINTER(C.c_size_t)]),
    "vklb_set_state": (C.c_int, [_P, _P, C.c_int32]),
    "vklb_set_tiling": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "vklb_set_variant": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "vklb_set_form": (C.c_int, [_P, C.c_int32]),
    "vklb_step": (C.c_int, [_P, C.c_int64]),
    "vklb_step_to": (C.c_int, [_P, C.c_double]),
    "vklb_sync": (C.c_int, [_P]),
    "vklb_moments": (C.c_int, [_P, _P, C.c_int32]),
    "vklb_conservation_totals": (C.c_int, [_P, _D]),
    "vklb_time": (C.c_int, [_P, _D, C.POINTER(C.c_int64), _D]),
    "vklb_info": (C.c_int, [_P, C.POINTER(Info)]),
    "vklb_device_state": (C.c_int, [_P, C.POINTER(_P)]),
    "vklb_poison_next": (C.c_int, [_P]),
    "vklb_state_bytes": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
    "vklb_get_state": (C.c_int, [_P, _P, C.c_size_t]),
    "vklb_put_state": (C.c_int, [_P, _P, C.c_size_t]),
    "vklb_destroy": (C.c_int, [_P]),
    "vklb_strerror": (C.c_char_p, [C.c_int]),
    "vklb_batch_create": (C.c_int, [C.c_int32, C.POINTER(_P), C.POINTER(_P)]),
    "vklb_batch_set_tiling": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "vklb_batch_step": (C.c_int, [_P, C.c_int64, C.c_int32]),
    "vklb_batch_destroy": (C.c_int, [_P]),
    "vklb_launch_count": (C.c_int64, []),
    "vklb_selftest_wait_timeout": (C.c_int, [C.c_int64, _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def buffer_bytes(system, n, precision="fp32"):
    """Bytes of one distribution buffer (vklb_buffer_bytes) for Sim(buffers=...)."""
    n = tuple(int(v) for v in n)
    dim = len(n)
    grid = Grid(dim, (C.c_int64 * 2)(n[0], n[1] if dim == 2 else 1), (C.c_double * 2)(0.0, 0.0),
                (C.c_double * 2)(1.0, 1.0))
    out = C.c_size_t()
    _check(_lib.vklb_buffer_bytes(SYSTEM_KIND[system], D1Q3 if dim == 1 else D2Q5, C.byref(grid),
                                  PRECISION[precision], C.byref(out)), "vklb_buffer_bytes")
    return out.value


class VKLBError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {_lib.vklb_strerror(status).decode()} ({status})")


def _check(st, where):
    if st != OK:
        raise VKLBError(st, where)


def launch_count():
    return int(_lib.vklb_launch_count())


def selftest_wait_timeout(limit_ns=1_000_000, stream=None):
    """Status of a bounded device wait that is made to run out (ERR_TIMEOUT expected)."""
    return int(_lib.vklb_selftest_wait_timeout(int(limit_ns), _stream_handle(stream)))


def lib():
    return _lib


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Sim:
    """One simulation (see vklb_create).  ``system`` in advection / swe / euler /
    mhd_glm; ``n`` = (nx,) or (nx, ny); ``lo``/``hi`` domain corners; ``bc``
    "periodic", "characteristic" or "transmissive", or per axis in 2D, e.g.
    ("characteristic", "periodic") (vklb_bc); ``form``
    "moments" keeps U instead of f as the state (D2Q5, omega = 1; vklb_set_form);
    ``eta`` > 0 takes the subcharacteristic lattice speed of the centered set
    instead of the CFL rule (vklb_weight.eta); ``alpha_norm`` "global" (default) or
    "local" places the sigmoid weight's normaliser (vklb_weight.alpha_norm);
    ``buffers`` = two contiguous CUDA tensors of at least buffer_bytes() bytes
    each holds the distributions in the caller's memory (vklb_create_borrowed;
    the tensors are kept referenced for the simulation's lifetime)."""

    def __init__(self, system, n, lo, hi, bc="periodic", set_kind="weighted", c=0.05, k=2.0, omega=1.0,
                 cfl=0.9, dt=0.0, precision="fp32", gamma=1.4, g=9.81, ch_factor=6.0, adv_speed=(1.0, 0.0),
                 stream=None, form="distributions", eta=0.0, alpha_norm="global", buffers=None):
        n = tuple(int(v) for v in n)
        dim = len(n)
        lo = tuple(float(v) for v in np.atleast_1d(lo))
        hi = tuple(float(v) for v in np.atleast_1d(hi))
        s = System(SYSTEM_KIND[system], float(gamma), float(g), float(ch_factor),
                   (C.c_double * 2)(*[float(v) for v in adv_speed]))
        grid = Grid(dim, (C.c_int64 * 2)(n[0], n[1] if dim == 2 else 1),
                    (C.c_double * 2)(lo[0], lo[1] if dim == 2 else 0.0),
                    (C.c_double * 2)(hi[0], hi[1] if dim == 2 else 1.0))
        axes = (bc,) * 2 if isinstance(bc, str) else tuple(bc) + (bc[-1],) * (2 - len(bc))
        kinds = [BC_KIND[b_] for b_ in axes]
        b = BC((C.c_int32 * 2)(*kinds), (C.c_int32 * 2)(*kinds))
        w = Weight(SET_KIND[set_kind], float(c), float(k), float(omega), float(cfl), float(eta),
                   ALPHA_NORM[alpha_norm])
        self._h = _P()
        self.system, self.n, self.dim = system, n, dim
        self.precision = precision
        self._stream = stream
        lat = D1Q3 if dim == 1 else D2Q5
        if buffers is None:
            _check(_lib.vklb_create(C.byref(s), lat, C.byref(grid), C.byref(b), C.byref(w), float(dt),
                                    PRECISION[precision], _stream_handle(stream), C.byref(self._h)), "vklb_create")
        else:
            # two caller-owned device buffers (torch CUDA tensors), borrowed for
            # the simulation's lifetime
            need = buffer_bytes(system, n, precision)
            for t in buffers:
                if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
                    raise ValueError("buffers: need two contiguous CUDA tensors")
                if t.numel() * t.element_size() < need:
                    raise ValueError(f"buffers: need {need} bytes each")
            self._buffers = tuple(buffers)
            ptrs = (_P * 2)(buffers[0].data_ptr(), buffers[1].data_ptr())
            _check(_lib.vklb_create_borrowed(C.byref(s), lat, C.byref(grid), C.byref(b), C.byref(w), float(dt),
                                             PRECISION[precision], _stream_handle(stream), ptrs, need,
                                             C.byref(self._h)), "vklb_create_borrowed")
        self.info = Info()
        _check(_lib.vklb_info(self._h, C.byref(self.info)), "vklb_info")
        self.p = self.info.p
        self.shape = (self.p,) + tuple(reversed(n))
        if form != "distributions":
            self.set_form(form)

    # ------------------------------------------------------------------ core
    @property
    def handle(self):
        return self._h

    def _check_device_array(self, U, what):
        """A torch CUDA tensor handed to the library as a device pointer of
        p * cells doubles: float64, contiguous, of the state's shape (the
        library cannot check a device pointer's extent)."""
        if str(U.dtype) != "torch.float64" or not U.is_contiguous() or tuple(U.shape) != self.shape:
            raise ValueError(f"{what}: need a contiguous float64 CUDA tensor of shape {self.shape}, "
                             f"got {U.dtype} {tuple(U.shape)} contiguous={U.is_contiguous()}")

    def set_state(self, U):
        """U: numpy float64 [p, (ny,) nx] on the host, or a torch CUDA float64 tensor."""
        if hasattr(U, "is_cuda") and U.is_cuda:
            self._check_device_array(U, "set_state")
            _check(_lib.vklb_set_state(self._h, _P(U.data_ptr()), 1), "vklb_set_state")
            return
        U = np.ascontiguousarray(U, dtype=np.float64)
        if U.shape != self.shape:
            raise ValueError(f"state shape {U.shape} != {self.shape}")
        _check(_lib.vklb_set_state(self._h, U.ctypes.data_as(_P), 0), "vklb_set_state")

    def set_tiling(self, tx, ty):
        """Step-kernel tile: tx cells by ty rows per block; ty = -1 fits the
        grid to whole waves of resident blocks (resolved height in info.tile_y)."""
        _check(_lib.vklb_set_tiling(self._h, int(tx), int(ty)), "vklb_set_tiling")
        _check(_lib.vklb_info(self._h, C.byref(self.info)), "vklb_info")

    def set_form(self, form):
        """"distributions" (0) or "moments" (1); the state must be set afterwards."""
        code = {"distributions": 0, "moments": 1}.get(form, form)
        _check(_lib.vklb_set_form(self._h, int(code)), "vklb_set_form")
        _check(_lib.vklb_info(self._h, C.byref(self.info)), "vklb_info")

    def set_variant(self, variant, stages=0):
        """0: plain coalesced loads; 1: bulk-copy (TMA) row pipeline with ``stages`` rows in flight."""
        _check(_lib.vklb_set_variant(self._h, int(variant), int(stages)), "vklb_set_variant")
        _check(_lib.vklb_info(self._h, C.byref(self.info)), "vklb_info")

    def step(self, n=1):
        _check(_lib.vklb_step(self._h, int(n)), "vklb_step")

    def step_to(self, t_end):
        _check(_lib.vklb_step_to(self._h, float(t_end)), "vklb_step_to")

    def sync(self):
        _check(_lib.vklb_sync(self._h), "vklb_sync")

    def moments(self, out=None):
        """U = sum_q f_q as float64: numpy on the host, or into a torch CUDA tensor ``out``."""
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            self._check_device_array(out, "moments")
            _check(_lib.vklb_moments(self._h, _P(out.data_ptr()), 1), "vklb_moments")
            return out
        if out is not None:
            if not (out.dtype == np.float64 and out.flags.c_contiguous and out.shape == self.shape):
                raise ValueError(f"moments: need a C-contiguous float64 array of shape {self.shape}")
            _check(_lib.vklb_moments(self._h, out.ctypes.data_as(_P), 0), "vklb_moments")
            return out
        U = np.empty(self.shape, dtype=np.float64)
        _check(_lib.vklb_moments(self._h, U.ctypes.data_as(_P), 0), "vklb_moments")
        return U

    def totals(self):
        t = np.empty(self.p, dtype=np.float64)
        _check(_lib.vklb_conservation_totals(self._h, t.ctypes.data_as(_D)), "vklb_conservation_totals")
        return t

    def time(self):
        t = C.c_double()
        n = C.c_int64()
        xi = C.c_double()
        _check(_lib.vklb_time(self._h, C.byref(t), C.byref(n), C.byref(xi)), "vklb_time")
        return t.value, n.value, xi.value

    def poison_next(self):
        """Fill the buffer the next step writes with NaN (vklb_poison_next)."""
        _check(_lib.vklb_poison_next(self._h), "vklb_poison_next")

    def device_state(self):
        p = _P()
        _check(_lib.vklb_device_state(self._h, C.byref(p)), "vklb_device_state")
        return p.value

    def get_state(self):
        nb = C.c_size_t()
        _check(_lib.vklb_state_bytes(self._h, C.byref(nb)), "vklb_state_bytes")
        buf = np.empty(nb.value, dtype=np.uint8)
        _check(_lib.vklb_get_state(self._h, buf.ctypes.data_as(_P), nb.value), "vklb_get_state")
        return buf

    def put_state(self, blob):
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(_lib.vklb_put_state(self._h, blob.ctypes.data_as(_P), blob.size), "vklb_put_state")

    def close(self):
        if self._h:
            _check(_lib.vklb_destroy(self._h), "vklb_destroy")
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Batched stepping of simulations that share system, precision and weight."""

    def __init__(self, sims, tile=None):
        self.sims = list(sims)
        arr = (_P * len(self.sims))(*[s.handle for s in self.sims])
        self._h = _P()
        _check(_lib.vklb_batch_create(len(self.sims), arr, C.byref(self._h)), "vklb_batch_create")
        if tile is not None:
            self.set_tiling(*tile)

    def set_tiling(self, tx, ty):
        _check(_lib.vklb_batch_set_tiling(self._h, int(tx), int(ty)), "vklb_batch_set_tiling")

    def step(self, n=1, graph=True):
        _check(_lib.vklb_batch_step(self._h, int(n), 1 if graph else 0), "vklb_batch_step")

    def close(self):
        if self._h:
            _check(_lib.vklb_batch_destroy(self._h), "vklb_batch_destroy")
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
