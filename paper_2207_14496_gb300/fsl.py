"""Thin Python binding of libfsl (C ABI in include/fsl.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides the device workspace (one uint8 tensor) and
the CUDA stream.  Importing this module loads ``_build/libfsl.so`` and raises
if it has not been built; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfsl.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libfsl.so not found at {LIB_PATH}; build it with "
        "`python -m paper_2207_14496_gb300.build` (or __graft_entry__.build())")

_lib = ctypes.CDLL(LIB_PATH)

D3Q19, D3Q27 = 19, 27
SRT, TRT = 0, 1
FP64, FP32, MIXED_FP16, MIXED_BF16 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp16": MIXED_FP16, "bf16": MIXED_BF16}
REFILL = {"eq": 0, "eq_neq": 1, "geq": 2, "ext": 3, "avg": 4}
OPT_SIMPLE_FLUX, OPT_GEQ_LITERAL_NU, OPT_NEQ_LITERAL_MEAN, OPT_LAPLACE_LITERAL = 1, 2, 4, 8

OBS_TOTAL_MASS, OBS_COLUMN_HEIGHT, OBS_FRONT, OBS_HEIGHT = 1, 2, 3, 4
OBS_MAX_VELOCITY, OBS_STATUS, OBS_STEP, OBS_COUNTS = 5, 6, 7, 8
OBS_LOST_MASS, OBS_TRACE = 9, 10
OBS_FIELD_PDF, OBS_FIELD_TYPES, OBS_FIELD_PHI, OBS_FIELD_MASS, OBS_FIELD_KAPPA = 16, 17, 18, 19, 20
OBS_FIELD_BUBBLE, OBS_FIELD_PRESSURE = 21, 22
OPT_BUBBLES = 16
OPT_BUBBLE_GAS_ONLY = 32

STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "workspace", -4: "unstable",
          -5: "timeout", -6: "state"}
ERR_UNSTABLE = -4


class fsl_config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("collision", ctypes.c_int),
        ("trt_magic", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("refill", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("nu", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("sigma", ctypes.c_double),
        ("p_volume", ctypes.c_double),
        ("eps_phi", ctypes.c_double),
        ("options", ctypes.c_uint),
        ("les_cs", ctypes.c_double),
        ("free_slip", ctypes.c_int * 3),
    ]


_VP = ctypes.c_void_p
_SZ = ctypes.c_size_t
_lib.fsl_workspace_bytes.argtypes = [ctypes.POINTER(fsl_config), ctypes.POINTER(_SZ)]
_lib.fsl_create.argtypes = [ctypes.POINTER(fsl_config), _VP, _SZ, _VP, ctypes.POINTER(_VP)]
_lib.fsl_init_fill.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_double]
_lib.fsl_step.argtypes = [_VP, ctypes.c_int]
_lib.fsl_observe.argtypes = [_VP, ctypes.c_int, _VP, _SZ]
_lib.fsl_set_trace.argtypes = [_VP, ctypes.c_int]
_lib.fsl_trace_capacity.restype = ctypes.c_int
_lib.fsl_state_bytes.argtypes = [_VP, ctypes.POINTER(_SZ)]
_lib.fsl_save.argtypes = [_VP, _VP, _SZ]
_lib.fsl_load.argtypes = [_VP, _VP, _SZ]
_lib.fsl_destroy.argtypes = [_VP]
_lib.fsl_lattice_table.argtypes = [ctypes.c_int, _VP, _VP]
_lib.fsl_launches_per_step.argtypes = [_VP]
_lib.fsl_launches_per_step.restype = ctypes.c_int
_lib.fsl_kernel_stats.argtypes = [_VP, ctypes.c_int, ctypes.c_int, _VP]
_lib.fsl_kernel_stats.restype = ctypes.c_int
_lib.fsl_set_variant.argtypes = [_VP, ctypes.c_int]
_lib.fsl_set_variant.restype = ctypes.c_int
_lib.fsl_get_variant.argtypes = [_VP]
_lib.fsl_get_variant.restype = ctypes.c_int
_lib.fsl_total_mass_noalloc.argtypes = [ctypes.POINTER(fsl_config), _VP, _VP, _VP, _VP, _VP, _VP]
_lib.fsl_total_mass_noalloc.restype = ctypes.c_int
_lib.fsl_batch_create.argtypes = [_VP, ctypes.c_int, _VP, ctypes.c_int, ctypes.POINTER(_VP)]
_lib.fsl_batch_create.restype = ctypes.c_int
_lib.fsl_batch_step.argtypes = [_VP, ctypes.c_int]
_lib.fsl_batch_step.restype = ctypes.c_int
_lib.fsl_batch_destroy.argtypes = [_VP]
_lib.fsl_batch_destroy.restype = ctypes.c_int
_lib.fsl_adjoint_workspace_bytes.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_SZ)]
_lib.fsl_adjoint_workspace_bytes.restype = ctypes.c_int
_lib.fsl_adjoint_create.argtypes = [_VP, ctypes.c_int, ctypes.c_int, _VP, _SZ, ctypes.POINTER(_VP)]
_lib.fsl_adjoint_create.restype = ctypes.c_int
_lib.fsl_adjoint_forward.argtypes = [_VP, _VP]
_lib.fsl_adjoint_forward.restype = ctypes.c_int
_lib.fsl_adjoint_backward.argtypes = [_VP, _VP, _VP]
_lib.fsl_adjoint_backward.restype = ctypes.c_int
_lib.fsl_adjoint_destroy.argtypes = [_VP]
_lib.fsl_adjoint_destroy.restype = ctypes.c_int
_lib.fsl_selftest_wait.argtypes = [_VP]
_lib.fsl_selftest_wait.restype = ctypes.c_int
_lib.fsl_status_string.argtypes = [ctypes.c_int]
_lib.fsl_status_string.restype = ctypes.c_char_p
_lib.fsl_last_error.restype = ctypes.c_char_p
for _name in ("fsl_workspace_bytes", "fsl_create", "fsl_init_fill", "fsl_step", "fsl_observe",
              "fsl_set_trace", "fsl_state_bytes", "fsl_save", "fsl_load", "fsl_destroy",
              "fsl_lattice_table"):
    getattr(_lib, _name).restype = ctypes.c_int

EXPORTED = ("fsl_workspace_bytes", "fsl_create", "fsl_init_fill", "fsl_step", "fsl_observe",
            "fsl_set_trace", "fsl_trace_capacity", "fsl_state_bytes", "fsl_save", "fsl_load",
            "fsl_destroy", "fsl_lattice_table", "fsl_launches_per_step", "fsl_kernel_stats",
            "fsl_status_string", "fsl_last_error", "fsl_total_mass_noalloc", "fsl_set_variant",
            "fsl_get_variant", "fsl_batch_create", "fsl_batch_step", "fsl_batch_destroy",
            "fsl_adjoint_workspace_bytes", "fsl_adjoint_create", "fsl_adjoint_forward",
            "fsl_adjoint_backward", "fsl_adjoint_destroy", "fsl_selftest_wait")
VARIANTS = {"default": 0, "pair": 1, "pair_r128": 2, "pair_r96": 3, "tma": 4, "quad64": 5,
            "warp_tma": 6, "pair_pipe": 7, "pair_r80": 8, "cpa": 9, "cpa_deep": 10,
            "cpa_r96": 11, "seg": 12, "seg_r128": 13,
            "cell": 14, "cell_r80": 15, "tma_r96": 16}
KERNEL_STREAM_COLLIDE = 1
KERNEL_BULK_PASS = 2


class FslError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.fsl_status_string(code).decode()
        if code == -2:
            msg += ": " + _lib.fsl_last_error().decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def _check(code: int, where: str):
    if code != 0:
        raise FslError(code, where)


def make_config(params: dict, precision: str = "fp64") -> fsl_config:
    """Build an fsl_config from a workload parameter dictionary (see inputs)."""
    c = fsl_config()
    c.lattice = int(params.get("q", 19))
    c.collision = TRT if params.get("collision", "srt") == "trt" else SRT
    c.trt_magic = float(params.get("magic", 3.0 / 16.0))
    c.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    c.refill = REFILL[params.get("refill", "eq")]
    c.nx, c.ny, c.nz = (int(v) for v in params["shape"])
    per = params.get("periodic", (True, False, True))
    for a in range(3):
        c.periodic[a] = 1 if per[a] else 0
    c.nu = float(params["nu"])
    g = params.get("g", (0.0, 0.0, 0.0))
    for a in range(3):
        c.gravity[a] = float(g[a])
    c.sigma = float(params.get("sigma", 0.0))
    c.p_volume = float(params.get("p_v", 1.0 / 3.0))
    c.eps_phi = float(params.get("eps", 1e-2))
    c.options = int(params.get("options", 0))
    c.les_cs = float(params.get("les_cs", 0.0))
    fs = params.get("free_slip", (False, False, False))
    for a in range(3):
        c.free_slip[a] = 1 if fs[a] else 0
    return c


def workspace_bytes(params: dict, precision: str = "fp64") -> int:
    c = make_config(params, precision)
    n = _SZ()
    _check(_lib.fsl_workspace_bytes(ctypes.byref(c), ctypes.byref(n)), "fsl_workspace_bytes")
    return int(n.value)


def lattice_table(q: int):
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    _check(_lib.fsl_lattice_table(q, c.ctypes.data, w.ctypes.data), "fsl_lattice_table")
    return c, w


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class Sim:
    """One FSLBM domain on the current CUDA device.

    The workspace is a torch uint8 tensor owned by this object; the stream is
    a dedicated torch stream (so that steps can be captured into CUDA graphs)
    unless one is passed.
    """

    def __init__(self, params: dict, precision: str = "fp64", device: int = 0, stream=None):
        import torch

        self.params = dict(params)
        self.precision = precision
        self.cfg = make_config(params, precision)
        self.q = self.cfg.lattice
        self.shape = (self.cfg.nx, self.cfg.ny, self.cfg.nz)
        self.N = self.cfg.nx * self.cfg.ny * self.cfg.nz
        self.device = torch.device("cuda", device)
        n = _SZ()
        _check(_lib.fsl_workspace_bytes(ctypes.byref(self.cfg), ctypes.byref(n)),
               "fsl_workspace_bytes")
        self.bytes = int(n.value)
        self.workspace = torch.empty(self.bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._base = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        h = ctypes.c_void_p()
        _check(_lib.fsl_create(ctypes.byref(self.cfg), ctypes.c_void_p(self._base), self.bytes,
                               ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
               "fsl_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.fsl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_variant(self, variant):
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        _check(_lib.fsl_set_variant(self.h, v), "fsl_set_variant")

    def variant(self) -> int:
        return int(_lib.fsl_get_variant(self.h))

    def launches_per_step(self) -> int:
        return int(_lib.fsl_launches_per_step(self.h))

    def kernel_stats(self, reps: int = 10, kernel: int = KERNEL_STREAM_COLLIDE) -> dict:
        out = np.zeros(4)
        _check(_lib.fsl_kernel_stats(self.h, int(kernel), int(reps), _ptr(out)), "fsl_kernel_stats")
        return dict(ms=float(out[0]), bytes=float(out[1]), n_liquid=int(out[2]),
                    n_interface=int(out[3]))

    def init_fill(self, phi, u0=None, obstacle=None, h_ref=float("nan")):
        phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(-1))
        assert phi.size == self.N
        keep = [phi]
        up = None
        if u0 is not None:
            u0 = np.ascontiguousarray(np.asarray(u0, dtype=np.float64).reshape(-1))
            assert u0.size == 3 * self.N
            keep.append(u0)
            up = _ptr(u0)
        op = None
        if obstacle is not None:
            obstacle = np.ascontiguousarray(np.asarray(obstacle, dtype=np.uint8).reshape(-1))
            keep.append(obstacle)
            op = _ptr(obstacle)
        _check(_lib.fsl_init_fill(self.h, _ptr(phi), up, op, float(h_ref)), "fsl_init_fill")

    def init_workload(self, w: dict):
        self.init_fill(w["phi"], w.get("u0"), w.get("obstacle"), w.get("h_ref", float("nan")))

    def step(self, n: int = 1):
        _check(_lib.fsl_step(self.h, int(n)), "fsl_step")

    def set_trace(self, every: int):
        _check(_lib.fsl_set_trace(self.h, int(every)), "fsl_set_trace")

    # -- observation ------------------------------------------------------------
    def _obs(self, what: int, out: np.ndarray):
        _check(_lib.fsl_observe(self.h, what, _ptr(out), out.nbytes), f"fsl_observe({what})")
        return out

    def _scalar(self, what):
        return float(self._obs(what, np.zeros(1))[0])

    def total_mass(self):
        return self._scalar(OBS_TOTAL_MASS)

    def column_height(self):
        return self._scalar(OBS_COLUMN_HEIGHT)

    def front(self):
        return self._scalar(OBS_FRONT)

    def height(self):
        return self._scalar(OBS_HEIGHT)

    def max_velocity(self):
        return self._scalar(OBS_MAX_VELOCITY)

    def lost_mass(self):
        return self._scalar(OBS_LOST_MASS)

    def status(self):
        v = self._obs(OBS_STATUS, np.zeros(2, dtype=np.int64))
        return int(v[0]), int(v[1])

    def selftest_wait(self):
        """Make one bounded device wait give up (fsl_selftest_wait): the
        handle then reports the timeout status."""
        _check(_lib.fsl_selftest_wait(self.h), "fsl_selftest_wait")

    @property
    def step_count(self) -> int:
        return int(self._obs(OBS_STEP, np.zeros(1, dtype=np.int64))[0])

    def counts(self):
        return tuple(int(v) for v in self._obs(OBS_COUNTS, np.zeros(4, dtype=np.int64)))

    def trace(self, n: int):
        out = np.zeros((n, 3))
        _check(_lib.fsl_observe(self.h, OBS_TRACE, _ptr(out), out.nbytes), "fsl_observe(trace)")
        return out

    def _grid(self):
        nx, ny, nz = self.shape
        return (nz, ny, nx)

    def pdfs(self):
        return self._obs(OBS_FIELD_PDF, np.zeros(self.q * self.N)).reshape((self.q,) + self._grid())

    def types(self):
        return self._obs(OBS_FIELD_TYPES, np.zeros(self.N, dtype=np.uint8)).reshape(self._grid())

    def phi(self):
        return self._obs(OBS_FIELD_PHI, np.zeros(self.N)).reshape(self._grid())

    def mass(self):
        return self._obs(OBS_FIELD_MASS, np.zeros(self.N)).reshape(self._grid())

    def kappa(self):
        return self._obs(OBS_FIELD_KAPPA, np.zeros(self.N)).reshape(self._grid())

    def bubbles(self):
        """Bubble of every cell (dense index of its smallest cell, -1 none)."""
        return self._obs(OBS_FIELD_BUBBLE, np.zeros(self.N, dtype=np.int32)).reshape(self._grid())

    def pressure(self):
        """Volume pressure seen by every cell."""
        return self._obs(OBS_FIELD_PRESSURE, np.zeros(self.N)).reshape(self._grid())

    # -- checkpoint -------------------------------------------------------------
    def save(self) -> np.ndarray:
        n = _SZ()
        _check(_lib.fsl_state_bytes(self.h, ctypes.byref(n)), "fsl_state_bytes")
        buf = np.zeros(int(n.value), dtype=np.uint8)
        _check(_lib.fsl_save(self.h, _ptr(buf), buf.nbytes), "fsl_save")
        return buf

    def load(self, buf: np.ndarray):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(_lib.fsl_load(self.h, _ptr(buf), buf.nbytes), "fsl_load")


class Batch:
    """Many independent simulations stepped together: one CUDA-graph launch
    per `chunk` steps, each member an independent branch of the graph.  The
    members keep their own state and stay usable (observe, save, load)."""

    def __init__(self, sims, chunk: int = 8, stream=None):
        import torch

        self.sims = list(sims)
        if not self.sims:
            raise ValueError("a batch needs at least one simulation")
        dev = self.sims[0].device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        arr = (_VP * len(self.sims))(*[s.h.value for s in self.sims])
        b = ctypes.c_void_p()
        _check(_lib.fsl_batch_create(ctypes.cast(arr, _VP), len(self.sims),
                                     ctypes.c_void_p(self.stream.cuda_stream), int(chunk),
                                     ctypes.byref(b)), "fsl_batch_create")
        self.b = b

    def step(self, n: int = 1):
        _check(_lib.fsl_batch_step(self.b, int(n)), "fsl_batch_step")

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            _lib.fsl_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Adjoint:
    """Discrete adjoint of `nsteps` steps of `sim` from its current state,
    checkpointed every `every` steps (see fsl_adjoint_* in include/fsl.h)."""

    def __init__(self, sim, nsteps: int, every: int = 100):
        import torch

        self.sim = sim
        self.nsteps = int(nsteps)
        n = _SZ()
        _check(_lib.fsl_adjoint_workspace_bytes(sim.h, self.nsteps, int(every), ctypes.byref(n)),
               "fsl_adjoint_workspace_bytes")
        self.bytes = int(n.value)
        self.workspace = torch.empty(self.bytes + 256, dtype=torch.uint8, device=sim.device)
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        a = ctypes.c_void_p()
        _check(_lib.fsl_adjoint_create(sim.h, self.nsteps, int(every), ctypes.c_void_p(base),
                                       self.bytes, ctypes.byref(a)), "fsl_adjoint_create")
        self.a = a

    def forward(self) -> np.ndarray:
        """Run the steps; the column height after each step."""
        col = np.zeros(self.nsteps)
        _check(_lib.fsl_adjoint_forward(self.a, _ptr(col)), "fsl_adjoint_forward")
        return col

    def backward(self, dj_dcolumn) -> dict:
        dj = np.ascontiguousarray(np.asarray(dj_dcolumn, dtype=np.float64))
        assert dj.size == self.nsteps
        nx, ny, nz = self.sim.shape
        out = np.zeros(4 + 2 * self.sim.N)
        _check(_lib.fsl_adjoint_backward(self.a, _ptr(dj), _ptr(out)), "fsl_adjoint_backward")
        n = self.sim.N
        return dict(nu=float(out[0]), g=out[1:4].copy(),
                    drho0=out[4:4 + n].reshape(nz, ny, nx),
                    dphi0=out[4 + n:4 + 2 * n].reshape(nz, ny, nx))

    def close(self):
        if getattr(self, "a", None) is not None and self.a.value:
            _lib.fsl_adjoint_destroy(self.a)
            self.a = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def raw_library():
    """The loaded ctypes library (for the C-ABI symbol checks)."""
    return _lib
