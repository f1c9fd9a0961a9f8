"""Python handle on the plain FP64 CPU oracle (``fslbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use this module; the CUDA library never imports it and it
imports nothing of the CUDA library.  Workloads reach it as plain parameter
dictionaries plus seeded initial fill levels from the input generators.

Parity pinned by the ``-m "not gpu"`` tests (lattice moments, Guo moments,
mass conservation, resting pool, standing-wave frequency and damping,
Young-Laplace jump, TRT Poiseuille, hand-built refilling neighbourhoods,
normal/curvature exactness, free-slip plug flow, Smagorinsky closure, one
periodic layer = D2Q9, and the bubble model: library labelling, p V through
compression, merge and split, pressures unchanged by a mirrored grid), and
on hand-built states: the mass flux with every pair of Thuerey classes (R5),
the excess-mass receivers and shares and the lost-mass accumulator (R3),
the conflict priority (R6), the refilling means (R7), the obstacle-narrowed
normals (R11), the trace observables (R14) and the wave's cell convention
(R13).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fslbm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle_fsl.so")
_lock = threading.Lock()
_lib = None

REFILL = {"eq": 0, "eq_neq": 1, "geq": 2, "ext": 3, "avg": 4}
OPT_SIMPLE_FLUX = 1
OPT_GEQ_LITERAL_NU = 2
OPT_NEQ_LITERAL_MEAN = 4
OPT_LAPLACE_LITERAL = 8
OPT_BUBBLES = 16
OPT_BUBBLE_GAS_ONLY = 32   # bubbles from gas cells alone, interface cells attached

GAS, IFACE, LIQUID, OBST = 0, 1, 2, 3


class _Config(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int),
        ("trt", ctypes.c_int),
        ("magic", ctypes.c_double),
        ("refill", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("nu", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("sigma", ctypes.c_double),
        ("p_v", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("options", ctypes.c_uint),
        ("les_cs", ctypes.c_double),
        ("free_slip", ctypes.c_int * 3),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    # OpenMP for the order-free per-cell loops where the compiler has it;
    # without it the same source builds sequential
    r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> int:
    """Threads for the oracle's order-free per-cell loops (results are bit
    for bit those of one thread); returns the count in effect (1 without
    OpenMP)."""
    return int(_load().orc_set_threads(int(n)))


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [ctypes.POINTER(_Config)]
        lib.orc_destroy.argtypes = [P]
        lib.orc_init_fill.argtypes = [P, dp, dp, ctypes.c_void_p, ctypes.c_double]
        lib.orc_set_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads(1)
        lib.orc_step.restype = ctypes.c_long
        lib.orc_step.argtypes = [P, ctypes.c_long]
        for name in ("orc_num_cells", "orc_step_count", "orc_unstable_step"):
            getattr(lib, name).restype = ctypes.c_long
            getattr(lib, name).argtypes = [P]
        for name in ("orc_lost_mass", "orc_total_mass", "orc_front", "orc_height",
                     "orc_max_velocity"):
            getattr(lib, name).restype = ctypes.c_double
            getattr(lib, name).argtypes = [P]
        lib.orc_column_height.restype = ctypes.c_double
        lib.orc_column_height.argtypes = [P, ctypes.c_int]
        lib.orc_last_counts.argtypes = [P, ctypes.POINTER(ctypes.c_long)]
        lib.orc_get_types.argtypes = [P, ctypes.c_void_p]
        lib.orc_get_bubbles.argtypes = [P, ctypes.c_void_p, dp]
        lib.orc_bubble_probe.argtypes = [P, ctypes.c_void_p, dp, ctypes.c_int]
        for name in ("orc_get_pdfs", "orc_get_phi", "orc_get_mass", "orc_get_kappa"):
            getattr(lib, name).argtypes = [P, dp]
        lib.orc_normal_at.argtypes = [P, ctypes.c_long, dp]
        lib.orc_curvature_at.restype = ctypes.c_double
        lib.orc_curvature_at.argtypes = [P, ctypes.c_long]
        lib.orc_set_state.argtypes = [P, ctypes.c_void_p, dp, dp, dp]
        lib.orc_refill_probe.argtypes = [P, ctypes.c_long, ctypes.c_void_p, dp]
        lib.orc_feq.restype = ctypes.c_double
        lib.orc_feq.argtypes = [P, ctypes.c_int] + [ctypes.c_double] * 4
        lib.orc_guo.restype = ctypes.c_double
        lib.orc_guo.argtypes = [P, ctypes.c_int] + [ctypes.c_double] * 6
        lib.orc_lattice.argtypes = [P, ctypes.POINTER(ctypes.c_int), dp, ctypes.POINTER(ctypes.c_int)]
        lib.orc_relaxation.argtypes = [P, dp]
        _lib = lib
        return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One FSLBM domain advanced by the CPU oracle.

    ``params`` keys: q (19|27), collision ('srt'|'trt'), magic, refill
    ('eq'|'eq_neq'|'geq'|'ext'|'avg'), shape (nx, ny, nz), periodic (3 bools),
    nu, g (3), sigma, p_v, eps, options (int bit set), les_cs (Smagorinsky
    constant, 0 = off), free_slip (3 bools: walls of that axis are free-slip).
    """

    def __init__(self, params: dict):
        self.lib = _load()
        c = _Config()
        c.q = int(params.get("q", 19))
        c.trt = 1 if params.get("collision", "srt") == "trt" else 0
        c.magic = float(params.get("magic", 3.0 / 16.0))
        c.refill = REFILL[params.get("refill", "eq")]
        nx, ny, nz = params["shape"]
        c.nx, c.ny, c.nz = int(nx), int(ny), int(nz)
        per = params.get("periodic", (True, False, True))
        for a in range(3):
            c.periodic[a] = 1 if per[a] else 0
        c.nu = float(params["nu"])
        g = params.get("g", (0.0, 0.0, 0.0))
        for a in range(3):
            c.g[a] = float(g[a])
        c.sigma = float(params.get("sigma", 0.0))
        c.p_v = float(params.get("p_v", 1.0 / 3.0))
        c.eps = float(params.get("eps", 1e-2))
        c.options = int(params.get("options", 0))
        c.les_cs = float(params.get("les_cs", 0.0))
        fs = params.get("free_slip", (False, False, False))
        for a in range(3):
            c.free_slip[a] = 1 if fs[a] else 0
        self.q = c.q
        self.shape = (c.nx, c.ny, c.nz)
        self.N = c.nx * c.ny * c.nz
        self._cfg = c
        self.h = self.lib.orc_create(ctypes.byref(c))
        if not self.h:
            raise ValueError("oracle rejected the configuration")

    def close(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state ---------------------------------------------------------------
    def init_fill(self, phi, u0=None, obstacle=None, h_ref=float("nan")):
        """phi: (nz, ny, nx) or flat, x fastest; u0: (..., 3) or None."""
        phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(-1))
        assert phi.size == self.N
        u0p = None
        if u0 is not None:
            u0 = np.ascontiguousarray(np.asarray(u0, dtype=np.float64).reshape(-1))
            assert u0.size == 3 * self.N
            u0p = _dptr(u0)
        obp = None
        if obstacle is not None:
            obstacle = np.ascontiguousarray(np.asarray(obstacle, dtype=np.uint8).reshape(-1))
            obp = obstacle.ctypes.data_as(ctypes.c_void_p)
        self.lib.orc_init_fill(self.h, _dptr(phi), u0p, obp, float(h_ref))

    def step(self, n: int = 1) -> int:
        return int(self.lib.orc_step(self.h, int(n)))

    def set_state(self, types, phi, pdfs, mass=None):
        types = np.ascontiguousarray(np.asarray(types, dtype=np.uint8).reshape(-1))
        phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(-1))
        pdfs = np.ascontiguousarray(np.asarray(pdfs, dtype=np.float64).reshape(-1))
        assert pdfs.size == self.q * self.N
        mp = None
        if mass is not None:
            mass = np.ascontiguousarray(np.asarray(mass, dtype=np.float64).reshape(-1))
            mp = _dptr(mass)
        self.lib.orc_set_state(self.h, types.ctypes.data_as(ctypes.c_void_p), _dptr(phi),
                               _dptr(pdfs), mp)

    # -- fields (shape (nz, ny, nx); PDFs (q, nz, ny, nx)) ----------------------
    def _grid(self):
        nx, ny, nz = self.shape
        return (nz, ny, nx)

    def types(self):
        out = np.empty(self.N, dtype=np.uint8)
        self.lib.orc_get_types(self.h, out.ctypes.data_as(ctypes.c_void_p))
        return out.reshape(self._grid())

    def pdfs(self):
        out = np.empty(self.q * self.N, dtype=np.float64)
        self.lib.orc_get_pdfs(self.h, _dptr(out))
        return out.reshape((self.q,) + self._grid())

    def phi(self):
        out = np.empty(self.N, dtype=np.float64)
        self.lib.orc_get_phi(self.h, _dptr(out))
        return out.reshape(self._grid())

    def bubbles(self):
        """(label of every cell, -1 none; volume pressure seen by every cell),
        each of shape (nz, ny, nx)."""
        lab = np.empty(self.N, dtype=np.int64)
        p = np.empty(self.N, dtype=np.float64)
        self.lib.orc_get_bubbles(self.h, lab.ctypes.data_as(ctypes.c_void_p), _dptr(p))
        return lab.reshape(self._grid()), p.reshape(self._grid())

    def mass(self):
        out = np.empty(self.N, dtype=np.float64)
        self.lib.orc_get_mass(self.h, _dptr(out))
        return out.reshape(self._grid())

    def kappa(self):
        out = np.empty(self.N, dtype=np.float64)
        self.lib.orc_get_kappa(self.h, _dptr(out))
        return out.reshape(self._grid())

    # -- observables ----------------------------------------------------------
    @property
    def step_count(self) -> int:
        return int(self.lib.orc_step_count(self.h))

    @property
    def unstable_step(self) -> int:
        return int(self.lib.orc_unstable_step(self.h))

    def total_mass(self) -> float:
        return float(self.lib.orc_total_mass(self.h))

    def lost_mass(self) -> float:
        return float(self.lib.orc_lost_mass(self.h))

    def column_height(self, i0: int = 0) -> float:
        return float(self.lib.orc_column_height(self.h, int(i0)))

    def front(self) -> float:
        return float(self.lib.orc_front(self.h))

    def height(self) -> float:
        return float(self.lib.orc_height(self.h))

    def max_velocity(self) -> float:
        return float(self.lib.orc_max_velocity(self.h))

    def last_counts(self):
        out = (ctypes.c_long * 3)()
        self.lib.orc_last_counts(self.h, out)
        return tuple(int(v) for v in out)

    # -- single-function probes --------------------------------------------------
    def normal_at(self, x: int):
        out = np.zeros(3)
        self.lib.orc_normal_at(self.h, int(x), _dptr(out))
        return out

    def curvature_at(self, x: int) -> float:
        return float(self.lib.orc_curvature_at(self.h, int(x)))

    def bubble_probe(self, types, phi, first: bool):
        """Set types and fill levels and run only the bubble bookkeeping."""
        types = np.ascontiguousarray(np.asarray(types, dtype=np.uint8).reshape(-1))
        phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(-1))
        self.lib.orc_bubble_probe(self.h, types.ctypes.data_as(ctypes.c_void_p), _dptr(phi),
                                  1 if first else 0)
        return self.bubbles()

    def refill_probe(self, x: int, new_mask):
        new_mask = np.ascontiguousarray(np.asarray(new_mask, dtype=np.uint8).reshape(-1))
        out = np.zeros(self.q)
        self.lib.orc_refill_probe(self.h, int(x), new_mask.ctypes.data_as(ctypes.c_void_p),
                                  _dptr(out))
        return out

    def feq(self, i, rho, u):
        return float(self.lib.orc_feq(self.h, int(i), float(rho), *map(float, u)))

    def guo(self, i, u, F):
        return float(self.lib.orc_guo(self.h, int(i), *map(float, u), *map(float, F)))

    def lattice(self):
        c = (ctypes.c_int * (3 * self.q))()
        w = np.zeros(self.q)
        opp = (ctypes.c_int * self.q)()
        self.lib.orc_lattice(self.h, c, _dptr(w), opp)
        return np.array(list(c)).reshape(self.q, 3), w, np.array(list(opp))

    def relaxation(self):
        out = np.zeros(4)
        self.lib.orc_relaxation(self.h, _dptr(out))
        return dict(tau=out[0], omega=out[1], lam_e=out[2], lam_o=out[3])
