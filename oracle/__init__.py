"""Python access to the double-precision CPU oracle in ``su3_oracle.c``.

TEST INFRASTRUCTURE.  The oracle is the plain, slow checker that the CUDA
library is compared against.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product package
never does, and this module imports nothing from the product package.

All arrays use the canonical layout ``U[layer][site][mu][row][col][re,im]``
(float64), site = i_s - 1 with x^1 fastest (Sec. 2, eq. i_s).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_uint32, c_uint64

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "su3_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
MAXD = 8


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (no FMA contraction, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        try:  # OpenMP over the sites of a phase (optional: the result is the same without it)
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def set_threads(n: int) -> None:
    """Threads for the sites of one phase (OpenMP; 1 by default).  Any
    number gives the same links bit for bit."""
    lib().orc_set_threads(int(n))


def available_threads() -> int:
    """Host cores OpenMP would use (1 when built without OpenMP)."""
    return int(lib().orc_available_threads())


class Geom(ctypes.Structure):
    _fields_ = [
        ("D", c_int32),
        ("dims", c_int32 * MAXD),
        ("nlayers", c_int32),
        ("glue_mask", c_int32),
        ("rng_period", c_int32 * MAXD),
        ("layer_blind", c_int32),
    ]


_lib = None


def _configure(L):
    gp = POINTER(Geom)
    dp = POINTER(c_double)
    L.orc_nsites.argtypes = [gp]
    L.orc_nsites.restype = c_int64
    L.orc_site_index.argtypes = [gp, POINTER(c_int32)]
    L.orc_site_index.restype = c_int64
    L.orc_site_coords.argtypes = [gp, c_int64, POINTER(c_int32)]
    L.orc_colour.argtypes = [gp, POINTER(c_int32)]
    L.orc_colour.restype = c_int
    L.orc_neighbour_table.argtypes = [gp, POINTER(c_int64)]
    L.orc_philox4x32_10.argtypes = [POINTER(c_uint32), POINTER(c_uint32), POINTER(c_uint32)]
    L.orc_cold_start.argtypes = [gp, dp]
    L.orc_hot_start.argtypes = [gp, c_uint64, dp]
    L.orc_staple.argtypes = [gp, dp, c_int, c_int64, c_int, dp]
    L.orc_su2_samples.argtypes = [c_double, c_int, c_uint64, c_int64, c_int, dp, POINTER(c_int32)]
    L.orc_link_heatbath.argtypes = [dp, dp, c_double, c_int, c_uint64, c_uint32, c_uint32, c_int, c_int,
                                    POINTER(c_uint64)]
    L.orc_link_chain.argtypes = [dp, dp, c_double, c_int, c_uint64, c_int64, dp]
    L.orc_sweep.argtypes = [gp, dp, c_double, c_double, c_int, c_uint64, c_int64, c_int, POINTER(c_uint64), dp, dp]
    L.orc_phase.argtypes = [gp, dp, c_double, c_double, c_int, c_uint64, c_int64, c_int, c_int, c_int64, c_int64,
                            POINTER(c_uint64), dp, dp]
    L.orc_staple_weighted.argtypes = [gp, dp, c_int, c_int64, c_int, c_double, c_double, dp]
    L.orc_action_weighted.argtypes = [gp, dp, c_double, c_double]
    L.orc_action_weighted.restype = c_double
    L.orc_set_threads.argtypes = [c_int]
    L.orc_set_threads.restype = None
    L.orc_available_threads.argtypes = []
    L.orc_available_threads.restype = c_int
    L.orc_reunitarize.argtypes = [gp, dp]
    L.orc_reunitarize_matrix.argtypes = [dp]
    L.orc_plaquette.argtypes = [gp, dp, c_int, dp]
    L.orc_polyakov.argtypes = [gp, dp, c_int, dp]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


class use_library:
    """Context manager: route every oracle call to another build of
    su3_oracle.c (the mutation tests load deliberately broken copies)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = lib()
        _lib = _configure(ctypes.CDLL(self.path))
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(POINTER(c_double))


def make_geom(dims, nlayers=1, glue_mask=0, rng_period=None, layer_blind=False) -> Geom:
    g = Geom()
    g.D = len(dims)
    for i, n in enumerate(dims):
        g.dims[i] = int(n)
    g.nlayers = int(nlayers)
    g.glue_mask = int(glue_mask)
    if rng_period is not None:
        for i, p in enumerate(rng_period):
            g.rng_period[i] = int(p)
    g.layer_blind = int(bool(layer_blind))
    return g


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: four 32-bit counter words, two key words."""
    c = (c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def su2_samples(alpha: float, hits: int, seed: int, n: int, subgroup: int = 0):
    """n SU(2) heatbath draws of one subgroup (0, 1, 2) at fixed alpha, draw i
    at counter (i, 0); returns (x[n,4], accepted[n])."""
    x = np.zeros((n, 4), dtype=np.float64)
    acc = np.zeros(n, dtype=np.int32)
    lib().orc_su2_samples(alpha, hits, seed, n, subgroup, _dp(x), acc.ctypes.data_as(POINTER(c_int32)))
    return x, acc.astype(bool)


def link_heatbath(u: np.ndarray, A: np.ndarray, beta: float, hits: int, seed: int, site_key: int, sweep: int,
                  colour: int, mu: int):
    """One Cabibbo-Marinari update of a single 3x3 complex link u with staple A."""
    u18 = np.ascontiguousarray(np.stack([u.real, u.imag], -1), dtype=np.float64).reshape(18)
    A18 = np.ascontiguousarray(np.stack([A.real, A.imag], -1), dtype=np.float64).reshape(18)
    st = (c_uint64 * 2)()
    lib().orc_link_heatbath(_dp(u18), _dp(A18), beta, hits, seed, site_key, sweep, colour, mu, st)
    out = u18.reshape(3, 3, 2)
    return out[..., 0] + 1j * out[..., 1], (int(st[0]), int(st[1]))


def link_chain(A: np.ndarray, beta: float, hits: int, seed: int, n: int, u0: np.ndarray | None = None):
    """n CM updates of one link in the frozen staple A; returns Re Tr(U A) per step."""
    if u0 is None:
        u0 = np.eye(3, dtype=np.complex128)
    u18 = np.ascontiguousarray(np.stack([u0.real, u0.imag], -1), dtype=np.float64).reshape(18)
    A18 = np.ascontiguousarray(np.stack([A.real, A.imag], -1), dtype=np.float64).reshape(18)
    out = np.zeros(n, dtype=np.float64)
    lib().orc_link_chain(_dp(u18), _dp(A18), beta, hits, seed, n, _dp(out))
    return out


def reunitarize_matrix(m: np.ndarray) -> np.ndarray:
    u18 = np.ascontiguousarray(np.stack([m.real, m.imag], -1), dtype=np.float64).reshape(18)
    lib().orc_reunitarize_matrix(_dp(u18))
    o = u18.reshape(3, 3, 2)
    return o[..., 0] + 1j * o[..., 1]


def to_complex(U: np.ndarray) -> np.ndarray:
    """Canonical float64 links [..., 3, 3, 2] -> complex128 [..., 3, 3]."""
    return U[..., 0] + 1j * U[..., 1]


def from_complex(M: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.stack([M.real, M.imag], -1), dtype=np.float64)


class Lattice:
    """Links on a torus (nlayers=1) or double-layered torus (nlayers=2)."""

    def __init__(self, dims, nlayers=1, glue_mask=None, rng_period=None, layer_blind=False):
        dims = [int(n) for n in dims]
        if glue_mask is None:
            glue_mask = (1 << len(dims)) - 1 if nlayers == 2 else 0
        self.dims = dims
        self.D = len(dims)
        self.nlayers = nlayers
        self.glue_mask = glue_mask
        self.geom = make_geom(dims, nlayers, glue_mask, rng_period, layer_blind)
        self.V = int(np.prod(dims))
        self.U = np.zeros((nlayers, self.V, self.D, 3, 3, 2), dtype=np.float64)
        self.sweeps_done = 0

    @property
    def nlinks(self) -> int:
        return self.nlayers * self.V * self.D

    def _g(self):
        return ctypes.byref(self.geom)

    def cold_start(self):
        lib().orc_cold_start(self._g(), _dp(self.U))
        self.sweeps_done = 0
        return self

    def hot_start(self, seed: int):
        lib().orc_hot_start(self._g(), seed, _dp(self.U))
        self.sweeps_done = 0
        return self

    def sweep(self, beta: float, hits: int, seed: int, n: int = 1, sweep0: int | None = None, margins=None,
              kmins=None, beta1: float | None = None):
        """n checkerboard sweeps; returns [proposals, accepts].  margins and
        kmins, if given, are float64 arrays of nlinks entries (initialised to
        +inf) that receive per link the smallest accept-test margin and the
        smallest SU(2) subgroup norm k seen.  beta1 (DLT only): coupling of
        the plaquettes with a link in layer 1 (default: beta)."""
        if sweep0 is None:
            sweep0 = self.sweeps_done
        st = (c_uint64 * 2)()
        mp = _dp(margins) if margins is not None else None
        kp = _dp(kmins) if kmins is not None else None
        lib().orc_sweep(self._g(), _dp(self.U), beta, beta if beta1 is None else beta1, hits, seed, sweep0, n, st,
                        mp, kp)
        self.sweeps_done = sweep0 + n
        return int(st[0]), int(st[1])

    def phase(self, beta: float, hits: int, seed: int, sweep: int, colour: int, mu: int, s_begin: int = 0,
              s_end: int | None = None):
        """One (colour, direction) phase over sites [s_begin, s_end) of each
        layer; returns [proposals, accepts]."""
        st = (c_uint64 * 2)()
        lib().orc_phase(self._g(), _dp(self.U), beta, beta, hits, seed, sweep, colour, mu, s_begin,
                        self.V if s_end is None else s_end, st, None, None)
        return int(st[0]), int(st[1])

    def reunitarize(self):
        lib().orc_reunitarize(self._g(), _dp(self.U))

    def plaquette(self, layer: int = -1):
        out = np.zeros(3)
        lib().orc_plaquette(self._g(), _dp(self.U), layer, _dp(out))
        return float(out[0]), float(out[1]), float(out[2])

    def polyakov(self, layer: int = -1) -> complex:
        out = np.zeros(2)
        lib().orc_polyakov(self._g(), _dp(self.U), layer, _dp(out))
        return complex(out[0], out[1])

    def staple(self, layer: int, site: int, mu: int) -> np.ndarray:
        A = np.zeros(18)
        lib().orc_staple(self._g(), _dp(self.U), layer, site, mu, _dp(A))
        A = A.reshape(3, 3, 2)
        return A[..., 0] + 1j * A[..., 1]

    def staple_weighted(self, layer: int, site: int, mu: int, beta0: float, beta1: float) -> np.ndarray:
        A = np.zeros(18)
        lib().orc_staple_weighted(self._g(), _dp(self.U), layer, site, mu, beta0, beta1, _dp(A))
        A = A.reshape(3, 3, 2)
        return A[..., 0] + 1j * A[..., 1]

    def action_weighted(self, beta0: float, beta1: float) -> float:
        """sum over plaquettes of beta_p (1/3) Re Tr U_p (Sec. 2.2 tagging)."""
        return float(lib().orc_action_weighted(self._g(), _dp(self.U), beta0, beta1))

    def neighbour_table(self) -> np.ndarray:
        out = np.zeros((self.nlayers, self.V, self.D, 2), dtype=np.int64)
        lib().orc_neighbour_table(self._g(), out.ctypes.data_as(POINTER(c_int64)))
        return out

    def site_index(self, x) -> int:
        a = (c_int32 * MAXD)(*[int(v) for v in x])
        return int(lib().orc_site_index(self._g(), a))

    def site_coords(self, s: int):
        a = (c_int32 * MAXD)()
        lib().orc_site_coords(self._g(), s, a)
        return [int(a[i]) for i in range(self.D)]

    def colour(self, x) -> int:
        a = (c_int32 * MAXD)(*[int(v) for v in x])
        return int(lib().orc_colour(self._g(), a))

    def links(self) -> np.ndarray:
        """complex128 view [layer, site, mu, 3, 3]."""
        return to_complex(self.U)

    def set_links(self, M: np.ndarray):
        self.U[...] = from_complex(M).reshape(self.U.shape)
