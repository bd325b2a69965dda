"""Python binding of libsu3gb300: the checkerboard Cabibbo-Marinari SU(3)
heatbath on a GB300 GPU (after Berg, arXiv:0904.0642).

The binding only marshals arguments to the C ABI declared in
``include/su3.h``; every step of the method runs in the CUDA kernels of the
shared library.  Functions carry the C names (``su3_lattice_create``,
``su3_sweep``, ...) and raise :class:`Su3Error` on a non-OK status; the
classes :class:`Lattice`, :class:`Ensemble` and :class:`Server` wrap the
handles.  There is no CPU fallback: importing the package fails loudly when
the shared library has not been built (``python -m
paper_0904_0642_gb300.build`` or ``__graft_entry__.build()``).

PyTorch is optional plumbing: a ``torch.cuda.Stream`` may be passed as the
stream and a CUDA tensor as the link buffer.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, byref, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_uint64,
                    c_void_p)

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SU3_DEBUG_BOUNDS=1 selects the build with device bounds checks (see
# su3_bounds_status in include/su3.h)
LIB_PATH = os.path.join(_HERE, "libsu3gb300_dbg.so" if os.environ.get("SU3_DEBUG_BOUNDS") == "1" else "libsu3gb300.so")
MAX_D = 4

SU3_OK, SU3_EINVAL, SU3_ENOMEM, SU3_ECUDA, SU3_ETIMEOUT, SU3_EBUSY, SU3_ENOTFOUND = 0, -1, -2, -3, -4, -5, -6
SU3_PBC, SU3_DLT = 0, 1
SU3_FP64_18, SU3_FP32_12, SU3_FP32_18 = 0, 1, 2
SU3_START_COLD, SU3_START_HOT = 0, 1
SU3_LINKS_FP64_18, SU3_LINKS_FP32_12 = 0, 1

EXPORTED = [
    "su3_config_init", "su3_link_bytes", "su3_lattice_create", "su3_lattice_create_ex", "su3_lattice_destroy",
    "su3_sweep", "su3_reunitarize", "su3_plaquette", "su3_polyakov", "su3_measure_async", "su3_measurements",
    "su3_get_links", "su3_set_links", "su3_stage_links", "su3_stage_links_ex", "su3_apply_links", "su3_measurement_latest", "su3_measurement_latest_async", "su3_synchronize", "su3_wait", "su3_ensemble_wait", "su3_stats", "su3_action", "su3_action_reset", "su3_set_sweep_counter", "su3_lattice_info", "su3_set_launch",
    "su3_autotune", "su3_use_graph", "su3_use_pdl", "su3_set_profiling", "su3_get_profile", "su3_ensemble_create", "su3_ensemble_destroy", "su3_ensemble_sweep",
    "su3_ensemble_measure", "su3_ensemble_get_links", "su3_ensemble_measurements", "su3_ensemble_set_launch", "su3_ensemble_autotune", "su3_ensemble_use_graph",
    "su3_ensemble_set_profiling", "su3_ensemble_get_profile",
    "su3_server_create", "su3_server_submit", "su3_server_poll", "su3_server_wait", "su3_server_load",
    "su3_server_destroy", "su3_server_stats", "su3_last_error", "su3_version", "su3_measure_noalloc",
    "su3_inject_fault", "su3_bounds_status", "su3_bounds_selftest",
]


class Su3Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


class su3_config(Structure):
    _fields_ = [
        ("D", c_int32), ("dims", c_int32 * MAX_D), ("boundary", c_int32), ("glue_mask", c_int32),
        ("beta", c_double), ("seed", c_uint64), ("storage", c_int32), ("start", c_int32), ("hits", c_int32),
        ("reunit_every", c_int32), ("measure_every", c_int32), ("measure_capacity", c_int32),
        ("layer_blind", c_int32), ("rng_period", c_int32 * MAX_D), ("stream", c_void_p), ("link_buffer", c_void_p),
        ("link_buffer_bytes", c_size_t), ("beta1", c_double), ("ndiv", c_int32 * MAX_D),
    ]


class su3_profile(Structure):
    _fields_ = [
        ("update_ms", c_double), ("update_launches", c_int64), ("reunit_ms", c_double),
        ("reunit_launches", c_int64), ("measure_ms", c_double), ("measure_launches", c_int64),
    ]


class su3_job(Structure):
    _fields_ = [("cfg", su3_config), ("sweeps", c_int32), ("links_in", c_void_p), ("links_out", c_void_p)]


class su3_result(Structure):
    _fields_ = [
        ("job_id", c_uint64), ("status", c_int32), ("nlayers", c_int32), ("plaquette", c_double * 3),
        ("polyakov", c_double * 2), ("layer_plaquette", c_double * 2), ("proposals", c_uint64),
        ("accepts", c_uint64), ("submit_s", c_double), ("start_s", c_double), ("finish_s", c_double),
    ]


_lib = None


def lib():
    """The loaded shared library; raises ImportError when it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_0904_0642_gb300.build` "
                              "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, sz = c_void_p, POINTER(c_double), c_size_t
        u64p = POINTER(c_uint64)
        sig = {
            "su3_config_init": (None, [POINTER(su3_config)]),
            "su3_link_bytes": (sz, [POINTER(su3_config)]),
            "su3_lattice_create": (c_int, [c_int, POINTER(c_int), c_int, c_double, c_uint64, POINTER(vp)]),
            "su3_lattice_create_ex": (c_int, [POINTER(su3_config), POINTER(vp)]),
            "su3_lattice_destroy": (None, [vp]),
            "su3_sweep": (c_int, [vp, c_int, c_int]),
            "su3_reunitarize": (c_int, [vp]),
            "su3_plaquette": (c_int, [vp, c_int, dp, dp, dp]),
            "su3_polyakov": (c_int, [vp, c_int, dp, dp]),
            "su3_measure_async": (c_int, [vp, vp]),
            "su3_measurements": (c_int, [vp, dp, sz, POINTER(sz)]),
            "su3_get_links": (c_int, [vp, dp, sz]),
            "su3_set_links": (c_int, [vp, dp, sz]),
            "su3_stage_links": (c_int, [vp, dp, sz]),
            "su3_stage_links_ex": (c_int, [vp, c_void_p, sz, c_int]),
            "su3_measurement_latest": (c_int, [vp, dp, sz]),
            "su3_measurement_latest_async": (c_int, [vp, dp, sz]),
            "su3_synchronize": (c_int, [vp]),
            "su3_wait": (c_int, [vp, c_double]),
            "su3_ensemble_wait": (c_int, [vp, c_double]),
            "su3_apply_links": (c_int, [vp]),
            "su3_stats": (c_int, [vp, u64p, u64p, u64p]),
            "su3_set_sweep_counter": (c_int, [vp, c_uint64]),
            "su3_action": (c_int, [vp, dp, dp]),
            "su3_action_reset": (c_int, [vp]),
            "su3_lattice_info": (c_int, [vp, POINTER(sz), POINTER(sz)]),
            "su3_set_launch": (c_int, [vp, c_int, c_int, c_int]),
            "su3_autotune": (c_int, [vp, POINTER(c_int), POINTER(c_int), POINTER(c_int), dp]),
            "su3_use_graph": (c_int, [vp, c_int]),
            "su3_use_pdl": (c_int, [vp, c_int]),
            "su3_set_profiling": (c_int, [vp, c_int]),
            "su3_get_profile": (c_int, [vp, POINTER(su3_profile), c_int]),
            "su3_ensemble_set_profiling": (c_int, [vp, c_int]),
            "su3_ensemble_get_profile": (c_int, [vp, POINTER(su3_profile), c_int]),
            "su3_ensemble_create": (c_int, [POINTER(su3_config), c_int, vp, POINTER(vp)]),
            "su3_ensemble_destroy": (None, [vp]),
            "su3_ensemble_sweep": (c_int, [vp, c_int]),
            "su3_ensemble_measure": (c_int, [vp, dp]),
            "su3_ensemble_get_links": (c_int, [vp, c_int, dp, sz]),
            "su3_ensemble_measurements": (c_int, [vp, c_int, dp, sz, POINTER(sz)]),
            "su3_ensemble_set_launch": (c_int, [vp, c_int, c_int, c_int]),
            "su3_ensemble_autotune": (c_int, [vp, POINTER(c_int), POINTER(c_int), POINTER(c_int), dp]),
            "su3_ensemble_use_graph": (c_int, [vp, c_int]),
            "su3_server_create": (c_int, [sz, c_int, POINTER(vp)]),
            "su3_server_submit": (c_int, [vp, POINTER(su3_job), u64p]),
            "su3_server_poll": (c_int, [vp, c_uint64, POINTER(su3_result)]),
            "su3_server_wait": (c_int, [vp, c_uint64, c_double, POINTER(su3_result)]),
            "su3_server_load": (c_int, [vp, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
            "su3_server_destroy": (None, [vp]),
            "su3_last_error": (c_char_p, []),
            "su3_version": (c_char_p, []),
            "su3_measure_noalloc": (c_int, [POINTER(su3_config), vp, vp, vp]),
            "su3_inject_fault": (c_int, [c_char_p, c_int]),
            "su3_server_stats": (c_int, [vp, u64p, dp]),
            "su3_bounds_status": (c_int, [u64p, POINTER(c_int64), POINTER(c_int64)]),
            "su3_bounds_selftest": (c_int, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != SU3_OK:
        raise Su3Error(status, lib().su3_last_error().decode())


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(POINTER(c_double))


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


# ---------------------------------------------------------------- C-named wrappers


def su3_config_init() -> su3_config:
    c = su3_config()
    lib().su3_config_init(byref(c))
    return c


def su3_link_bytes(cfg: su3_config) -> int:
    return int(lib().su3_link_bytes(byref(cfg)))


def su3_lattice_create(D, dims, boundary, beta, seed) -> int:
    h = c_void_p()
    arr = (c_int * len(dims))(*dims)
    _check(lib().su3_lattice_create(D, arr, boundary, beta, seed, byref(h)))
    return h.value


def su3_lattice_create_ex(cfg: su3_config) -> int:
    h = c_void_p()
    _check(lib().su3_lattice_create_ex(byref(cfg), byref(h)))
    return h.value


def su3_lattice_destroy(h):
    lib().su3_lattice_destroy(h)


def su3_sweep(h, n: int, hits: int):
    _check(lib().su3_sweep(h, n, hits))


def su3_reunitarize(h):
    _check(lib().su3_reunitarize(h))


def su3_plaquette(h, layer: int = -1):
    t, s, ti = c_double(), c_double(), c_double()
    _check(lib().su3_plaquette(h, layer, byref(t), byref(s), byref(ti)))
    return t.value, s.value, ti.value


def su3_polyakov(h, layer: int = -1) -> complex:
    re, im = c_double(), c_double()
    _check(lib().su3_polyakov(h, layer, byref(re), byref(im)))
    return complex(re.value, im.value)


def su3_measure_async(h, device_ptr: int):
    _check(lib().su3_measure_async(h, device_ptr))


def su3_measurements(h, nlayers: int, max_entries: int = 1 << 16) -> np.ndarray:
    per = 5 * (nlayers + 1)
    out = np.zeros((max_entries, per), dtype=np.float64)
    cnt = c_size_t()
    _check(lib().su3_measurements(h, _dp(out), max_entries, byref(cnt)))
    return out[: cnt.value].reshape(cnt.value, nlayers + 1, 5)


def su3_get_links(h, out: np.ndarray):
    _check(lib().su3_get_links(h, _dp(out), out.size))


def su3_set_links(h, links: np.ndarray):
    links = np.ascontiguousarray(links, dtype=np.float64)
    _check(lib().su3_set_links(h, _dp(links), links.size))


def su3_stage_links(h, links: np.ndarray):
    """Start the asynchronous copy of links (contiguous float64, canonical
    layout); the caller keeps `links` alive and unchanged until a
    synchronising call after su3_apply_links."""
    _check(lib().su3_stage_links(h, _dp(links), links.size))


def su3_apply_links(h):
    _check(lib().su3_apply_links(h))


def su3_stage_links_ex(h, links: np.ndarray, fmt: int):
    _check(lib().su3_stage_links_ex(h, links.ctypes.data, links.size, fmt))


def su3_measurement_latest(h, nlayers: int) -> np.ndarray:
    out = np.zeros(5 * (nlayers + 1), dtype=np.float64)
    _check(lib().su3_measurement_latest(h, _dp(out), out.size))
    return out.reshape(nlayers + 1, 5)


def su3_measurement_latest_async(h, out: np.ndarray):
    """out: float64, C-contiguous, >= 5 * (nlayers + 1) values, ideally in
    page-locked memory; valid after the stream reaches the copy."""
    _check(lib().su3_measurement_latest_async(h, _dp(out), out.size))


def su3_synchronize(h):
    _check(lib().su3_synchronize(h))


def su3_wait(h, timeout_s: float):
    _check(lib().su3_wait(h, float(timeout_s)))


def su3_ensemble_wait(h, timeout_s: float):
    _check(lib().su3_ensemble_wait(h, float(timeout_s)))


def su3_stats(h):
    p, a, s = c_uint64(), c_uint64(), c_uint64()
    _check(lib().su3_stats(h, byref(p), byref(a), byref(s)))
    return p.value, a.value, s.value


def su3_action(h):
    """(booked, direct) action; see include/su3.h."""
    b, d = c_double(), c_double()
    _check(lib().su3_action(h, byref(b), byref(d)))
    return b.value, d.value


def su3_action_reset(h):
    _check(lib().su3_action_reset(h))


def su3_set_sweep_counter(h, sweeps: int):
    _check(lib().su3_set_sweep_counter(h, sweeps))


def su3_lattice_info(h):
    n, b = c_size_t(), c_size_t()
    _check(lib().su3_lattice_info(h, byref(n), byref(b)))
    return n.value, b.value


def su3_set_launch(h, variant: int, threads: int, ctas_per_sm: int = 0):
    _check(lib().su3_set_launch(h, variant, threads, ctas_per_sm))


def su3_autotune(h):
    v, t, c, us = c_int(), c_int(), c_int(), c_double()
    _check(lib().su3_autotune(h, byref(v), byref(t), byref(c), byref(us)))
    return v.value, t.value, c.value, us.value


def su3_use_graph(h, on: bool):
    _check(lib().su3_use_graph(h, int(bool(on))))


def su3_use_pdl(h, on: bool):
    _check(lib().su3_use_pdl(h, int(bool(on))))


def su3_set_profiling(h, on: bool):
    _check(lib().su3_set_profiling(h, int(bool(on))))


def su3_get_profile(h, reset: bool = False) -> dict:
    p = su3_profile()
    _check(lib().su3_get_profile(h, byref(p), int(bool(reset))))
    return {k: getattr(p, k) for k, _ in su3_profile._fields_}


def su3_bounds_status():
    """(site, index, extent) of the first device bounds violation recorded by
    a debug-bounds build, site 0 when none; raises Su3Error (SU3_ECUDA)
    when one was recorded."""
    site, idx, ext = c_uint64(), c_int64(), c_int64()
    st = lib().su3_bounds_status(byref(site), byref(idx), byref(ext))
    rec = (site.value, idx.value, ext.value)
    if st != SU3_OK:
        raise Su3Error(st, lib().su3_last_error().decode() + f" {rec}")
    return rec


def su3_bounds_selftest():
    _check(lib().su3_bounds_selftest())


def su3_inject_fault(site: str, count: int = 1):
    """Arm a host-side failure for tests of the error paths (see include/su3.h)."""
    _check(lib().su3_inject_fault(site.encode(), int(count)))


def su3_measure_noalloc(cfg: su3_config, links_ptr: int, device_out_ptr: int, stream=None):
    """Measure links the caller holds on the device without any allocation
    (for callers that cannot call cudaMalloc); see include/su3.h."""
    _check(lib().su3_measure_noalloc(byref(cfg), links_ptr, device_out_ptr, _stream_handle(stream)))


def su3_last_error() -> str:
    return lib().su3_last_error().decode()


def su3_version() -> str:
    return lib().su3_version().decode()


def _tuned(h, cfgs, cache, run, apply):
    """Autotune through the launch-shape cache (paper_0904_0642_gb300.tuning)."""
    from . import tuning
    path = cache or os.environ.get("SU3_TUNE_CACHE")
    if not path:
        return run(h)
    key = tuning.key_of(cfgs, su3_version())
    hit = tuning.lookup(path, key)
    if hit is not None:
        apply(hit[0], hit[1], hit[2])
        return hit
    shape = run(h)
    tuning.store(path, key, shape)
    return shape


# ---------------------------------------------------------------- classes


def make_config(dims, boundary=SU3_PBC, beta=6.0, seed=1, storage=SU3_FP64_18, start=SU3_START_COLD, hits=2,
                glue_mask=0, reunit_every=0, measure_every=0, measure_capacity=0, layer_blind=False,
                rng_period=None, stream=None, buffer=None, beta1=None, ndiv=None) -> su3_config:
    c = su3_config_init()
    c.D = len(dims)
    for i, n in enumerate(dims):
        c.dims[i] = int(n)
    c.boundary = boundary
    c.beta = float(beta)
    c.seed = int(seed)
    c.storage = storage
    c.start = start
    c.hits = int(hits)
    c.glue_mask = int(glue_mask)
    c.reunit_every = int(reunit_every)
    c.measure_every = int(measure_every)
    c.measure_capacity = int(measure_capacity)
    c.layer_blind = int(bool(layer_blind))
    c.beta1 = -1.0 if beta1 is None else float(beta1)
    if rng_period is not None:
        for i, p in enumerate(rng_period):
            c.rng_period[i] = int(p)
    if ndiv is not None:  # sublattices per direction (Sec. 2.4), on one device
        for i, k in enumerate(ndiv):
            c.ndiv[i] = int(k)
    sh = _stream_handle(stream)
    c.stream = sh
    if buffer is not None:  # a CUDA tensor (torch) or (ptr, nbytes)
        if isinstance(buffer, tuple):
            c.link_buffer, c.link_buffer_bytes = buffer
        else:
            c.link_buffer = int(buffer.data_ptr())
            c.link_buffer_bytes = int(buffer.numel() * buffer.element_size())
    return c


class Lattice:
    """One chain on the GPU: a torus (SU3_PBC) or a double-layered torus."""

    def __init__(self, dims, **kw):
        self._buffer = kw.get("buffer")  # keep a caller buffer alive
        self.cfg = make_config(dims, **kw)
        self.dims = list(dims)
        self.D = len(dims)
        self.nlayers = 2 if self.cfg.boundary == SU3_DLT else 1
        self.V = int(np.prod(dims))
        self.h = su3_lattice_create_ex(self.cfg)

    def close(self):
        if getattr(self, "h", None):
            su3_lattice_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def nlinks(self) -> int:
        return self.nlayers * self.V * self.D

    def sweep(self, n=1, hits=None):
        su3_sweep(self.h, n, self.cfg.hits if hits is None else hits)

    def reunitarize(self):
        su3_reunitarize(self.h)

    def plaquette(self, layer=-1):
        return su3_plaquette(self.h, layer)

    def polyakov(self, layer=-1):
        return su3_polyakov(self.h, layer)

    def measurements(self, max_entries=1 << 16):
        return su3_measurements(self.h, self.nlayers, max_entries)

    def get_links(self) -> np.ndarray:
        out = np.zeros((self.nlayers, self.V, self.D, 3, 3, 2), dtype=np.float64)
        su3_get_links(self.h, out)
        return out

    def set_links(self, links: np.ndarray):
        su3_set_links(self.h, links)

    def stage_links(self, links: np.ndarray, fmt=SU3_LINKS_FP64_18):
        """Queue links for su3_apply_links: canonical float64 (fmt
        SU3_LINKS_FP64_18) or rows 1, 2 as float32 (SU3_LINKS_FP32_12, 12 per
        link); the copy runs while earlier sweeps run.  Pinned host memory
        makes it asynchronous."""
        dt = np.float64 if fmt == SU3_LINKS_FP64_18 else np.float32
        links = np.ascontiguousarray(links, dtype=dt)
        su3_stage_links_ex(self.h, links, fmt)
        self._staged = (getattr(self, "_staged", (None, None))[1], links)  # alive until copied

    def latest_measurement(self) -> np.ndarray:
        """The last measurement recorded by measure_every: [layer.., all] x
        (total, space, time, poly_re, poly_im)."""
        return su3_measurement_latest(self.h, self.nlayers)

    def latest_measurement_async(self, out: np.ndarray):
        """Queue the copy of the last recorded measurement into `out`
        (5 * (nlayers + 1) float64, page-locked for an asynchronous copy);
        read it after synchronize() or an event on the lattice's stream."""
        su3_measurement_latest_async(self.h, out)

    def synchronize(self):
        su3_synchronize(self.h)

    def wait(self, timeout_s: float):
        """Wait for the queued work at most timeout_s seconds (Su3Error with
        SU3_ETIMEOUT after that; the work keeps running)."""
        su3_wait(self.h, timeout_s)

    def apply_links(self):
        su3_apply_links(self.h)

    def measure_into(self, device_ptr: int):
        """Plaquette and Polyakov values of every layer and of the whole
        lattice into device memory (5 * (nlayers + 1) doubles), queued."""
        su3_measure_async(self.h, device_ptr)

    def stats(self):
        return su3_stats(self.h)

    def set_sweep_counter(self, n):
        su3_set_sweep_counter(self.h, n)

    def action(self):
        return su3_action(self.h)

    def action_reset(self):
        su3_action_reset(self.h)

    def set_launch(self, threads, ctas_per_sm=0, variant=0):
        su3_set_launch(self.h, variant, threads, ctas_per_sm)

    def autotune(self, cache: str | None = None):
        """Time the launch shapes and keep the fastest: (variant, threads,
        ctas_per_sm, us_per_sweep).  cache (or $SU3_TUNE_CACHE): a JSON
        file of earlier results for the same shape class; a hit is applied
        without timing, a miss is timed and stored."""
        return _tuned(self.h, [self.cfg], cache, su3_autotune, lambda v, t, c: su3_set_launch(self.h, v, t, c))

    def use_graph(self, on=True):
        su3_use_graph(self.h, on)

    def use_pdl(self, on=True):
        su3_use_pdl(self.h, on)

    def set_profiling(self, on=True):
        su3_set_profiling(self.h, on)

    def profile(self, reset=False):
        return su3_get_profile(self.h, reset)


class Ensemble:
    """Independent chains advanced together by one fused launch per phase."""

    def __init__(self, configs, stream=None):
        arr = (su3_config * len(configs))(*configs)
        self.n = len(configs)
        self.cfgs = list(configs)
        h = c_void_p()
        _check(lib().su3_ensemble_create(arr, self.n, _stream_handle(stream), byref(h)))
        self.h = h.value

    def close(self):
        if getattr(self, "h", None):
            lib().su3_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1):
        _check(lib().su3_ensemble_sweep(self.h, n))

    def wait(self, timeout_s: float):
        su3_ensemble_wait(self.h, timeout_s)

    def measure(self) -> np.ndarray:
        out = np.zeros((self.n, 5), dtype=np.float64)
        _check(lib().su3_ensemble_measure(self.h, _dp(out)))
        return out

    def get_links(self, chain) -> np.ndarray:
        c = self.cfgs[chain]
        nl = 2 if c.boundary == SU3_DLT else 1
        V = int(np.prod([c.dims[i] for i in range(c.D)]))
        out = np.zeros((nl, V, c.D, 3, 3, 2), dtype=np.float64)
        _check(lib().su3_ensemble_get_links(self.h, chain, _dp(out), out.size))
        return out

    def measurements(self, chain, max_entries=1 << 16) -> np.ndarray:
        c = self.cfgs[chain]
        nl = 2 if c.boundary == SU3_DLT else 1
        out = np.zeros((max_entries, 5 * (nl + 1)), dtype=np.float64)
        cnt = c_size_t()
        _check(lib().su3_ensemble_measurements(self.h, chain, _dp(out), max_entries, byref(cnt)))
        return out[: cnt.value].reshape(cnt.value, nl + 1, 5)

    def set_launch(self, threads, ctas_per_sm=0, variant=0):
        _check(lib().su3_ensemble_set_launch(self.h, variant, threads, ctas_per_sm))

    def autotune(self, cache: str | None = None):
        """As Lattice.autotune, for the fused launch of all chains."""
        def run(h):
            v, t, c, us = c_int(), c_int(), c_int(), c_double()
            _check(lib().su3_ensemble_autotune(h, byref(v), byref(t), byref(c), byref(us)))
            return v.value, t.value, c.value, us.value

        def apply(v, t, c):
            _check(lib().su3_ensemble_set_launch(self.h, v, t, c))

        return _tuned(self.h, self.cfgs, cache, run, apply)

    def use_graph(self, on=True):
        _check(lib().su3_ensemble_use_graph(self.h, int(bool(on))))

    def set_profiling(self, on=True):
        _check(lib().su3_ensemble_set_profiling(self.h, int(bool(on))))

    def profile(self, reset=False) -> dict:
        p = su3_profile()
        _check(lib().su3_ensemble_get_profile(self.h, byref(p), int(bool(reset))))
        return {k: getattr(p, k) for k, _ in su3_profile._fields_}


class Server:
    """Continuous-batching job server (see su3_server_* in include/su3.h)."""

    def __init__(self, hbm_budget_bytes=0, max_slots=64):
        h = c_void_p()
        _check(lib().su3_server_create(hbm_budget_bytes, max_slots, byref(h)))
        self.h = h.value
        self._buffers = {}  # job id -> host link buffers the worker reads or writes

    def close(self):
        if getattr(self, "h", None):
            lib().su3_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, cfg: su3_config, sweeps: int, links_in: np.ndarray | None = None,
               links_out: np.ndarray | None = None) -> int:
        """links_in: start configuration (canonical float64 layout, C-contiguous);
        links_out: array of the same shape that receives the final links."""
        job = su3_job()
        job.cfg = cfg
        job.sweeps = int(sweeps)
        keep = []
        for name, a in (("links_in", links_in), ("links_out", links_out)):
            if a is not None:
                if a.dtype != np.float64 or not a.flags.c_contiguous:
                    raise ValueError(f"{name} must be a C-contiguous float64 array")
                setattr(job, name, a.ctypes.data)
                keep.append(a)
        jid = c_uint64()
        _check(lib().su3_server_submit(self.h, byref(job), byref(jid)))
        if keep:
            self._buffers[jid.value] = keep
        return jid.value

    def poll(self, job_id):
        r = su3_result()
        st = lib().su3_server_poll(self.h, job_id, byref(r))
        if st == SU3_EBUSY:
            return None
        _check(st)
        self._buffers.pop(job_id, None)
        return r

    def wait(self, job_id, timeout_s=60.0):
        r = su3_result()
        _check(lib().su3_server_wait(self.h, job_id, timeout_s, byref(r)))
        self._buffers.pop(job_id, None)
        return r

    def load(self):
        q, r, f = c_int(), c_int(), c_int()
        _check(lib().su3_server_load(self.h, byref(q), byref(r), byref(f)))
        return q.value, r.value, f.value

    def stats(self):
        """(rounds run, their device time in ms)."""
        n, ms = c_uint64(), c_double()
        _check(lib().su3_server_stats(self.h, byref(n), byref(ms)))
        return n.value, ms.value
