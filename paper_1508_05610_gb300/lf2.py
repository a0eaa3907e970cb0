"""Thin ctypes binding of liblf2 (C ABI in include/lf2.h).

Functions keep the C names and argument order; this module only marshals arguments,
raises ``LF2Error`` on a non-zero status, and converts numpy / torch arrays to pointers.
Every computation runs in the library's CUDA kernels: there is no Python or CPU fallback,
and loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "liblf2.so")
DEBUG_LIB_PATH = os.path.join(_HERE, "lib", "liblf2_debug.so")  # built with index checks (--debug-bounds)

LF2_OK, LF2_ERR_INVALID, LF2_ERR_UNSUPPORTED, LF2_ERR_NOMEM, LF2_ERR_CUDA, LF2_ERR_TIMEOUT, LF2_ERR_STATE = range(7)
LF2_F64, LF2_F32_KAHAN, LF2_F32 = 0, 1, 2
LF2_MAX_COMP = 6
LF2_KERNEL_AUTO, LF2_KERNEL_SITE, LF2_KERNEL_STREAM, LF2_KERNEL_TBLOCK = 0, 1, 2, 3

PRECISIONS = {"f64": LF2_F64, "f32k": LF2_F32_KAHAN, "f32": LF2_F32}


class lf2_params(ctypes.Structure):
    _fields_ = [("dx", ctypes.c_double), ("dt", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("eta", ctypes.c_double), ("m2", ctypes.c_double)]


class lf2_energy_t(ctypes.Structure):
    _fields_ = [("kinetic", ctypes.c_double), ("gradient", ctypes.c_double), ("potential", ctypes.c_double),
                ("total", ctypes.c_double), ("sum", ctypes.c_double * 6), ("sum_sq", ctypes.c_double * 6)]

    def as_dict(self, ncomp=2):
        return {"kinetic": self.kinetic, "gradient": self.gradient, "potential": self.potential,
                "total": self.total, "sum": np.array(self.sum[:ncomp]), "sum_sq": np.array(self.sum_sq[:ncomp])}


class lf2_step_config(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("zchunk", ctypes.c_int),
                ("depth", ctypes.c_int), ("cx", ctypes.c_int), ("cluster", ctypes.c_int)]


class LF2Error(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__(f"{where}: status {status} ({STATUS_NAMES.get(status, '?')}): {message}")
        self.status = status


STATUS_NAMES = {0: "LF2_OK", 1: "LF2_ERR_INVALID", 2: "LF2_ERR_UNSUPPORTED", 3: "LF2_ERR_NOMEM",
                4: "LF2_ERR_CUDA", 5: "LF2_ERR_TIMEOUT", 6: "LF2_ERR_STATE"}

_vp = ctypes.c_void_p
_lock = threading.Lock()
_lib = None

# name -> argtypes (all return int status unless listed in _RESTYPES)
SIGNATURES = {
    "lf2_lattice_create": [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(_vp)],
    "lf2_lattice_destroy": [_vp],
    "lf2_lattice_sites": [_vp, ctypes.POINTER(ctypes.c_longlong)],
    "lf2_field_alloc": [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)],
    "lf2_field_wrap": [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp)],
    "lf2_field_free": [_vp],
    "lf2_field_buffer": [_vp, ctypes.c_int, ctypes.POINTER(_vp)],
    "lf2_field_upload": [_vp, ctypes.POINTER(ctypes.c_double), _vp],
    "lf2_field_download": [_vp, ctypes.POINTER(ctypes.c_double), _vp],
    "lf2_field_update_halo": [_vp, _vp],
    "lf2_power_spectrum": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _vp],
    "lf2_field_derivative": [_vp, _vp, ctypes.c_int, ctypes.c_double, _vp],
    "lf2_field_write": [_vp, ctypes.c_int, ctypes.c_char_p, _vp],
    "lf2_field_read": [_vp, ctypes.c_int, ctypes.c_char_p, _vp],
    "lf2_leapfrog_init": [_vp, _vp, ctypes.POINTER(lf2_params), _vp],
    "lf2_leapfrog": [_vp, _vp, ctypes.POINTER(lf2_params), ctypes.c_int, _vp],
    "lf2_leapfrog_ex": [_vp, _vp, ctypes.POINTER(lf2_params), ctypes.c_int, ctypes.POINTER(lf2_step_config), _vp],
    "lf2_energy": [_vp, _vp, ctypes.POINTER(lf2_params), ctypes.POINTER(lf2_energy_t), _vp],
    "lf2_energy_device": [_vp, _vp, ctypes.POINTER(lf2_params), _vp, _vp],
    "lf2_energy_noalloc": [_vp, _vp, ctypes.POINTER(lf2_params), ctypes.POINTER(lf2_energy_t), _vp],
    "lf2_leapfrog_energy": [_vp, _vp, ctypes.POINTER(lf2_params), ctypes.c_int, _vp, _vp],
    "lf2_field_check": [_vp, _vp],
    "lf2_debug_bounds": [ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int],
    "lf2_field_compare": [_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp],
    "lf2_ensemble_create": [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(lf2_params),
                            ctypes.POINTER(_vp)],
    "lf2_ensemble_run": [_vp, ctypes.c_int, _vp],
    "lf2_ensemble_tune": [_vp, ctypes.c_int, ctypes.POINTER(lf2_step_config), _vp],
    "lf2_ensemble_set_config": [_vp, ctypes.POINTER(lf2_step_config)],
    "lf2_ensemble_destroy": [_vp],
    "lf2_tune": [_vp, _vp, ctypes.POINTER(lf2_params), ctypes.c_int, ctypes.POINTER(lf2_step_config), _vp],
    "lf2_tune_lookup": [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.POINTER(lf2_step_config)],
    "lf2_status_string": [ctypes.c_int],
    "lf2_last_error": [],
    "lf2_version": [],
}
_RESTYPES = {"lf2_status_string": ctypes.c_char_p, "lf2_last_error": ctypes.c_char_p, "lf2_version": ctypes.c_char_p}


def load(path: str = LIB_PATH):
    """Loads liblf2.so; raises if it is missing (build it with paper_1508_05610_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"liblf2.so not built ({path}); run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, args in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = _RESTYPES.get(name, ctypes.c_int)
            _lib = lib
    return _lib


def _call(name, *args):
    lib = load()
    st = getattr(lib, name)(*args)
    if st != LF2_OK:
        raise LF2Error(st, name, lib.lf2_last_error().decode())
    return st


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def params(dx=1.0, dt=0.1, lam=1.0, eta=1.0, m2=0.0) -> lf2_params:
    return lf2_params(dx, dt, lam, eta, m2)


# --------------------------------------------------------------------- C-named calls
def lf2_lattice_create(sizes, dim=3, halo=1):
    arr = (ctypes.c_int * len(sizes))(*sizes)
    out = _vp()
    _call("lf2_lattice_create", dim, arr, halo, ctypes.byref(out))
    return out


def lf2_lattice_destroy(lat):
    _call("lf2_lattice_destroy", lat)


def lf2_lattice_sites(lat):
    out = ctypes.c_longlong()
    _call("lf2_lattice_sites", lat, ctypes.byref(out))
    return out.value


def lf2_field_alloc(lat, ncomp, prec):
    out = _vp()
    _call("lf2_field_alloc", lat, ncomp, prec, ctypes.byref(out))
    return out


def lf2_field_wrap(lat, ncomp, prec, dev_ptrs):
    arr = (_vp * len(dev_ptrs))(*dev_ptrs)
    out = _vp()
    _call("lf2_field_wrap", lat, ncomp, prec, arr, len(dev_ptrs), ctypes.byref(out))
    return out


def lf2_field_free(f):
    _call("lf2_field_free", f)


def lf2_field_buffer(f, which=0):
    out = _vp()
    _call("lf2_field_buffer", f, which, ctypes.byref(out))
    return out.value


def lf2_field_upload(f, host: np.ndarray, stream=None):
    a = np.ascontiguousarray(host, dtype=np.float64)
    _call("lf2_field_upload", f, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_ptr(stream))


def lf2_field_download(f, shape, stream=None, out=None) -> np.ndarray:
    a = np.empty(shape, dtype=np.float64) if out is None else out
    _call("lf2_field_download", f, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_ptr(stream))
    return a


def lf2_field_write(f, path, which=0, stream=None):
    _call("lf2_field_write", f, int(which), os.fsencode(path), _stream_ptr(stream))


def lf2_field_read(f, path, which=0, stream=None):
    _call("lf2_field_read", f, int(which), os.fsencode(path), _stream_ptr(stream))


def lf2_power_spectrum(f, comp=0, nbins=32, dx=1.0, stream=None):
    """(mean power, mean |k|, mode count) per shell b = floor(|m|), as numpy arrays; comp = -1 sums
    the components' powers."""
    power, kmean, count = np.zeros(nbins), np.zeros(nbins), np.zeros(nbins)
    dp = ctypes.POINTER(ctypes.c_double)
    _call("lf2_power_spectrum", f, int(comp), int(nbins), float(dx), power.ctypes.data_as(dp),
          kmean.ctypes.data_as(dp), count.ctypes.data_as(dp), _stream_ptr(stream))
    return power, kmean, count


def lf2_field_derivative(src, dst, dim, dx=1.0, stream=None):
    _call("lf2_field_derivative", src, dst, int(dim), float(dx), _stream_ptr(stream))


def lf2_field_update_halo(f, stream=None):
    _call("lf2_field_update_halo", f, _stream_ptr(stream))


def lf2_leapfrog_init(phi, pi, p: lf2_params, stream=None):
    _call("lf2_leapfrog_init", phi, pi, ctypes.byref(p), _stream_ptr(stream))


def lf2_leapfrog(phi, pi, p: lf2_params, nsteps, stream=None):
    _call("lf2_leapfrog", phi, pi, ctypes.byref(p), int(nsteps), _stream_ptr(stream))


def lf2_leapfrog_ex(phi, pi, p: lf2_params, nsteps, kernel=LF2_KERNEL_AUTO, tile_y=0, zchunk=0, depth=0,
                    stream=None, tile_x=0, cx=0, cluster=0):
    cfg = lf2_step_config(kernel, tile_x, tile_y, zchunk, depth, cx, cluster)
    _call("lf2_leapfrog_ex", phi, pi, ctypes.byref(p), int(nsteps), ctypes.byref(cfg), _stream_ptr(stream))


def lf2_energy(phi, pi, p: lf2_params, stream=None, ncomp=2) -> dict:
    e = lf2_energy_t()
    _call("lf2_energy", phi, pi, ctypes.byref(p), ctypes.byref(e), _stream_ptr(stream))
    return e.as_dict(ncomp)


def lf2_energy_device(phi, pi, p: lf2_params, dev_out_ptr, stream=None):
    """Enqueues the energy reduction; writes an lf2_energy_t record to device memory."""
    _call("lf2_energy_device", phi, pi, ctypes.byref(p), dev_out_ptr, _stream_ptr(stream))


def lf2_leapfrog_energy(phi, pi, p: lf2_params, nsteps, dev_records_ptr, stream=None):
    """nsteps leapfrog steps, one kernel each, that also write the energy record of the state at
    the start of every step (nsteps x 16 doubles of device memory at dev_records_ptr)."""
    _call("lf2_leapfrog_energy", phi, pi, ctypes.byref(p), int(nsteps), dev_records_ptr, _stream_ptr(stream))


def lf2_field_check(f, stream=None):
    """Raises LF2Error (LF2_ERR_TIMEOUT) if a grid barrier of the last multi-step
    lf2_leapfrog_energy run on f gave up."""
    _call("lf2_field_check", f, _stream_ptr(stream))


def lf2_debug_bounds(reset=False) -> int:
    """Index violations counted by the debug library (LF2Error LF2_ERR_UNSUPPORTED otherwise)."""
    n = ctypes.c_ulonglong(0)
    _call("lf2_debug_bounds", ctypes.byref(n), 1 if reset else 0)
    return int(n.value)


def lf2_field_compare(f, ref_ptr, ref_prec, which=0, stream=None) -> dict:
    """Error norms of buffer `which` of f against a device array (FP64 on the device):
    max_abs_diff, max_abs_ref, sum_sq_diff, sum_sq_ref, and the derived relmax / rel_l2."""
    out = (ctypes.c_double * 4)()
    _call("lf2_field_compare", f, int(which), ref_ptr, int(ref_prec), out, _stream_ptr(stream))
    d = {"max_abs_diff": out[0], "max_abs_ref": out[1], "sum_sq_diff": out[2], "sum_sq_ref": out[3]}
    d["relmax"] = out[0] / out[1] if out[1] > 0 else float("nan")
    d["rel_l2"] = (out[2] / out[3]) ** 0.5 if out[3] > 0 else float("nan")
    return d


ENERGY_RECORD_FIELDS = ["kinetic", "gradient", "potential", "total"] + [f"sum{a}" for a in range(6)] + \
    [f"sum_sq{a}" for a in range(6)]


def lf2_energy_noalloc(phi, pi, p: lf2_params, stream=None, ncomp=2) -> dict:
    """lf2_energy without any allocation (fixed scratch inside the library)."""
    e = lf2_energy_t()
    _call("lf2_energy_noalloc", phi, pi, ctypes.byref(p), ctypes.byref(e), _stream_ptr(stream))
    return e.as_dict(ncomp)


LF2_TUNE_FORCE, LF2_TUNE_ONE_STEP = 1, 2


def _cfg_dict(c):
    return {"kernel": c.kernel, "tile_x": c.tile_x, "tile_y": c.tile_y, "zchunk": c.zchunk, "depth": c.depth,
            "cx": c.cx, "cluster": c.cluster}


def lf2_tune(phi, pi, p: lf2_params, flags=0, stream=None) -> dict:
    """Times kernel configurations on a proxy of phi's lattice; returns the chosen one."""
    c = lf2_step_config()
    _call("lf2_tune", phi, pi, ctypes.byref(p), int(flags), ctypes.byref(c), _stream_ptr(stream))
    return _cfg_dict(c)


def lf2_tune_lookup(sizes, ncomp, prec) -> dict:
    arr = (ctypes.c_int * 3)(*sizes)
    c = lf2_step_config()
    _call("lf2_tune_lookup", arr, ncomp, prec, ctypes.byref(c))
    return _cfg_dict(c)


def lf2_ensemble_create(phis, pis, params_list):
    n = len(phis)
    a = (_vp * n)(*phis)
    b = (_vp * n)(*pis)
    c = (lf2_params * n)(*params_list)
    out = _vp()
    _call("lf2_ensemble_create", n, a, b, c, ctypes.byref(out))
    return out


def lf2_ensemble_run(e, nsteps, stream=None):
    _call("lf2_ensemble_run", e, int(nsteps), _stream_ptr(stream))


def lf2_ensemble_tune(e, flags=0, stream=None) -> dict:
    c = lf2_step_config()
    _call("lf2_ensemble_tune", e, int(flags), ctypes.byref(c), _stream_ptr(stream))
    return _cfg_dict(c)


def lf2_ensemble_set_config(e, kernel=LF2_KERNEL_TBLOCK, tile_x=0, tile_y=0, zchunk=0, depth=0, cx=0):
    c = lf2_step_config(kernel, tile_x, tile_y, zchunk, depth, cx)
    _call("lf2_ensemble_set_config", e, ctypes.byref(c))


def lf2_ensemble_destroy(e):
    _call("lf2_ensemble_destroy", e)


def lf2_status_string(s):
    return load().lf2_status_string(s).decode()


def lf2_last_error():
    return load().lf2_last_error().decode()


def lf2_version():
    return load().lf2_version().decode()


# ---------------------------------------------------------------- small conveniences
class System:
    """A lattice with its phi and pi fields (owned), for tests, smoke and bench.

    ``shape`` is (nx, ny, nz); host arrays are (nz, ny, nx, ncomp) float64."""

    def __init__(self, shape, ncomp, prec):
        self.shape = tuple(shape)
        self.ncomp = ncomp
        self.prec = PRECISIONS[prec] if isinstance(prec, str) else prec
        self.lat = lf2_lattice_create(self.shape)
        self.phi = lf2_field_alloc(self.lat, ncomp, self.prec)
        self.pi = lf2_field_alloc(self.lat, ncomp, self.prec)

    @property
    def host_shape(self):
        nx, ny, nz = self.shape
        return (nz, ny, nx, self.ncomp)

    def upload(self, phi, pi, stream=None):
        lf2_field_upload(self.phi, phi, stream)
        lf2_field_upload(self.pi, pi, stream)

    def download(self, stream=None):
        return (lf2_field_download(self.phi, self.host_shape, stream),
                lf2_field_download(self.pi, self.host_shape, stream))

    def close(self):
        if self.lat is not None:
            lf2_field_free(self.phi)
            lf2_field_free(self.pi)
            lf2_lattice_destroy(self.lat)
            self.lat = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
