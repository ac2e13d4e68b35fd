"""Python binding of libqcdgb300 (include/qcd.h): the checkerboard Monte Carlo
sweep of SU(2)/SU(3) Wilson lattice gauge theory at finite temperature in a
constant Abelian background field, on one GB300.

Argument marshalling only: every step of the sweep and of the measurements
runs in the library's CUDA kernels.  There is no CPU fallback; when the
compiled library is missing every call raises.  PyTorch supplies the CUDA
stream (``torch.cuda.current_stream()`` unless one is given).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqcdgb300.so")

QCD_OK = 0
QCD_ERR_INVALID_ARG = -1
QCD_ERR_OOM = -2
QCD_ERR_CUDA = -3
QCD_ERR_TIMEOUT = -4
QCD_ERR_NOT_SUPPORTED = -5
QCD_FP64_PLAIN = 0
QCD_FP32_COMPRESSED = 1
QCD_COLD = 0
QCD_HOT = 1
QCD_HEATBATH = 0
QCD_OVERRELAX = 1
QCD_OVERRELAX_REUNIT = 2
QCD_OVERRELAX_MEASURE = 3
QCD_FIELD_LINKS = 0
QCD_FIELD_FROZEN = 1

# Every symbol include/qcd.h declares, with ctypes (restype, argtypes).
_vp, _i, _d, _u32, _u64, _sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t)
_P = ctypes.POINTER
SIGNATURES = {
    "qcd_lattice_create": (_i, [_P(_vp), _i, _i, _i, _d, _i, _i, _i, _u64, _vp]),
    "qcd_lattice_create_ex": (_i, [_P(_vp), _i, _i, _i, _d, _i, _i, _i, _i, _i, _u64, _vp]),
    "qcd_lattice_create_split": (_i, [_P(_vp), _i, _i, _i, _d, _i, _i, _i, _i, _i, _u64, _vp, _i]),
    "qcd_get_residency": (_i, [_vp, _P(_sz), _P(_sz), _P(_i)]),
    "qcd_lattice_destroy": (_i, [_vp]),
    "qcd_get_field_mode": (_i, [_vp, _P(_i)]),
    "qcd_set_nhit": (_i, [_vp, _i]),
    "qcd_sweep": (_i, [_vp, _i, _i, _u64]),
    "qcd_phase": (_i, [_vp, _i, _i, _i, _u64]),
    "qcd_measure_fused_finish": (_i, [_vp, _P(_d)]),
    "qcd_reunitarize": (_i, [_vp]),
    "qcd_measure": (_i, [_vp, _P(_d), _P(_d)]),
    "qcd_measure_async": (_i, [_vp, _vp]),
    "qcd_working_sweep": (_i, [_vp, _i, _i, _u64, _vp, _i]),
    "qcd_measure_bare": (_i, [_vp, _P(_d)]),
    "qcd_get_links": (_i, [_vp, _P(_d)]),
    "qcd_set_links": (_i, [_vp, _P(_d)]),
    "qcd_link_bytes": (_i, [_vp, _P(_sz)]),
    "qcd_copy_links_in": (_i, [_vp, _vp, _sz]),
    "qcd_copy_links_out": (_i, [_vp, _vp, _sz]),
    "qcd_get_sweep": (_i, [_vp, _P(_u32)]),
    "qcd_set_sweep": (_i, [_vp, _u32]),
    "qcd_get_exhausted": (_i, [_vp, _P(ctypes.c_ulonglong)]),
    "qcd_set_block": (_i, [_vp, _i]),
    "qcd_get_block": (_i, [_vp, _P(_i)]),
    "qcd_save": (_i, [_vp, ctypes.c_char_p]),
    "qcd_lattice_load": (_i, [_P(_vp), ctypes.c_char_p, _i, _vp]),
    "qcd_set_profiling": (_i, [_vp, _i]),
    "qcd_get_profile": (_i, [_vp, _P(_d), _P(ctypes.c_ulonglong)]),
    "qcd_measure_noalloc": (_i, [_vp, _sz, _i, _i, _i, _i, _i, _i, _P(_d), _P(_d), _vp]),
    "qcd_batch_create": (_i, [_P(_vp), _i, _i, _P(_i), _P(_i), _P(_d), _P(_i), _i, _i, _u64, _vp]),
    "qcd_batch_destroy": (_i, [_vp]),
    "qcd_batch_sweep": (_i, [_vp, _i, _i, _u64, _P(_d)]),
    "qcd_batch_get_links": (_i, [_vp, _i, _P(_d)]),
    "qcd_batch_set_links": (_i, [_vp, _i, _P(_d)]),
    "qcd_batch_get_sweep": (_i, [_vp, _P(_u32)]),
    "qcd_batch_link_bytes": (_i, [_vp, _P(_sz)]),
    "qcd_batch_set_block": (_i, [_vp, _i]),
    "qcd_batch_get_shape": (_i, [_vp, _P(_i), _P(_i)]),
    "qcd_batch_set_wait": (_i, [_vp, _d]),
    "qcd_batch_set_wave_bytes": (_i, [_vp, _sz]),
    "qcd_batch_get_waves": (_i, [_vp, _P(_i), _P(_sz)]),
    "qcd_batch_inject_stall": (_i, [_vp, _i]),
    "qcd_on_create": (_i, [_P(_vp), _i, _i, _i, _d, _d, _d, _i, _i, _u64, _vp]),
    "qcd_on_destroy": (_i, [_vp]),
    "qcd_on_set_nhit": (_i, [_vp, _i]),
    "qcd_on_set_block": (_i, [_vp, _i]),
    "qcd_on_sweep": (_i, [_vp, _i, _u64]),
    "qcd_on_phase": (_i, [_vp, _i, _u64]),
    "qcd_on_measure": (_i, [_vp, _P(_d)]),
    "qcd_on_get_field": (_i, [_vp, _P(_d)]),
    "qcd_on_set_field": (_i, [_vp, _P(_d)]),
    "qcd_on_get_sweep": (_i, [_vp, _P(_u32)]),
    "qcd_on_set_sweep": (_i, [_vp, _u32]),
    "qcd_on_get_accepted": (_i, [_vp, _P(ctypes.c_ulonglong)]),
    "qcd_probe_fp64_rate": (_i, [_P(_d), _vp]),
    "qcd_last_error": (ctypes.c_char_p, []),
}
QCD_NOALLOC_SCRATCH_BYTES = 512 * 1024
QCD_PROF_HEATBATH, QCD_PROF_OVERRELAX, QCD_PROF_REUNIT, QCD_PROF_MEASURE = 0, 1, 2, 3
QCD_PROF_N = 4


class QcdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("qcd error %d: %s" % (code, msg))
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libqcdgb300.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != QCD_OK:
        raise QcdError(rc, lib().qcd_last_error().decode())


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- the C ABI, one Python function per entry point ------------------------

def qcd_lattice_create(group, Ns, Nt, beta, flux=0, precision=QCD_FP32_COMPRESSED,
                       start=QCD_HOT, seed=1, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().qcd_lattice_create(ctypes.byref(h), group, Ns, Nt, beta, flux, precision,
                                    start, seed, _stream_handle(stream)))
    return h


def qcd_lattice_create_ex(group, Ns, Nt, beta, flux=0, flux8=0, field_mode=QCD_FIELD_LINKS,
                          precision=QCD_FP32_COMPRESSED, start=QCD_HOT, seed=1,
                          stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().qcd_lattice_create_ex(ctypes.byref(h), group, Ns, Nt, beta, flux, flux8, field_mode,
                                       precision, start, seed, _stream_handle(stream)))
    return h


def qcd_lattice_create_split(group, Ns, Nt, beta, flux=0, flux8=0, field_mode=QCD_FIELD_LINKS,
                             precision=QCD_FP32_COMPRESSED, start=QCD_HOT, seed=1, stream=None,
                             nt_device=0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().qcd_lattice_create_split(ctypes.byref(h), group, Ns, Nt, beta, flux, flux8, field_mode,
                                          precision, start, seed, _stream_handle(stream), nt_device))
    return h


def qcd_get_residency(h):
    """(device bytes, host bytes, leading t-slices wholly in device memory)."""
    d, hb, nt = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int()
    _check(lib().qcd_get_residency(h, ctypes.byref(d), ctypes.byref(hb), ctypes.byref(nt)))
    return d.value, hb.value, nt.value


def qcd_get_field_mode(h) -> int:
    v = ctypes.c_int()
    _check(lib().qcd_get_field_mode(h, ctypes.byref(v)))
    return v.value


def qcd_working_sweep(h, n_heatbath: int, n_overrelax: int, seed: int, host_out_ptr=None, wait: bool = True):
    """Sweeps and a measurement of the result.  Without host_out_ptr (or with
    wait) the five results {P, P_s, P_t, Re L, Im L} are returned."""
    if host_out_ptr is None:
        out = (ctypes.c_double * 5)()
        _check(lib().qcd_working_sweep(h, n_heatbath, n_overrelax, seed, ctypes.cast(out, ctypes.c_void_p), 1))
        return list(out)
    _check(lib().qcd_working_sweep(h, n_heatbath, n_overrelax, seed, host_out_ptr, 1 if wait else 0))
    return None


def qcd_measure_async(h, host_out_ptr: int) -> None:
    """Enqueue the measurement; the five doubles land at host_out_ptr once the
    lattice's stream is synchronized."""
    _check(lib().qcd_measure_async(h, host_out_ptr))


def qcd_lattice_destroy(h) -> None:
    _check(lib().qcd_lattice_destroy(h))


def qcd_set_nhit(h, nhit: int) -> None:
    _check(lib().qcd_set_nhit(h, nhit))


def qcd_sweep(h, n_heatbath: int, n_overrelax: int, seed: int) -> None:
    _check(lib().qcd_sweep(h, n_heatbath, n_overrelax, seed))


def qcd_phase(h, kind: int, parity: int, mu: int, seed: int) -> None:
    _check(lib().qcd_phase(h, kind, parity, mu, seed))


def qcd_measure_fused_finish(h):
    """[P, P_s, P_t, Re L, Im L, P_1, P_2, P_3] of a last pass run phase by
    phase with qcd_phase (P_mu: mean plaquette of the planes (mu, nu < mu))."""
    out = (ctypes.c_double * 8)()
    _check(lib().qcd_measure_fused_finish(h, out))
    return list(out)


def qcd_reunitarize(h) -> None:
    _check(lib().qcd_reunitarize(h))


def qcd_measure(h):
    p = (ctypes.c_double * 3)()
    l = (ctypes.c_double * 2)()
    _check(lib().qcd_measure(h, p, l))
    return list(p), list(l)


def qcd_measure_bare(h):
    p = (ctypes.c_double * 3)()
    _check(lib().qcd_measure_bare(h, p))
    return list(p)


def qcd_get_links(h, V: int, N: int) -> np.ndarray:
    out = np.empty((V, 4, N, N, 2), np.float64)
    _check(lib().qcd_get_links(h, _dptr(out)))
    return out[..., 0] + 1j * out[..., 1]


def qcd_set_links(h, links) -> None:
    a = np.asarray(links)
    if np.iscomplexobj(a):
        a = np.stack([a.real, a.imag], axis=-1)
    a = np.ascontiguousarray(a, dtype=np.float64)
    _check(lib().qcd_set_links(h, _dptr(a)))


def qcd_link_bytes(h) -> int:
    n = ctypes.c_size_t()
    _check(lib().qcd_link_bytes(h, ctypes.byref(n)))
    return n.value


def qcd_copy_links_in(h, host_ptr: int, nbytes: int) -> None:
    _check(lib().qcd_copy_links_in(h, host_ptr, nbytes))


def qcd_copy_links_out(h, host_ptr: int, nbytes: int) -> None:
    _check(lib().qcd_copy_links_out(h, host_ptr, nbytes))


def qcd_get_sweep(h) -> int:
    v = ctypes.c_uint32()
    _check(lib().qcd_get_sweep(h, ctypes.byref(v)))
    return v.value


def qcd_set_sweep(h, sweep: int) -> None:
    _check(lib().qcd_set_sweep(h, sweep))


def qcd_get_exhausted(h) -> int:
    v = ctypes.c_ulonglong()
    _check(lib().qcd_get_exhausted(h, ctypes.byref(v)))
    return v.value


def qcd_set_block(h, threads: int) -> None:
    _check(lib().qcd_set_block(h, threads))


def qcd_get_block(h) -> int:
    v = ctypes.c_int()
    _check(lib().qcd_get_block(h, ctypes.byref(v)))
    return v.value


def qcd_save(h, path: str) -> None:
    _check(lib().qcd_save(h, os.fsencode(path)))


def qcd_lattice_load(path: str, precision=QCD_FP32_COMPRESSED, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().qcd_lattice_load(ctypes.byref(h), os.fsencode(path), precision, _stream_handle(stream)))
    return h


def qcd_set_profiling(h, enable: bool) -> None:
    _check(lib().qcd_set_profiling(h, int(bool(enable))))


def qcd_get_profile(h):
    """(ms[QCD_PROF_N], launches[QCD_PROF_N]) accumulated since profiling was
    enabled: heat-bath, overrelaxation, reunitarization, measurement."""
    ms = (ctypes.c_double * QCD_PROF_N)()
    n = (ctypes.c_ulonglong * QCD_PROF_N)()
    _check(lib().qcd_get_profile(h, ms, n))
    return list(ms), list(n)


def qcd_measure_noalloc(links_dev_ptr: int, link_bytes: int, group: int, precision: int, Ns: int, Nt: int,
                        flux: int = 0, flux8: int = 0, stream=None):
    """Measurement that allocates nothing, on link storage the caller holds on
    the device (``links_dev_ptr``, ``link_bytes`` bytes in the layout
    qcd_copy_links_out produces).  Returns ([P, P_s, P_t], [Re L, Im L])."""
    p = (ctypes.c_double * 3)()
    l = (ctypes.c_double * 2)()
    _check(lib().qcd_measure_noalloc(links_dev_ptr, link_bytes, group, precision, Ns, Nt, flux, flux8, p, l,
                                     _stream_handle(stream)))
    return list(p), list(l)


def qcd_probe_fp64_rate(stream=None) -> float:
    """Measured FP64 FMA rate of the current device, flops/s."""
    v = ctypes.c_double()
    _check(lib().qcd_probe_fp64_rate(ctypes.byref(v), _stream_handle(stream)))
    return v.value


def qcd_last_error() -> str:
    return lib().qcd_last_error().decode()


def qcd_batch_create(group, Ns, Nt, beta, flux, precision=QCD_FP32_COMPRESSED, start=QCD_HOT,
                     seed=1, stream=None) -> ctypes.c_void_p:
    n = len(Ns)
    h = ctypes.c_void_p()
    ia = lambda v: (ctypes.c_int * n)(*[int(x) for x in v])
    _check(lib().qcd_batch_create(ctypes.byref(h), n, group, ia(Ns), ia(Nt),
                                  (ctypes.c_double * n)(*[float(x) for x in beta]), ia(flux),
                                  precision, start, seed, _stream_handle(stream)))
    return h


def qcd_batch_destroy(h) -> None:
    _check(lib().qcd_batch_destroy(h))


def qcd_batch_sweep(h, n: int, n_sweeps: int, n_overrelax: int, seed: int, measure: bool = True):
    """Returns the measurements as an (n, n_sweeps, 5) array (or None)."""
    out = np.empty((n, n_sweeps, 5), np.float64) if measure else None
    _check(lib().qcd_batch_sweep(h, n_sweeps, n_overrelax, seed, _dptr(out) if measure else None))
    return out


def qcd_batch_get_links(h, index: int, V: int) -> np.ndarray:
    out = np.empty((V, 4, 2, 2, 2), np.float64)
    _check(lib().qcd_batch_get_links(h, index, _dptr(out)))
    return out[..., 0] + 1j * out[..., 1]


def qcd_batch_set_links(h, index: int, links) -> None:
    a = np.asarray(links)
    if np.iscomplexobj(a):
        a = np.stack([a.real, a.imag], axis=-1)
    _check(lib().qcd_batch_set_links(h, index, _dptr(np.ascontiguousarray(a, dtype=np.float64))))


def qcd_batch_get_sweep(h) -> int:
    v = ctypes.c_uint32()
    _check(lib().qcd_batch_get_sweep(h, ctypes.byref(v)))
    return v.value


def qcd_batch_link_bytes(h) -> int:
    v = ctypes.c_size_t()
    _check(lib().qcd_batch_link_bytes(h, ctypes.byref(v)))
    return v.value


def qcd_batch_set_block(h, threads: int) -> None:
    _check(lib().qcd_batch_set_block(h, threads))


def qcd_batch_get_shape(h):
    t, c = ctypes.c_int(), ctypes.c_int()
    _check(lib().qcd_batch_get_shape(h, ctypes.byref(t), ctypes.byref(c)))
    return t.value, c.value


def qcd_batch_set_wave_bytes(h, nbytes: int) -> None:
    _check(lib().qcd_batch_set_wave_bytes(h, nbytes))


def qcd_batch_get_waves(h):
    """(number of waves, wave budget in bytes)."""
    w, b = ctypes.c_int(), ctypes.c_size_t()
    _check(lib().qcd_batch_get_waves(h, ctypes.byref(w), ctypes.byref(b)))
    return w.value, b.value


def qcd_batch_set_wait(h, seconds: float) -> None:
    _check(lib().qcd_batch_set_wait(h, seconds))


def qcd_batch_inject_stall(h, lattice: int) -> None:
    _check(lib().qcd_batch_inject_stall(h, lattice))


class Batch:
    """Owning wrapper around one ``qcd_batch`` handle (SU(2) lattices)."""

    def __init__(self, Ns, Nt, beta, flux, precision=QCD_FP32_COMPRESSED, start=QCD_HOT, seed=1,
                 stream=None):
        self.Ns, self.Nt = list(Ns), list(Nt)
        self.n = len(self.Ns)
        self.V = [ns ** 3 * nt for ns, nt in zip(self.Ns, self.Nt)]
        self.seed = seed
        self.h = qcd_batch_create(2, Ns, Nt, beta, flux, precision, start, seed, stream)

    def close(self):
        if self.h:
            qcd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n_sweeps=1, n_or=1, seed=None, measure=True):
        return qcd_batch_sweep(self.h, self.n, n_sweeps, n_or, self.seed if seed is None else seed, measure)

    def get_links(self, i):
        return qcd_batch_get_links(self.h, i, self.V[i])

    def set_links(self, i, links):
        qcd_batch_set_links(self.h, i, links)

    @property
    def sweep_counter(self):
        return qcd_batch_get_sweep(self.h)


class Lattice:
    """Owning wrapper around one ``qcd_lattice`` handle."""

    def __init__(self, group, Ns, Nt, beta, flux=0, precision=QCD_FP32_COMPRESSED,
                 start=QCD_HOT, seed=1, stream=None, nhit=10, field_mode=QCD_FIELD_LINKS, flux8=0,
                 nt_device=None):
        """nt_device: None for a device-resident lattice, else the number of
        leading t-slices kept in device memory (the rest in host memory)."""
        self.group, self.Ns, self.Nt = group, Ns, Nt
        self.V = Ns ** 3 * Nt
        self.beta, self.flux, self.precision, self.seed = beta, flux, precision, seed
        self.field_mode, self.flux8 = field_mode, flux8
        if nt_device is None:
            self.h = qcd_lattice_create_ex(group, Ns, Nt, beta, flux, flux8, field_mode, precision, start,
                                           seed, stream)
        else:
            self.h = qcd_lattice_create_split(group, Ns, Nt, beta, flux, flux8, field_mode, precision, start,
                                              seed, stream, nt_device)
        if nhit != 10:
            qcd_set_nhit(self.h, nhit)

    def close(self):
        if self.h:
            qcd_lattice_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n_hb=1, n_or=1, seed=None):
        qcd_sweep(self.h, n_hb, n_or, self.seed if seed is None else seed)

    def phase(self, kind, parity, mu, seed=None):
        qcd_phase(self.h, kind, parity, mu, self.seed if seed is None else seed)

    def reunitarize(self):
        qcd_reunitarize(self.h)

    def measure(self):
        return qcd_measure(self.h)

    def measure_bare(self):
        return qcd_measure_bare(self.h)

    def get_links(self):
        return qcd_get_links(self.h, self.V, self.group)

    def set_links(self, links):
        qcd_set_links(self.h, links)

    @property
    def sweep_counter(self):
        return qcd_get_sweep(self.h)

    @sweep_counter.setter
    def sweep_counter(self, v):
        qcd_set_sweep(self.h, v)

    def save(self, path):
        qcd_save(self.h, path)

    @classmethod
    def load(cls, path, precision=QCD_FP32_COMPRESSED, stream=None):
        """A lattice restored from a checkpoint written by ``save``."""
        import struct
        with open(path, "rb") as f:
            head = f.read(80)
        group, _, Ns, Nt, flux = struct.unpack_from("<IIIIi", head, 12)
        seed, beta = struct.unpack_from("<Qd", head, 48)
        flux8 = struct.unpack_from("<i", head, 72)[0] if len(head) >= 76 else 0
        self = cls.__new__(cls)
        self.group, self.Ns, self.Nt = group, Ns, Nt
        self.V = Ns ** 3 * Nt
        self.beta, self.flux, self.precision, self.seed = beta, flux, precision, seed
        self.h = qcd_lattice_load(path, precision, stream)
        self.field_mode = qcd_get_field_mode(self.h)
        self.flux8 = flux8
        return self

    @property
    def exhausted(self):
        return qcd_get_exhausted(self.h)

    @property
    def link_bytes(self):
        return qcd_link_bytes(self.h)


# ---------------------------------------------------------------------------
# O(N) model
# ---------------------------------------------------------------------------
def qcd_on_create(N, Ns, Nt, kappa, lam, delta, precision=QCD_FP32_COMPRESSED, start=QCD_HOT, seed=1,
                  stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().qcd_on_create(ctypes.byref(h), N, Ns, Nt, kappa, lam, delta, precision, start, seed,
                               _stream_handle(stream)))
    return h


def qcd_on_destroy(h) -> None:
    _check(lib().qcd_on_destroy(h))


def qcd_on_set_nhit(h, nhit: int) -> None:
    _check(lib().qcd_on_set_nhit(h, nhit))


def qcd_on_set_block(h, threads: int) -> None:
    _check(lib().qcd_on_set_block(h, threads))


def qcd_on_sweep(h, n_sweeps: int, seed: int) -> None:
    _check(lib().qcd_on_sweep(h, n_sweeps, seed))


def qcd_on_phase(h, parity: int, seed: int) -> None:
    _check(lib().qcd_on_phase(h, parity, seed))


def qcd_on_measure(h):
    out = (ctypes.c_double * 7)()
    _check(lib().qcd_on_measure(h, out))
    return list(out)


def qcd_on_get_field(h, V: int, N: int) -> np.ndarray:
    out = np.zeros((V, N), np.float64)
    _check(lib().qcd_on_get_field(h, _dptr(out)))
    return out


def qcd_on_set_field(h, phi) -> None:
    a = np.ascontiguousarray(phi, dtype=np.float64)
    _check(lib().qcd_on_set_field(h, _dptr(a)))


def qcd_on_get_sweep(h) -> int:
    v = ctypes.c_uint32()
    _check(lib().qcd_on_get_sweep(h, ctypes.byref(v)))
    return v.value


def qcd_on_set_sweep(h, sweep: int) -> None:
    _check(lib().qcd_on_set_sweep(h, sweep))


def qcd_on_get_accepted(h) -> int:
    v = ctypes.c_ulonglong()
    _check(lib().qcd_on_get_accepted(h, ctypes.byref(v)))
    return v.value


class ONModel:
    """Owning wrapper around one ``qcd_on`` handle (O(N) model, N <= 4)."""

    def __init__(self, N, Ns, Nt, kappa, lam, delta, precision=QCD_FP32_COMPRESSED, start=QCD_HOT, seed=1,
                 stream=None, nhit=100):
        self.N, self.Ns, self.Nt = N, Ns, Nt
        self.V = Ns ** 3 * Nt
        self.kappa, self.lam, self.delta, self.precision, self.seed = kappa, lam, delta, precision, seed
        self.h = qcd_on_create(N, Ns, Nt, kappa, lam, delta, precision, start, seed, stream)
        if nhit != 100:
            qcd_on_set_nhit(self.h, nhit)

    def close(self):
        if self.h:
            qcd_on_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1, seed=None):
        qcd_on_sweep(self.h, n, self.seed if seed is None else seed)

    def phase(self, parity, seed=None):
        qcd_on_phase(self.h, parity, self.seed if seed is None else seed)

    def measure(self):
        return qcd_on_measure(self.h)

    def get_field(self):
        return qcd_on_get_field(self.h, self.V, self.N)

    def set_field(self, phi):
        qcd_on_set_field(self.h, phi)

    @property
    def sweep_counter(self):
        return qcd_on_get_sweep(self.h)

    @sweep_counter.setter
    def sweep_counter(self, v):
        qcd_on_set_sweep(self.h, v)

    @property
    def accepted(self):
        return qcd_on_get_accepted(self.h)
