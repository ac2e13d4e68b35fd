"""FP64 CPU oracle for the checkerboard SU(2)/SU(3) gauge sweep.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its binding) never imports it, and this package never
imports the product path.  The arithmetic lives in ``qcd_oracle.c`` (plain C,
FP64, full N x N complex matrices); this module only compiles it with gcc and
marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qcd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

HEATBATH = 0
OVERRELAX = 1
FIELD_LINKS = 0   # background as a phase on the dynamical y-links
FIELD_FROZEN = 1  # background on the frozen spatial links of the t = 0 slice

# -ffp-contract=off: no fused multiply-add, so the oracle rounds the same way
# on x86-64 and aarch64 hosts.
CFLAGS = ["-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
          "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wextra"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (skipped when up to date)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(os.path.join(_HERE, "qcd_oracle.h")))):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, i, d, u32, u64, l = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_uint32, ctypes.c_uint64, ctypes.c_long)
        P = ctypes.POINTER
        L.oracle_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
        L.oracle_uniform.argtypes = [u32]
        L.oracle_uniform.restype = d
        L.oracle_create.argtypes = [i, i, i, d, i, i, u32]
        L.oracle_create.restype = vp
        L.oracle_create_ex.argtypes = [i, i, i, d, i, i, u32, i]
        L.oracle_create_ex.restype = vp
        L.oracle_destroy.argtypes = [vp]
        L.oracle_set_threads.argtypes = [i]
        L.oracle_get_threads.argtypes = []
        L.oracle_get_threads.restype = i
        L.oracle_cold_start.argtypes = [vp]
        L.oracle_hot_start.argtypes = [vp, u64]
        L.oracle_sweep.argtypes = [vp, i, i, u64]
        L.oracle_phase.argtypes = [vp, i, i, i, u64]
        L.oracle_reunitarize.argtypes = [vp]
        L.oracle_measure.argtypes = [vp, P(d), P(d)]
        L.oracle_measure_bare.argtypes = [vp, P(d)]
        L.oracle_get_links.argtypes = [vp, P(d)]
        L.oracle_set_links.argtypes = [vp, P(d)]
        L.oracle_get_sweep.argtypes = [vp]
        L.oracle_get_sweep.restype = u32
        L.oracle_set_sweep.argtypes = [vp, u32]
        L.oracle_exhausted.argtypes = [vp]
        L.oracle_exhausted.restype = l
        L.oracle_staple.argtypes = [vp, l, i, P(d)]
        L.oracle_link_action.argtypes = [vp, l, i]
        L.oracle_link_action.restype = d
        L.oracle_link_update.argtypes = [vp, i, l, i, u64, P(d)]
        L.oracle_link_update.restype = i
        L.oracle_kp_samples.argtypes = [d, i, u64, l, P(d), P(i)]
        L.oracle_su2_samples.argtypes = [d, i, u64, l, P(d)]
        L.oracle_haar_samples.argtypes = [i, u64, l, P(d)]
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return lib().oracle_get_threads()


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(w: int) -> float:
    return lib().oracle_uniform(int(w) & 0xFFFFFFFF)


def kp_samples(alpha: float, nhit: int, seed: int, n: int):
    a0 = np.zeros(n, np.float64)
    tries = np.zeros(n, np.int32)
    lib().oracle_kp_samples(alpha, nhit, seed, n, _dptr(a0),
                            tries.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return a0, tries


def su2_samples(alpha: float, nhit: int, seed: int, n: int) -> np.ndarray:
    x = np.zeros((n, 4), np.float64)
    lib().oracle_su2_samples(alpha, nhit, seed, n, _dptr(x))
    return x


def haar_samples(N: int, seed: int, n: int) -> np.ndarray:
    """n Haar-random SU(N) matrices as complex (n, N, N)."""
    out = np.zeros((n, N, N, 2), np.float64)
    lib().oracle_haar_samples(N, seed, n, _dptr(out))
    return out[..., 0] + 1j * out[..., 1]


class OracleLattice:
    """One lattice held by the oracle, links in canonical order
    ``[t][z][y][x][mu][row][col]`` (x fastest), complex128."""

    def __init__(self, N: int, Ns: int, Nt: int, beta: float, flux: int = 0,
                 nhit: int = 10, lattice_id: int = 0, field_mode: int = FIELD_LINKS):
        self.N, self.Ns, self.Nt = N, Ns, Nt
        self.V = Ns ** 3 * Nt
        self.beta, self.flux, self.nhit, self.field_mode = beta, flux, nhit, field_mode
        h = lib().oracle_create_ex(N, Ns, Nt, beta, flux, nhit, lattice_id, field_mode)
        if not h:
            raise ValueError("oracle_create rejected the arguments")
        self._h = h

    def close(self) -> None:
        if self._h:
            lib().oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cold_start(self) -> None:
        lib().oracle_cold_start(self._h)

    def hot_start(self, seed: int) -> None:
        lib().oracle_hot_start(self._h, seed)

    def sweep(self, n_hb: int, n_or: int, seed: int) -> None:
        lib().oracle_sweep(self._h, n_hb, n_or, seed)

    def phase(self, kind: int, parity: int, mu: int, seed: int) -> None:
        lib().oracle_phase(self._h, kind, parity, mu, seed)

    def reunitarize(self) -> None:
        lib().oracle_reunitarize(self._h)

    def measure(self):
        p = (ctypes.c_double * 3)()
        l = (ctypes.c_double * 2)()
        lib().oracle_measure(self._h, p, l)
        return list(p), list(l)

    def measure_bare(self):
        p = (ctypes.c_double * 3)()
        lib().oracle_measure_bare(self._h, p)
        return list(p)

    @property
    def sweep_counter(self) -> int:
        return lib().oracle_get_sweep(self._h)

    @sweep_counter.setter
    def sweep_counter(self, v: int) -> None:
        lib().oracle_set_sweep(self._h, v)

    @property
    def exhausted(self) -> int:
        return lib().oracle_exhausted(self._h)

    def get_links(self) -> np.ndarray:
        out = np.zeros((self.V, 4, self.N, self.N, 2), np.float64)
        lib().oracle_get_links(self._h, _dptr(out))
        return out[..., 0] + 1j * out[..., 1]

    def set_links(self, links) -> None:
        a = np.asarray(links)
        if np.iscomplexobj(a):
            a = np.stack([a.real, a.imag], axis=-1)
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.size == self.V * 4 * self.N * self.N * 2
        lib().oracle_set_links(self._h, _dptr(a))

    def staple(self, s: int, mu: int) -> np.ndarray:
        out = np.zeros((self.N, self.N, 2), np.float64)
        lib().oracle_staple(self._h, s, mu, _dptr(out))
        return out[..., 0] + 1j * out[..., 1]

    def link_action(self, s: int, mu: int) -> float:
        return lib().oracle_link_action(self._h, s, mu)

    def link_update(self, kind: int, s: int, mu: int, seed: int):
        out = np.zeros((self.N, self.N, 2), np.float64)
        ex = lib().oracle_link_update(self._h, kind, s, mu, seed, _dptr(out))
        return out[..., 0] + 1j * out[..., 1], ex


def site_index(Ns: int, x: int, y: int, z: int, t: int) -> int:
    return x + Ns * (y + Ns * (z + Ns * t))


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(_LIB)
