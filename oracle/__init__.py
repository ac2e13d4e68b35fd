"""FP64 CPU oracle for the checkerboard SU(2)/SU(3) gauge sweep and for the
O(N) model sweep by multi-hit Metropolis.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its binding) never imports it, and this package never
imports the product path.  The arithmetic lives in ``qcd_oracle.c`` (plain C,
FP64, full N x N complex matrices) and ``on_oracle.c`` (the O(N) model); this
module only compiles them with gcc and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("qcd_oracle.c", "on_oracle.c")]
_HDRS = [os.path.join(_HERE, f) for f in ("qcd_oracle.h", "on_oracle.h")]
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
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(f) for f in _SRCS + _HDRS)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", *CFLAGS, "-o", tmp, *_SRCS, "-lm"]
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
        L.oracle_create_ex.argtypes = [i, i, i, d, i, i, i, u32, i]
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
        L.oracle_reunitarize_phase.argtypes = [vp, i, i]
        L.oracle_reunitarize_matrix.argtypes = [i, P(d)]
        L.oracle_measure_planes.argtypes = [vp, P(d)]
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
        L.on_create.argtypes = [i, i, i, d, d, d, i, u32]
        L.on_create.restype = vp
        L.on_destroy.argtypes = [vp]
        L.on_cold_start.argtypes = [vp]
        L.on_hot_start.argtypes = [vp, u64]
        L.on_phase.argtypes = [vp, i, u64]
        L.on_sweep.argtypes = [vp, i, u64]
        L.on_site_update.argtypes = [vp, l, u64, P(d)]
        L.on_site_update.restype = i
        L.on_local_action.argtypes = [vp, l, P(d)]
        L.on_local_action.restype = d
        L.on_action.argtypes = [vp]
        L.on_action.restype = d
        L.on_measure.argtypes = [vp, P(d)]
        L.on_get_field.argtypes = [vp, P(d)]
        L.on_set_field.argtypes = [vp, P(d)]
        L.on_get_sweep.argtypes = [vp]
        L.on_get_sweep.restype = u32
        L.on_set_sweep.argtypes = [vp, u32]
        L.on_accepted.argtypes = [vp]
        L.on_accepted.restype = ctypes.c_longlong
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


def reunitarize_matrix(m: np.ndarray) -> np.ndarray:
    """The reunitarization of one N x N complex matrix (a copy)."""
    N = m.shape[-1]
    a = np.ascontiguousarray(np.stack([m.real, m.imag], axis=-1), dtype=np.float64)
    lib().oracle_reunitarize_matrix(N, _dptr(a))
    return a[..., 0] + 1j * a[..., 1]


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
                 nhit: int = 10, lattice_id: int = 0, field_mode: int = FIELD_LINKS,
                 flux8: int = 0):
        self.N, self.Ns, self.Nt = N, Ns, Nt
        self.V = Ns ** 3 * Nt
        self.beta, self.flux, self.nhit, self.field_mode = beta, flux, nhit, field_mode
        self.flux8 = flux8
        h = lib().oracle_create_ex(N, Ns, Nt, beta, flux, flux8, nhit, lattice_id, field_mode)
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

    def reunitarize_phase(self, parity: int, mu: int) -> None:
        lib().oracle_reunitarize_phase(self._h, parity, mu)

    def measure_planes(self):
        """Mean plaquette of the planes (x,y), (x,z), (y,z), (x,t), (y,t),
        (z,t), effective links."""
        p = (ctypes.c_double * 6)()
        lib().oracle_measure_planes(self._h, p)
        return list(p)

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


class OracleON:
    """One O(N) model lattice held by the oracle, field in canonical order
    ``[t][z][y][x][c]`` (x fastest), float64 of shape (V, N)."""

    def __init__(self, N: int, Ns: int, Nt: int, kappa: float, lam: float, delta: float,
                 nhit: int = 100, lattice_id: int = 0):
        self.N, self.Ns, self.Nt = N, Ns, Nt
        self.V = Ns ** 3 * Nt
        self.kappa, self.lam, self.delta, self.nhit = kappa, lam, delta, nhit
        h = lib().on_create(N, Ns, Nt, kappa, lam, delta, nhit, lattice_id)
        if not h:
            raise ValueError("on_create rejected the arguments")
        self._h = h

    def close(self) -> None:
        if self._h:
            lib().on_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cold_start(self) -> None:
        lib().on_cold_start(self._h)

    def hot_start(self, seed: int) -> None:
        lib().on_hot_start(self._h, seed)

    def phase(self, parity: int, seed: int) -> None:
        lib().on_phase(self._h, parity, seed)

    def sweep(self, n: int, seed: int) -> None:
        lib().on_sweep(self._h, n, seed)

    def site_update(self, s: int, seed: int):
        out = np.zeros(4, np.float64)
        acc = lib().on_site_update(self._h, s, seed, _dptr(out))
        return out[: self.N], acc

    def local_action(self, s: int, phi) -> float:
        p = np.zeros(4, np.float64)
        p[: self.N] = phi
        return lib().on_local_action(self._h, s, _dptr(p))

    def action(self) -> float:
        return lib().on_action(self._h)

    def measure(self):
        out = (ctypes.c_double * 7)()
        lib().on_measure(self._h, out)
        return list(out)

    def get_field(self) -> np.ndarray:
        out = np.zeros((self.V, self.N), np.float64)
        lib().on_get_field(self._h, _dptr(out))
        return out

    def set_field(self, phi) -> None:
        a = np.ascontiguousarray(phi, dtype=np.float64)
        assert a.size == self.V * self.N
        lib().on_set_field(self._h, _dptr(a))

    @property
    def sweep_counter(self) -> int:
        return lib().on_get_sweep(self._h)

    @sweep_counter.setter
    def sweep_counter(self, v: int) -> None:
        lib().on_set_sweep(self._h, v)

    @property
    def accepted(self) -> int:
        return lib().on_accepted(self._h)


def site_index(Ns: int, x: int, y: int, z: int, t: int) -> int:
    return x + Ns * (y + Ns * (z + Ns * t))


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(_LIB)
