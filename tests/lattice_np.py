"""Brute-force numpy helpers for pins (test code, independent of the oracle's
C source and of the CUDA library).

Links are complex arrays ``U[s, mu, N, N]`` with s = x + Ns (y + Ns (z + Ns t)).
"""
import numpy as np


def coords(Ns, Nt, s):
    x = s % Ns
    y = (s // Ns) % Ns
    z = (s // Ns ** 2) % Ns
    t = s // Ns ** 3
    return [x, y, z, t]


def index(Ns, c):
    return c[0] + Ns * (c[1] + Ns * (c[2] + Ns * c[3]))


def shift(Ns, Nt, s, mu, step):
    c = coords(Ns, Nt, s)
    ext = Nt if mu == 3 else Ns
    c[mu] = (c[mu] + step) % ext
    return index(Ns, c)


def background(N, Ns, Nt, flux, s, mu, flux8=0):
    """B_mu(x) on y-links: exp(i p3 H3 + i p8 H8), H3 = diag(1, -1[, 0]),
    H8 = diag(1, 1, -2) (sqrt(3) lambda8, SU(3) only), p = 2 pi n x / Ns^2."""
    b = np.eye(N, dtype=complex)
    if mu == 1 and (flux or flux8):
        x = coords(Ns, Nt, s)[0]
        unit = 2 * np.pi * x / Ns ** 2
        h = np.array([1.0, -1.0, 0.0][:N]) * flux + (np.array([1.0, 1.0, -2.0]) * flux8 if N == 3 else 0.0)
        b = np.diag(np.exp(1j * unit * h))
    return b


def effective(U, Ns, Nt, flux, flux8=0):
    N = U.shape[-1]
    out = U.copy()
    if flux or flux8:
        for s in range(U.shape[0]):
            out[s, 1] = U[s, 1] @ background(N, Ns, Nt, flux, s, 1, flux8)
    return out


def plaquette_value(Ut, Ns, Nt, s, mu, nu):
    N = Ut.shape[-1]
    a = Ut[s, mu]
    b = Ut[shift(Ns, Nt, s, mu, 1), nu]
    c = Ut[shift(Ns, Nt, s, nu, 1), mu]
    d = Ut[s, nu]
    return np.trace(a @ b @ c.conj().T @ d.conj().T).real / N


def plaquettes(Ut, Ns, Nt):
    V = Ut.shape[0]
    ps = pt = 0.0
    for s in range(V):
        for mu in range(4):
            for nu in range(mu + 1, 4):
                p = plaquette_value(Ut, Ns, Nt, s, mu, nu)
                if nu == 3:
                    pt += p
                else:
                    ps += p
    return (ps + pt) / (6 * V), ps / (3 * V), pt / (3 * V)


def polyakov(Ut, Ns, Nt):
    N = Ut.shape[-1]
    V3 = Ns ** 3
    acc = 0j
    for sx in range(V3):
        p = np.eye(N, dtype=complex)
        for t in range(Nt):
            p = p @ Ut[sx + V3 * t, 3]
        acc += np.trace(p) / N
    return acc / V3


def link_plaquette_sum(Ut, Ns, Nt, s, mu, X):
    """Sum over the 6 plaquettes holding link (s, mu) of Re Tr, with the link
    replaced by X (real-linear in X)."""
    total = 0.0
    for nu in range(4):
        if nu == mu:
            continue
        s_pmu = shift(Ns, Nt, s, mu, 1)
        s_pnu = shift(Ns, Nt, s, nu, 1)
        s_mnu = shift(Ns, Nt, s, nu, -1)
        s_mnu_pmu = shift(Ns, Nt, s_mnu, mu, 1)
        # plaquette at x in the (mu, nu) plane
        total += np.trace(X @ Ut[s_pmu, nu] @ Ut[s_pnu, mu].conj().T @ Ut[s, nu].conj().T).real
        # plaquette at x - nu in the (mu, nu) plane, the link enters daggered
        total += np.trace(Ut[s_mnu, mu] @ Ut[s_mnu_pmu, nu] @ X.conj().T @ Ut[s_mnu, nu].conj().T).real
    return total


def staple_from_plaquettes(Ut, Ns, Nt, s, mu):
    """The matrix A with Re Tr(X A) = link_plaquette_sum(X) for all X:
    A_ji = f(E_ij) - i f(i E_ij)."""
    N = Ut.shape[-1]
    A = np.zeros((N, N), complex)
    for i in range(N):
        for j in range(N):
            E = np.zeros((N, N), complex)
            E[i, j] = 1.0
            A[j, i] = link_plaquette_sum(Ut, Ns, Nt, s, mu, E) - 1j * link_plaquette_sum(Ut, Ns, Nt, s, mu, 1j * E)
    return A


def unitarity_error(U):
    N = U.shape[-1]
    M = U.reshape(-1, N, N)
    e1 = np.abs(np.einsum("nki,nkj->nij", M.conj(), M) - np.eye(N)).max()
    e2 = np.abs(np.linalg.det(M) - 1.0).max()
    return e1, e2


def round_to_fp32_storage(U):
    """What FP32 storage keeps of links U[..., N, N]: SU(2) the quaternion
    entries (the first row and its mirror), SU(3) rows 1-2 rounded to FP32 with
    row 3 rebuilt as conj(row1 x row2) in FP64."""
    N = U.shape[-1]
    f32 = lambda z: z.real.astype(np.float32).astype(np.float64) + 1j * z.imag.astype(np.float32).astype(np.float64)
    R = np.array(U, dtype=complex)
    if N == 2:
        a, b = f32(U[..., 0, 0]), f32(U[..., 0, 1])
        R[..., 0, 0], R[..., 0, 1] = a, b
        R[..., 1, 0], R[..., 1, 1] = -np.conj(b), np.conj(a)
        return R
    R[..., :2, :] = f32(U[..., :2, :])
    R[..., 2, :] = np.conj(np.cross(R[..., 0, :], R[..., 1, :]))
    return R
