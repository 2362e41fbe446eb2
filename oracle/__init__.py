"""Plain FP64 CPU oracle for the sn-K build (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  It shares no code with the CUDA path: its
arithmetic lives in ``snk_oracle.c`` (plain C, double precision), compiled here
with gcc into ``_build/liboracle.so`` and called through ctypes.

Every routine follows a definition or the method's steps as the paper states
them (sections and equations cited in ``snk_oracle.c``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile snk_oracle.c with gcc (OpenMP, -O2, IEEE arithmetic)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.oracle_boys.argtypes = [ctypes.c_int, ctypes.c_double, _D]
            L.oracle_boys.restype = None
            for name in ("oracle_prim_A_os", "oracle_prim_A_md"):
                f = getattr(L, name)
                f.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_double, _D, ctypes.c_double, _D, _D]
                f.restype = ctypes.c_int
            L.oracle_prim_eri_md.argtypes = [ctypes.c_int] * 4 + [_D, ctypes.c_double] * 4 + [_D]
            L.oracle_prim_eri_md.restype = ctypes.c_int
            basis_args = [ctypes.c_int, _I, _I, _D, _D, _D]
            L.oracle_normalise.argtypes = basis_args + [_D, _D]
            L.oracle_collocation.argtypes = basis_args + [ctypes.c_long, _D, _D]
            L.oracle_shell_A.argtypes = basis_args + [ctypes.c_int, ctypes.c_int, _D, ctypes.c_int, _D]
            L.oracle_eri_K.argtypes = basis_args + [_D, _D]
            L.oracle_snk_K.argtypes = basis_args + [ctypes.c_long, _D, _D, _D, _D, ctypes.c_int]
            L.oracle_snk_K_entries.argtypes = basis_args + [ctypes.c_long, _D, _D, _D, ctypes.c_int,
                                                            _I, _I, _D, ctypes.c_int]
            L.oracle_g_rows.argtypes = basis_args + [ctypes.c_long, _D, _D, _D, ctypes.c_int, _I, _D,
                                                     ctypes.c_int]
            L.oracle_xc_point.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _D]
            L.oracle_collocation_grad.argtypes = basis_args + [ctypes.c_long, _D, _D, _D]
            L.oracle_vxc.argtypes = basis_args + [ctypes.c_long, _D, _D, _D, ctypes.c_int, _D, _D, ctypes.c_int]
            L.oracle_vxc_entries.argtypes = basis_args + [ctypes.c_long, _D, _D, _D, ctypes.c_int, ctypes.c_int,
                                                          _I, _I, _D, _D, ctypes.c_int]
            L.oracle_mlp_forward.argtypes = [_D, _D, ctypes.c_long, _D]
            L.oracle_mlp_loss_grad.argtypes = [_D, _D, _D, ctypes.c_long, ctypes.c_double, _D, _D]
            for name in ("oracle_normalise", "oracle_collocation", "oracle_shell_A", "oracle_eri_K",
                         "oracle_snk_K", "oracle_snk_K_entries", "oracle_g_rows", "oracle_mlp_forward", "oracle_mlp_loss_grad",
                         "oracle_xc_point", "oracle_collocation_grad", "oracle_vxc", "oracle_vxc_entries"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _basis_args(basis):
    arrs = (_i32(basis.l), _i32(basis.nprim), _f64(basis.center), _f64(basis.exps), _f64(basis.coefs))
    return arrs, [ctypes.c_int(int(arrs[0].shape[0])), _ip(arrs[0]), _ip(arrs[1]), _dp(arrs[2]),
                  _dp(arrs[3]), _dp(arrs[4])]


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def boys(nmax: int, T: float) -> np.ndarray:
    out = np.zeros(nmax + 1)
    lib().oracle_boys(nmax, float(T), _dp(out))
    return out


def prim_A(la, lb, A, alpha, B, beta, C, method="os") -> np.ndarray:
    """3c-CP integrals over raw primitives (no normalisation), (ncart(la), ncart(lb))."""
    out = np.zeros(ncart(la) * ncart(lb))
    f = lib().oracle_prim_A_os if method == "os" else lib().oracle_prim_A_md
    _check(f(la, lb, _dp(_f64(A)), float(alpha), _dp(_f64(B)), float(beta), _dp(_f64(C)), _dp(out)), "prim_A")
    return out.reshape(ncart(la), ncart(lb))


def prim_eri(ls, centers, exps) -> np.ndarray:
    """(ab|cd) over raw primitives by McMurchie-Davidson."""
    out = np.zeros(int(np.prod([ncart(l) for l in ls])))
    keep = [_f64(c) for c in centers]
    args = []
    for c, e in zip(keep, exps):
        args += [_dp(c), float(e)]
    _check(lib().oracle_prim_eri_md(*[int(l) for l in ls], *args, _dp(out)), "prim_eri")
    return out.reshape([ncart(l) for l in ls])


def normalise(basis):
    keep, args = _basis_args(basis)
    d = np.zeros(int(np.sum(basis.nprim)))
    nf = int(sum(ncart(int(l)) for l in basis.l))
    f = np.zeros(nf)
    _check(lib().oracle_normalise(*args, _dp(d), _dp(f)), "normalise")
    return d, f


def collocation(basis, xyz) -> np.ndarray:
    """Phi (n_points, n_functions), Eq. (collocation)."""
    keep, args = _basis_args(basis)
    xyz = _f64(xyz).reshape(-1, 3)
    nf = int(sum(ncart(int(l)) for l in basis.l))
    out = np.zeros((xyz.shape[0], nf))
    _check(lib().oracle_collocation(*args, ctypes.c_long(xyz.shape[0]), _dp(xyz), _dp(out)), "collocation")
    return out


def shell_A(basis, sa, sb, C, method="os") -> np.ndarray:
    """A_{mu lambda}(C) for the contracted normalised shells sa, sb."""
    keep, args = _basis_args(basis)
    out = np.zeros(ncart(int(basis.l[sa])) * ncart(int(basis.l[sb])))
    _check(lib().oracle_shell_A(*args, int(sa), int(sb), _dp(_f64(C)), 0 if method == "os" else 1, _dp(out)),
           "shell_A")
    return out.reshape(ncart(int(basis.l[sa])), ncart(int(basis.l[sb])))


def eri_K(basis, P) -> np.ndarray:
    """Exact exchange K_{mu nu} = sum (mu lambda|nu kappa) P_{lambda kappa}."""
    keep, args = _basis_args(basis)
    P = _f64(P)
    K = np.zeros_like(P)
    _check(lib().oracle_eri_K(*args, _dp(P), _dp(K)), "eri_K")
    return K


def snk_K(basis, grid, P, nthreads: int = 0) -> np.ndarray:
    """Unscreened sn-K, Eqs. (collocation), (fmat), (gmat), (usym_k), (sn_k)."""
    keep, args = _basis_args(basis)
    xyz, w, P = _f64(grid.xyz), _f64(grid.w), _f64(P)
    K = np.zeros_like(P)
    _check(lib().oracle_snk_K(*args, ctypes.c_long(w.shape[0]), _dp(xyz), _dp(w), _dp(P), _dp(K),
                              int(nthreads)), "snk_K")
    return K


def snk_K_entries(basis, grid, P, mu, nu, nthreads: int = 0) -> np.ndarray:
    """K_{mu_k nu_k} of the unscreened sn-K build, for the listed entries."""
    keep, args = _basis_args(basis)
    xyz, w, P = _f64(grid.xyz), _f64(grid.w), _f64(P)
    mu, nu = _i32(mu), _i32(nu)
    out = np.zeros(mu.shape[0])
    _check(lib().oracle_snk_K_entries(*args, ctypes.c_long(w.shape[0]), _dp(xyz), _dp(w), _dp(P),
                                      int(mu.shape[0]), _ip(mu), _ip(nu), _dp(out), int(nthreads)),
           "snk_K_entries")
    return out


def snk_K_entries_blocked(basis, grid, P, mu, nu, block: int = 16384, nthreads: int = 0,
                          progress=None) -> np.ndarray:
    """The same entries as snk_K_entries, over blocks of grid points: per
    block Phi (Eq. collocation, oracle C), F = Phi P (Eq. fmat) as a library
    matrix product, the G rows of the wanted functions (Eq. gmat, oracle C),
    and the partial sums Kt_{mu nu} = sum_i G_{mu i} Phi_{nu i} (Eq. usym_k);
    finally K = (Kt + Kt^T) / 2 per entry (Eq. sn_k).  For grids where
    streaming P once per point would dominate."""
    keep, args = _basis_args(basis)
    mu, nu = _i32(mu), _i32(nu)
    P = _f64(P)
    funs = np.unique(np.concatenate([mu, nu])).astype(np.int32)
    col = {int(f): t for t, f in enumerate(funs)}
    im = np.array([col[int(x)] for x in mu], dtype=np.int64)
    inn = np.array([col[int(x)] for x in nu], dtype=np.int64)
    s1 = np.zeros(mu.shape[0])
    s2 = np.zeros(mu.shape[0])
    n = grid.w.shape[0]
    for i0 in range(0, n, block):
        xyz = _f64(grid.xyz[i0:i0 + block]).reshape(-1, 3)
        w = _f64(grid.w[i0:i0 + block])
        phi = collocation(basis, xyz)                 # (b, nf)
        F = np.ascontiguousarray(phi @ P.T)            # F[i][lam] = sum_nu P_{lam nu} Phi_{nu i}
        G = np.zeros((w.shape[0], funs.shape[0]))
        _check(lib().oracle_g_rows(*args, ctypes.c_long(w.shape[0]), _dp(xyz), _dp(w), _dp(F),
                                   int(funs.shape[0]), _ip(funs), _dp(G), int(nthreads)), "g_rows")
        ph = phi[:, funs]
        s1 += np.einsum("ik,ik->k", G[:, im], ph[:, inn])
        s2 += np.einsum("ik,ik->k", G[:, inn], ph[:, im])
        if progress is not None:
            progress(min(n, i0 + block), n)
    return 0.5 * (s1 + s2)


MLP_WEIGHTS = 16 * 64 + 64 + 2 * (64 * 64 + 64) + 64 + 1


def mlp_forward(w, X) -> np.ndarray:
    """Learned-screen MLP output for each row of X (n x 16), FP64."""
    w, X = _f64(w), _f64(X).reshape(-1, 16)
    out = np.zeros(X.shape[0])
    _check(lib().oracle_mlp_forward(_dp(w), _dp(X), ctypes.c_long(X.shape[0]), _dp(out)), "mlp_forward")
    return out


def mlp_loss_grad(w, X, Y, under_weight=4.0):
    """Asymmetric squared-error loss and its gradient by backpropagation, FP64."""
    w, X, Y = _f64(w), _f64(X).reshape(-1, 16), _f64(Y).reshape(-1)
    g = np.zeros(MLP_WEIGHTS)
    loss = np.zeros(1)
    _check(lib().oracle_mlp_loss_grad(_dp(w), _dp(X), _dp(Y), ctypes.c_long(X.shape[0]), float(under_weight),
                                      _dp(g), _dp(loss)), "mlp_loss_grad")
    return float(loss[0]), g


# ---------------------------------------------------------------- exchange-correlation (Sec. II.C)

XC_LDA_X, XC_PBE_X, XC_PBE = 1, 2, 3


def xc_point(functional: int, rho: float, sigma: float) -> np.ndarray:
    """(eps, d eps / d rho, d eps / d sigma) of a spin-restricted functional
    (1 Slater exchange, 2 PBE exchange, 3 PBE exchange + correlation); eps is
    the energy per volume, sigma = |grad rho|^2 (Eq. exc_grid)."""
    out = np.zeros(3)
    _check(lib().oracle_xc_point(int(functional), float(rho), float(sigma), _dp(out)), "xc_point")
    return out


def collocation_grad(basis, xyz):
    """Phi (npts, nf) and grad Phi (npts, 3, nf) at the points (Eq. collocation)."""
    arrs, args = _basis_args(basis)
    xyz = _f64(xyz).reshape(-1, 3)
    nf = sum(ncart(int(x)) for x in arrs[0])
    phi = np.zeros((xyz.shape[0], nf))
    gphi = np.zeros((xyz.shape[0], 3, nf))
    _check(lib().oracle_collocation_grad(*args, ctypes.c_long(xyz.shape[0]), _dp(xyz), _dp(phi), _dp(gphi)),
           "collocation_grad")
    return phi, gphi


def vxc(basis, grid, P, functional: int, nthreads: int = 0):
    """(V^xc, E_xc) of the symmetric density matrix P on the grid: Eqs. fmat,
    den_grid, exc_grid, zmat and vxc_num, point by point, no screening."""
    arrs, args = _basis_args(basis)
    xyz, w, P = _f64(grid.xyz), _f64(grid.w), _f64(P)
    nf = P.shape[0]
    V = np.zeros((nf, nf))
    E = np.zeros(1)
    _check(lib().oracle_vxc(*args, ctypes.c_long(w.shape[0]), _dp(xyz), _dp(w), _dp(P), int(functional), _dp(V),
                            _dp(E), int(nthreads)), "vxc")
    return V, float(E[0])


def vxc_entries(basis, grid, P, functional: int, mu, nu, nthreads: int = 0):
    """(V^xc_{mu_k nu_k}, E_xc): the same computation as vxc(), accumulating
    only the requested entries of V."""
    arrs, args = _basis_args(basis)
    xyz, w, P = _f64(grid.xyz), _f64(grid.w), _f64(P)
    mu, nu = _i32(mu), _i32(nu)
    out = np.zeros(mu.shape[0])
    E = np.zeros(1)
    _check(lib().oracle_vxc_entries(*args, ctypes.c_long(w.shape[0]), _dp(xyz), _dp(w), _dp(P), int(functional),
                                    int(mu.shape[0]), _ip(mu), _ip(nu), _dp(out), _dp(E), int(nthreads)),
           "vxc_entries")
    return out, float(E[0])
