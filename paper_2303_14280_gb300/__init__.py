"""Python binding of libsnk, the GB300 sn-K exact-exchange build.

Argument marshalling only: every step of the build runs in the CUDA kernels of
``libsnk.so`` behind the C ABI of ``include/snk.h``.  There is no CPU fallback:
if the library is missing or no GPU is present the calls raise.

    eng = Engine(basis, grid)          # snk_create
    eng.set_density(P)                 # snk_set_density (NumPy) / _device (torch CUDA tensor)
    K = eng.build_K()                  # snk_build_K -> NumPy, or build_K(out=cuda_tensor)

    batch = Engine([b0, b1, ...], [g0, g1, ...])   # snk_create_batch: many molecules, shared launches
    batch.set_density([P0, P1, ...])
    Ks = batch.build_K()               # list of NumPy arrays

``basis`` needs the attributes l, nprim, atom, center, exps, coefs and
``grid`` the attributes xyz, w, atom (NumPy arrays), as produced by the
``synth`` generators.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["Engine", "SnkError", "lib", "options", "debug_boys", "debug_tc_gemm", "SYMBOLS"]

_lib = None
_lock = threading.Lock()

SNK_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "unsupported input", -3: "density matrix not symmetric",
          -4: "bad call order", -5: "out of memory", -6: "CUDA error", -7: "device wait timed out"}
SCREEN = {"none": 0, "link": 1, "learned": 2}
PRECISION = {"fp64": 0, "mixed": 1}
GEMM = {"fp64": 0, "df32": 1, "split": 2}
LISTS = ["ss", "ps", "pp", "ds", "dp", "dd"]

# every entry point declared in include/snk.h
SYMBOLS = ["snk_options_default", "snk_create", "snk_create_batch", "snk_n_molecules", "snk_molecule_functions",
           "snk_set_density", "snk_set_density_device", "snk_set_density_batch", "snk_build_K",
           "snk_build_K_device", "snk_build_K_batch", "snk_autotune", "snk_set_stream", "snk_get_stats",
           "snk_n_functions", "snk_last_error", "snk_status_string", "snk_destroy", "snk_debug_boys",
           "snk_debug_shell_A", "snk_debug_pair_bound", "snk_debug_batches", "snk_shell_A_noalloc",
           "snk_screen_load", "snk_learn_collect", "snk_mlp_train", "snk_mlp_eval", "snk_mlp_grad",
           "snk_set_density_multi", "snk_build_K_multi", "snk_set_allocator", "snk_debug_tc_gemm",
           "snk_debug_wait_timeout", "snk_build_Vxc", "snk_build_Vxc_device"]
MLP_FEATURES, MLP_WEIGHTS = 16, 9473
XC_LDA_X, XC_PBE_X, XC_PBE = 1, 2, 3   # functionals of snk_build_Vxc
MAX_DENSITIES = 2


class SnkError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"libsnk: {STATUS.get(status, status)}" + (f": {msg}" if msg else ""))


class SnkBasis(ctypes.Structure):
    _fields_ = [("n_shells", ctypes.c_int32), ("l", ctypes.POINTER(ctypes.c_int32)),
                ("nprim", ctypes.POINTER(ctypes.c_int32)), ("atom", ctypes.POINTER(ctypes.c_int32)),
                ("center", ctypes.POINTER(ctypes.c_double)), ("exps", ctypes.POINTER(ctypes.c_double)),
                ("coefs", ctypes.POINTER(ctypes.c_double))]


class SnkGrid(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("xyz", ctypes.POINTER(ctypes.c_double)),
                ("w", ctypes.POINTER(ctypes.c_double)), ("atom", ctypes.POINTER(ctypes.c_int32))]


class SnkOptions(ctypes.Structure):
    _fields_ = [("eps_basis", ctypes.c_double), ("eps_E", ctypes.c_double), ("eps_K", ctypes.c_double),
                ("batch_max", ctypes.c_int32), ("precision", ctypes.c_int32), ("screen", ctypes.c_int32),
                ("distance_bound", ctypes.c_int32), ("fp32_bound", ctypes.c_double),
                ("workspace_bytes", ctypes.c_int64), ("graph", ctypes.c_int32),
                ("learned_skip", ctypes.c_double), ("gemm", ctypes.c_int32), ("ds_integrals", ctypes.c_int32),
                ("learned_fp32", ctypes.c_double), ("tc_slices_hi", ctypes.c_int32),
                ("tc_slices_lo", ctypes.c_int32), ("eps_tile", ctypes.c_double), ("reserved", ctypes.c_double * 3)]


class SnkStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_points", "n_batches", "n_shells", "n_functions", "n_pairs",
                                               "pairs_kept", "pair_points")] + \
               [("integrals", ctypes.c_double), ("integral_flops", ctypes.c_double), ("gemm_flops", ctypes.c_double),
                ("n_chunks", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64), ("kernel_launches", ctypes.c_int64)] + \
               [(n, ctypes.c_double) for n in ("ms_screen", "ms_collocation", "ms_fgemm", "ms_integrals", "ms_kgemm",
                                                "ms_finish", "ms_build")] + \
               [("ms_integrals_class", ctypes.c_double * 6), ("integrals_class", ctypes.c_double * 6),
                ("flops_class", ctypes.c_double * 6), ("pairs_kept_fp32", ctypes.c_int64),
                ("integrals_fp32", ctypes.c_double), ("flops_fp32", ctypes.c_double),
                ("ms_integrals_fp32", ctypes.c_double), ("pairs_learned_skipped", ctypes.c_int64),
                ("gemm_flops_hi", ctypes.c_double), ("ms_integrals_class_fp32", ctypes.c_double * 6),
                ("colloc_bytes", ctypes.c_double), ("ms_gemm_split", ctypes.c_double),
                ("ms_gemm_hi", ctypes.c_double), ("ms_gemm_lo", ctypes.c_double), ("gemm_tc_flops", ctypes.c_double),
                ("pair_points_fp32", ctypes.c_double), ("pair_points_fp32_listed", ctypes.c_double)] + \
               [(n, ctypes.c_double) for n in ("ms_xc_collocation", "ms_xc_fgemm", "ms_xc_point", "ms_xc_vgemm",
                                                "xc_gemm_flops", "xc_colloc_bytes")]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_P = ctypes.c_void_p
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libsnk.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise SnkError(-6, f"{path} is missing; run paper_2303_14280_gb300.build.build()")
            L = ctypes.CDLL(path)
            L.snk_options_default.argtypes = [ctypes.POINTER(SnkOptions)]
            L.snk_options_default.restype = None
            L.snk_create.argtypes = [ctypes.POINTER(SnkBasis), ctypes.POINTER(SnkGrid), ctypes.POINTER(SnkOptions),
                                     ctypes.POINTER(_P)]
            L.snk_create_batch.argtypes = [ctypes.c_int32, ctypes.POINTER(SnkBasis), ctypes.POINTER(SnkGrid),
                                           ctypes.POINTER(SnkOptions), ctypes.POINTER(_P)]
            L.snk_n_molecules.argtypes = [_P]
            L.snk_n_molecules.restype = ctypes.c_int32
            L.snk_molecule_functions.argtypes = [_P, ctypes.c_int32]
            L.snk_molecule_functions.restype = ctypes.c_int64
            for name in ("snk_set_density", "snk_set_density_device", "snk_build_K", "snk_build_K_device",
                         "snk_set_density_batch", "snk_build_K_batch"):
                getattr(L, name).argtypes = [_P, _P]
            L.snk_autotune.argtypes = [_P, _I32]
            L.snk_build_Vxc.argtypes = [_P, ctypes.c_int32, _P, _P]
            L.snk_build_Vxc_device.argtypes = [_P, ctypes.c_int32, _P, _P]
            L.snk_set_density_multi.argtypes = [_P, ctypes.c_int32, _P]
            L.snk_build_K_multi.argtypes = [_P, _P]
            L.snk_set_stream.argtypes = [_P, _P]
            L.snk_set_allocator.argtypes = [_P, ALLOC_FN, FREE_FN, _P]
            L.snk_get_stats.argtypes = [_P, ctypes.POINTER(SnkStats)]
            L.snk_n_functions.argtypes = [_P]
            L.snk_n_functions.restype = ctypes.c_int64
            L.snk_last_error.argtypes = [_P]
            L.snk_last_error.restype = ctypes.c_char_p
            L.snk_status_string.argtypes = [ctypes.c_int]
            L.snk_status_string.restype = ctypes.c_char_p
            L.snk_destroy.argtypes = [_P]
            L.snk_destroy.restype = None
            L.snk_debug_boys.argtypes = [ctypes.c_int64, _D, ctypes.c_int, _D]
            L.snk_debug_tc_gemm.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _D, _D, ctypes.c_int32,
                                            _D]
            L.snk_debug_shell_A.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _D, _D]
            L.snk_debug_pair_bound.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _D]
            L.snk_debug_wait_timeout.argtypes = [_P, ctypes.c_int64]
            L.snk_debug_batches.argtypes = [_P, ctypes.POINTER(ctypes.c_int64), _I32, ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_int64)]
            L.snk_shell_A_noalloc.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, _P]
            _F = ctypes.POINTER(ctypes.c_float)
            L.snk_screen_load.argtypes = [_P, _F]
            L.snk_learn_collect.argtypes = [_P, ctypes.c_int32, ctypes.c_int64, _F, _F, ctypes.POINTER(ctypes.c_int64)]
            L.snk_mlp_train.argtypes = [_F, _F, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                        ctypes.c_float, ctypes.c_uint64, ctypes.c_int32, _F, _F]
            L.snk_mlp_eval.argtypes = [_F, _F, ctypes.c_int64, ctypes.c_int32, _F]
            L.snk_mlp_grad.argtypes = [_F, _F, _F, ctypes.c_int64, ctypes.c_float, _F, _F]
            _lib = L
    return _lib


def options(**kw) -> SnkOptions:
    """snk_options from the library defaults and keyword overrides: any field
    of snk_options (include/snk.h), `eps` for eps_basis = eps_E = eps_K, and
    names for screen ("none", "link", "learned"), precision ("fp64", "mixed")
    and gemm ("fp64", "df32", "split").  Unknown keys raise ValueError."""
    o = SnkOptions()
    lib().snk_options_default(ctypes.byref(o))
    fields = {f[0] for f in SnkOptions._fields_} - {"reserved"}
    for k, v in kw.items():
        if k != "eps" and k not in fields:
            raise ValueError(f"unknown option {k!r}; options are eps, {', '.join(sorted(fields))}")
        if k == "screen" and isinstance(v, str):
            v = SCREEN[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k == "gemm" and isinstance(v, str):
            v = GEMM[v]
        if k == "eps":
            o.eps_basis = o.eps_E = o.eps_K = float(v)
            continue
        setattr(o, k, v)
    return o


def _dptr(a):
    return a.ctypes.data_as(_D)


def debug_boys(T, nmax: int) -> np.ndarray:
    """Device Boys function F_0..F_nmax at the given T (test export)."""
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(-1)
    out = np.zeros((T.shape[0], nmax + 1))
    rc = lib().snk_debug_boys(T.shape[0], _dptr(T), nmax, _dptr(out))
    if rc != SNK_OK:
        raise SnkError(rc)
    return out


def debug_tc_gemm(A, B, slices=5) -> np.ndarray:
    """C = A B^T by the split-product tensor-core GEMM (test export)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[1]:
        raise ValueError("A (M, K) and B (N, K) with the same K")
    C = np.zeros((A.shape[0], B.shape[0]))
    rc = lib().snk_debug_tc_gemm(A.shape[0], B.shape[0], A.shape[1], _dptr(A), _dptr(B), int(slices), _dptr(C))
    if rc != SNK_OK:
        raise SnkError(rc, "snk_debug_tc_gemm")
    return C


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


def _current_device():
    """The CUDA device current in torch (the one snk_create binds the handle to)."""
    try:
        import torch
        return torch.cuda.current_device() if torch.cuda.is_available() else None
    except Exception:
        return None


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


def mlp_train(features, labels, epochs=20, batch=4096, lr=1e-3, under_weight=4.0, seed=0, weights=None):
    """Train the screen MLP on the GPU (snk_mlp_train); returns (weights, loss per epoch)."""
    X, Y = _f32(features, (-1, MLP_FEATURES)), _f32(labels, (-1,))
    w = np.zeros(MLP_WEIGHTS, dtype=np.float32) if weights is None else _f32(weights).copy()
    hist = np.zeros(max(epochs, 1), dtype=np.float32)
    rc = lib().snk_mlp_train(_fptr(X), _fptr(Y), X.shape[0], int(epochs), int(batch), float(lr), float(under_weight),
                             int(seed), 1 if weights is None else 0, _fptr(w), _fptr(hist))
    if rc != SNK_OK:
        raise SnkError(rc, "snk_mlp_train")
    return w, hist[:epochs]


def mlp_eval(weights, features, f16=False):
    """MLP predictions (snk_mlp_eval): FP32, or the FP16 tensor-core path."""
    w, X = _f32(weights), _f32(features, (-1, MLP_FEATURES))
    out = np.zeros(X.shape[0], dtype=np.float32)
    rc = lib().snk_mlp_eval(_fptr(w), _fptr(X), X.shape[0], 1 if f16 else 0, _fptr(out))
    if rc != SNK_OK:
        raise SnkError(rc, "snk_mlp_eval")
    return out


def mlp_grad(weights, features, labels, under_weight=4.0):
    """Loss and gradient of the screen MLP by the GPU training kernels (snk_mlp_grad)."""
    w, X, Y = _f32(weights), _f32(features, (-1, MLP_FEATURES)), _f32(labels, (-1,))
    g = np.zeros(MLP_WEIGHTS, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    rc = lib().snk_mlp_grad(_fptr(w), _fptr(X), _fptr(Y), X.shape[0], float(under_weight), _fptr(g), _fptr(loss))
    if rc != SNK_OK:
        raise SnkError(rc, "snk_mlp_grad")
    return float(loss[0]), g


SCREEN_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "screen_mlp.npz")


def trained_screen(path=SCREEN_WEIGHTS):
    """The shipped learned-screen weights and calibrated skip threshold
    (written by train_screen.py): (weights float32[MLP_WEIGHTS], threshold, meta dict)."""
    import json
    with np.load(path) as z:
        w = np.ascontiguousarray(z["weights"], dtype=np.float32)
        t = float(z["threshold"])
        meta = json.loads(str(z["meta"]))
    if w.size != MLP_WEIGHTS:
        raise ValueError(f"{path}: {w.size} weights, expected {MLP_WEIGHTS}")
    return w, t, meta


def _basis_struct(basis, keep):
    arrs = [np.ascontiguousarray(basis.l, dtype=np.int32), np.ascontiguousarray(basis.nprim, dtype=np.int32),
            np.ascontiguousarray(basis.atom, dtype=np.int32), np.ascontiguousarray(basis.center, dtype=np.float64),
            np.ascontiguousarray(basis.exps, dtype=np.float64), np.ascontiguousarray(basis.coefs, dtype=np.float64)]
    keep += arrs
    return SnkBasis(int(arrs[0].shape[0]), arrs[0].ctypes.data_as(_I32), arrs[1].ctypes.data_as(_I32),
                    arrs[2].ctypes.data_as(_I32), _dptr(arrs[3]), _dptr(arrs[4]), _dptr(arrs[5]))


def _grid_struct(grid, keep):
    arrs = [np.ascontiguousarray(grid.xyz, dtype=np.float64), np.ascontiguousarray(grid.w, dtype=np.float64),
            np.ascontiguousarray(grid.atom, dtype=np.int32)]
    keep += arrs
    return SnkGrid(int(arrs[1].shape[0]), _dptr(arrs[0]), _dptr(arrs[1]), arrs[2].ctypes.data_as(_I32))


class Engine:
    """One sn-K problem (basis + grid), or a batch of independent molecules
    (lists of bases and grids), on the current CUDA device."""

    def __init__(self, basis, grid, **opts):
        L = lib()
        self._h = None
        keep = []
        self.batched = isinstance(basis, (list, tuple))
        bases = list(basis) if self.batched else [basis]
        grids = list(grid) if self.batched else [grid]
        if len(bases) != len(grids) or not bases:
            raise ValueError("need one grid per basis")
        self.opts = options(**opts)
        h = _P()
        if self.batched:
            b = (SnkBasis * len(bases))(*[_basis_struct(x, keep) for x in bases])
            g = (SnkGrid * len(grids))(*[_grid_struct(x, keep) for x in grids])
            rc = L.snk_create_batch(len(bases), b, g, ctypes.byref(self.opts), ctypes.byref(h))
        else:
            b = _basis_struct(basis, keep)
            g = _grid_struct(grid, keep)
            rc = L.snk_create(ctypes.byref(b), ctypes.byref(g), ctypes.byref(self.opts), ctypes.byref(h))
        if rc != SNK_OK:
            raise SnkError(rc, "snk_create")
        self._h = h
        self._l = np.concatenate([np.asarray(x.l, dtype=np.int32) for x in bases])
        self.n_mol = int(L.snk_n_molecules(h))
        self.nfs = [int(L.snk_molecule_functions(h, m)) for m in range(self.n_mol)]
        self.nf = int(L.snk_n_functions(h))
        self.packed = sum(n * n for n in self.nfs)
        self.n_dens = 1
        self._stream = None
        self._alloc_cbs = None      # ctypes callbacks of set_allocator, kept alive with the handle
        self.device_index = _current_device()

    # -- plumbing ---------------------------------------------------------
    def _check(self, rc, what):
        if rc != SNK_OK:
            msg = lib().snk_last_error(self._h).decode()
            raise SnkError(rc, f"{what}: {msg}")

    def close(self):
        if getattr(self, "_h", None):
            lib().snk_destroy(self._h)   # may still call the allocator's free
            self._h = None
        self._alloc_cbs = None

    def set_allocator(self, alloc=None, free=None):
        """snk_set_allocator: alloc(nbytes) -> device address (int, 0 for
        failure) and free(address) take over every device buffer of the handle;
        both None goes back to cudaMalloc.  The loaded density is dropped (call
        set_density again).  An exception inside alloc counts as a failed
        allocation (SNK_ERR_OOM)."""
        if (alloc is None) != (free is None):
            raise ValueError("give both alloc and free, or neither")
        if alloc is None:
            self._check(lib().snk_set_allocator(self._h, ALLOC_FN(), FREE_FN(), None), "snk_set_allocator")
            self._alloc_cbs = None
            return

        def _a(nbytes, user):
            try:
                return int(alloc(int(nbytes)) or 0) or None
            except Exception:
                return None

        def _f(ptr, user):
            try:
                free(int(ptr))
            except Exception:
                pass

        cbs = (ALLOC_FN(_a), FREE_FN(_f))
        self._check(lib().snk_set_allocator(self._h, cbs[0], cbs[1], None), "snk_set_allocator")
        old, self._alloc_cbs = self._alloc_cbs, cbs
        del old

    def use_torch_allocator(self):
        """Route every device buffer of the handle through PyTorch's caching
        allocator (torch.empty on the engine's device), so that torch owns and
        accounts all of the library's memory."""
        import torch
        dev = torch.device("cuda", self.device_index)
        blocks = {}

        def alloc(nbytes):
            t = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            blocks[t.data_ptr()] = t
            return t.data_ptr()

        def free(ptr):
            blocks.pop(ptr, None)

        self.set_allocator(alloc, free)
        self._torch_blocks = blocks
        return blocks

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """Use a torch.cuda.Stream (or a raw cudaStream_t int) for all work."""
        ptr = getattr(stream, "cuda_stream", stream)
        self._stream = stream
        self._check(lib().snk_set_stream(self._h, _P(int(ptr) if ptr else None)), "snk_set_stream")

    # -- the sn-K build ---------------------------------------------------
    def set_density(self, P):
        """P: NumPy array (N_b x N_b, or the packed blocks), a list of NumPy
        arrays (one per molecule of a batch handle; for a single-molecule
        handle, up to MAX_DENSITIES densities built together), or a torch
        CUDA tensor (packed), float64, symmetric."""
        self.n_dens = 1
        if isinstance(P, (list, tuple)) and not self.batched:
            arrs = [np.ascontiguousarray(p, dtype=np.float64) for p in P]
            assert all(a.size == self.packed for a in arrs)
            ptrs = (_P * len(arrs))(*[a.ctypes.data for a in arrs])
            self._check(lib().snk_set_density_multi(self._h, len(arrs), ptrs), "snk_set_density_multi")
            self.n_dens = len(arrs)
            return
        if isinstance(P, (list, tuple)):
            arrs = [np.ascontiguousarray(p, dtype=np.float64) for p in P]
            assert [a.shape for a in arrs] == [(n, n) for n in self.nfs]
            ptrs = (_P * len(arrs))(*[a.ctypes.data for a in arrs])
            self._check(lib().snk_set_density_batch(self._h, ptrs), "snk_set_density_batch")
        elif _is_cuda_tensor(P):
            assert P.dtype.is_floating_point and P.element_size() == 8 and P.is_contiguous()
            assert P.numel() == self.packed
            self._check(lib().snk_set_density_device(self._h, _P(P.data_ptr())), "snk_set_density_device")
        else:
            Pn = np.ascontiguousarray(P, dtype=np.float64)
            assert Pn.size == self.packed
            self._check(lib().snk_set_density(self._h, _P(Pn.ctypes.data)), "snk_set_density")

    def build_K(self, out=None):
        """Host K (NumPy; a list of per-molecule arrays for a batch) by default;
        with out = a CUDA tensor (packed blocks) the build writes there and
        returns it once the work is enqueued on the engine's stream."""
        if self.n_dens > 1:
            Ks = [np.empty((self.nf, self.nf)) for _ in range(self.n_dens)]
            ptrs = (_P * len(Ks))(*[k.ctypes.data for k in Ks])
            self._check(lib().snk_build_K_multi(self._h, ptrs), "snk_build_K_multi")
            return Ks
        if out is not None and _is_cuda_tensor(out):
            assert out.element_size() == 8 and out.is_contiguous() and out.numel() == self.packed
            self._check(lib().snk_build_K_device(self._h, _P(out.data_ptr())), "snk_build_K_device")
            return out
        if self.batched and out is None:
            Ks = [np.empty((n, n)) for n in self.nfs]
            ptrs = (_P * len(Ks))(*[k.ctypes.data for k in Ks])
            self._check(lib().snk_build_K_batch(self._h, ptrs), "snk_build_K_batch")
            return Ks
        K = out if out is not None else np.empty((self.nf, self.nf))
        assert K.dtype == np.float64 and K.flags.c_contiguous and K.size == self.packed
        self._check(lib().snk_build_K(self._h, _P(K.ctypes.data)), "snk_build_K")
        return K

    def build_Vxc(self, functional, out=None):
        """(V^xc, E_xc) of the loaded density (snk_build_Vxc; Sec. II.C) for
        functional XC_LDA_X, XC_PBE_X or XC_PBE.  V is a host array (a list of
        per-molecule arrays and E_xc a list for a batch handle), or with out =
        a contiguous float64 CUDA tensor of the packed blocks on the engine's
        device, written there (E_xc is then read back, which waits for the
        engine's stream)."""
        fn = int(functional)
        E = np.zeros(max(self.n_mol, 1))
        Ep = _P(E.ctypes.data)
        if out is not None and _is_cuda_tensor(out):
            import torch
            if out.dtype != torch.float64 or not out.is_contiguous() or out.numel() != self.packed:
                raise ValueError("out must be a contiguous float64 tensor of the packed blocks (N_b^2 per molecule)")
            if out.device.index != self.device_index:
                raise ValueError(f"out must be on cuda:{self.device_index}, the engine's device")
            self._check(lib().snk_build_Vxc_device(self._h, fn, _P(out.data_ptr()), Ep), "snk_build_Vxc_device")
            return out, (list(E) if self.batched else float(E[0]))
        V = np.empty(self.packed)
        self._check(lib().snk_build_Vxc(self._h, fn, _P(V.ctypes.data), Ep), "snk_build_Vxc")
        if not self.batched:
            return V.reshape(self.nf, self.nf), float(E[0])
        out, off = [], 0
        for n in self.nfs:
            out.append(V[off:off + n * n].reshape(n, n))
            off += n * n
        return out, list(E)

    def screen_load(self, weights):
        """Load trained MLP weights for options screen='learned' (snk_screen_load)."""
        w = _f32(weights)
        assert w.size == MLP_WEIGHTS
        self._check(lib().snk_screen_load(self._h, _fptr(w)), "snk_screen_load")

    def learn_collect(self, stride=1, cap=1 << 22):
        """Training blocks of the loaded density (snk_learn_collect): (features, labels)."""
        feat = np.zeros((cap, MLP_FEATURES), dtype=np.float32)
        lab = np.zeros(cap, dtype=np.float32)
        n = ctypes.c_int64()
        self._check(lib().snk_learn_collect(self._h, int(stride), int(cap), _fptr(feat), _fptr(lab), ctypes.byref(n)),
                    "snk_learn_collect")
        return feat[:n.value].copy(), lab[:n.value].copy()

    def debug_wait_timeout(self, limit_ns: int) -> int:
        """snk_debug_wait_timeout: the status a build reports when a bounded
        device wait runs out (SNK_ERR_TIMEOUT), from a wait nothing completes."""
        return int(lib().snk_debug_wait_timeout(self._h, int(limit_ns)))

    def autotune(self) -> dict:
        """snk_autotune: FP32-list pairs per staging step chosen for each list."""
        runs = (ctypes.c_int32 * 12)()
        self._check(lib().snk_autotune(self._h, runs), "snk_autotune")
        names = [f"fp64_{n}" for n in LISTS] + [f"fp32_{n}" for n in LISTS]
        return dict(zip(names, list(runs)))

    def stats(self) -> dict:
        s = SnkStats()
        self._check(lib().snk_get_stats(self._h, ctypes.byref(s)), "snk_get_stats")
        out = {}
        for name, _ in SnkStats._fields_:
            v = getattr(s, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out

    # -- test exports -----------------------------------------------------
    def debug_shell_A(self, sa, sb, xyz):
        """Device 3c-CP block A_{mu lam}(r) of shells sa, sb at the points: (n, n_a, n_b)."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        na = (int(self._l[sa]) + 1) * (int(self._l[sa]) + 2) // 2
        nb = (int(self._l[sb]) + 1) * (int(self._l[sb]) + 2) // 2
        out = np.zeros((xyz.shape[0], na, nb))
        self._check(lib().snk_debug_shell_A(self._h, int(sa), int(sb), xyz.shape[0], _dptr(xyz), _dptr(out)),
                    "snk_debug_shell_A")
        return out

    def shell_A_noalloc(self, sa, sb, xyz, out):
        """snk_shell_A_noalloc: the same block as debug_shell_A for callers that
        cannot allocate device memory.  xyz (n, 3) and out (n, n_a, n_b) are
        contiguous float64 CUDA tensors owned by the caller; n <= 4096.  The
        work is enqueued on the engine's stream; the call does not wait."""
        import torch
        if not (_is_cuda_tensor(xyz) and _is_cuda_tensor(out)):
            raise ValueError("xyz and out must be CUDA tensors")
        if xyz.dtype != torch.float64 or out.dtype != torch.float64:
            raise ValueError("xyz and out must be float64")
        if not (xyz.is_contiguous() and out.is_contiguous()):
            raise ValueError("xyz and out must be contiguous")
        if xyz.device.index != self.device_index or out.device.index != self.device_index:
            raise ValueError(f"xyz and out must be on cuda:{self.device_index}, the engine's device")
        if not (0 <= int(sa) < self._l.shape[0] and 0 <= int(sb) < self._l.shape[0]):
            raise ValueError(f"shell index out of range 0..{self._l.shape[0] - 1}")
        na = (int(self._l[sa]) + 1) * (int(self._l[sa]) + 2) // 2
        nb = (int(self._l[sb]) + 1) * (int(self._l[sb]) + 2) // 2
        if xyz.dim() != 2 or xyz.shape[1] != 3:
            raise ValueError(f"xyz must be (n, 3), got {tuple(xyz.shape)}")
        n = xyz.shape[0]
        if tuple(out.shape) != (n, na, nb):
            raise ValueError(f"out must be {(n, na, nb)}, got {tuple(out.shape)}")
        self._check(lib().snk_shell_A_noalloc(self._h, int(sa), int(sb), int(n), _P(xyz.data_ptr()),
                                              _P(out.data_ptr())), "snk_shell_A_noalloc")
        return out

    def debug_pair_bound(self, sa, sb) -> float:
        v = ctypes.c_double()
        self._check(lib().snk_debug_pair_bound(self._h, int(sa), int(sb), ctypes.byref(v)), "snk_debug_pair_bound")
        return v.value

    def debug_batches(self):
        n = ctypes.c_int64()
        self._check(lib().snk_debug_batches(self._h, ctypes.byref(n), None, 0, None), "snk_debug_batches")
        counts = np.zeros(max(n.value, 1), dtype=np.int32)
        perm = np.zeros(int(self.stats()["n_points"]), dtype=np.int64)
        self._check(lib().snk_debug_batches(self._h, ctypes.byref(n), counts.ctypes.data_as(_I32), counts.shape[0],
                                            perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
                    "snk_debug_batches")
        return counts[:n.value], perm
