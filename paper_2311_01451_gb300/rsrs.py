"""Thin ctypes binding of librsrs (include/rsrs.h): argument marshalling only.

Every step of the method runs in the CUDA library.  Device blocks are torch
float64 CUDA tensors (column-major N x nrhs, i.e. a tensor of shape
(nrhs, N) or a Fortran-ordered view); PyTorch supplies device memory and the
current CUDA stream.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librsrs.so")

RSRS_OP_LOG2D, RSRS_OP_INVR3D, RSRS_OP_CALLBACK = 1, 2, 3
RSRS_PREC_FP64, RSRS_PREC_MIXED = 0, 1

STATUS = {0: "RSRS_OK", 1: "RSRS_E_INVAL", 2: "RSRS_E_UNDERSAMPLED", 3: "RSRS_E_SINGULAR",
          4: "RSRS_E_NONFINITE", 5: "RSRS_E_NOMEM", 6: "RSRS_E_CUDA", 7: "RSRS_E_CALLBACK",
          8: "RSRS_E_TIMEOUT", 9: "RSRS_E_NOT_CONVERGED"}

EXPORTS = ["rsrs_tree_build", "rsrs_tree_info", "rsrs_tree_perm", "rsrs_tree_schedule", "rsrs_tree_free",
           "rsrs_build", "rsrs_build_batched", "rsrs_refactor", "rsrs_solve", "rsrs_solve_noalloc", "rsrs_wait_selftest", "rsrs_grid_wait_selftest", "rsrs_convert_selftest", "rsrs_apply", "rsrs_refine", "rsrs_residual", "rsrs_matvec", "rsrs_factor_stats",
           "rsrs_factor_box", "rsrs_factor_root", "rsrs_factor_sketches", "rsrs_factor_free",
           "rsrs_status_string", "rsrs_last_error", "rsrs_kernel_class_name", "rsrs_stencil7_create", "rsrs_stencil7_matvec", "rsrs_stencil7_free", "rsrs_autotune", "rsrs_gmres"]

MATVEC_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_int64, C.c_int32, C.c_void_p, C.c_int64,
                        C.c_void_p, C.c_int64, C.c_void_p)


class Operator(C.Structure):
    _fields_ = [("kind", C.c_int), ("diag_shift", C.c_double), ("scale", C.c_double),
                ("fn", MATVEC_FN), ("ctx", C.c_void_p)]


RSRS_SAMPLE_TILE_DEFAULT, RSRS_SAMPLE_TILE_256x2, RSRS_SAMPLE_TILE_128x3, RSRS_SAMPLE_TILE_192x2 = 0, 1, 2, 3
RSRS_SAMPLE_TILE_256x4_K16, RSRS_SAMPLE_TILE_192x5_K16 = 4, 5
RSRS_SAMPLE_TILE_2x256x3_K16, RSRS_SAMPLE_TILE_2x192x4_K16 = 6, 7
RSRS_RESIDUAL_AUTO, RSRS_RESIDUAL_FP64, RSRS_RESIDUAL_FLOAT_FLOAT, RSRS_RESIDUAL_OZAKI = 0, 1, 2, 3


class Tune(C.Structure):
    """rsrs_tune_t: launch shapes (all zero = library defaults)."""
    _fields_ = [("sample_tile", C.c_int32), ("cpqr_cluster", C.c_int32), ("cpqr_threads", C.c_int32),
                ("residual_split", C.c_int32), ("reserved", C.c_int32 * 4)]

    def as_dict(self) -> dict:
        return {nm: int(getattr(self, nm)) for nm in ("sample_tile", "cpqr_cluster", "cpqr_threads",
                                                       "residual_split")}


class TuneReport(C.Structure):
    _fields_ = [("candidates", C.c_int), ("from_cache", C.c_int), ("default_ms", C.c_double),
                ("tuned_ms", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("p", C.c_int), ("proj_passes", C.c_int), ("seed", C.c_uint64),
                ("omega_host", C.c_void_p), ("psi_host", C.c_void_p), ("omega_dev", C.c_void_p),
                ("psi_dev", C.c_void_p), ("keep_sketches", C.c_int), ("profile", C.c_int),
                ("sample_kernel", C.c_int), ("mixed_cpqr", C.c_int), ("mixed_gemm", C.c_int),
                ("use_graph", C.c_int), ("residual_fp64", C.c_int), ("tune", Tune)]


def _tune(t) -> Tune:
    """A Tune from None, a Tune or a dict of its fields."""
    if t is None:
        return Tune()
    if isinstance(t, Tune):
        return t
    return Tune(**{k: int(v) for k, v in dict(t).items()})


NCLASS = 16


class TreeInfo(C.Structure):
    _fields_ = [("d", C.c_int), ("depth", C.c_int), ("n", C.c_int64), ("n_boxes", C.c_int64),
                ("n_leaves", C.c_int64), ("n_compress", C.c_int64), ("n_groups", C.c_int64),
                ("max_l", C.c_int64), ("root_size", C.c_int64), ("s_req", C.c_int64),
                ("s_req_mixed", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("s", C.c_int64), ("k", C.c_int64), ("n_boxes", C.c_int64),
                ("root_size", C.c_int64), ("factor_bytes", C.c_int64), ("work_bytes", C.c_int64),
                ("t_sample_ms", C.c_double), ("t_compress_ms", C.c_double), ("t_root_ms", C.c_double),
                ("kernel_launches", C.c_int64), ("class_ms", C.c_double * NCLASS),
                ("class_gflop", C.c_double * NCLASS), ("class_launches", C.c_int64 * NCLASS),
                ("solve_bytes", C.c_int64)]


class RefineReport(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double), ("history", C.c_double * 64),
                ("kernel_launches", C.c_int64), ("residual_kind", C.c_int32)]


class BoxView(C.Structure):
    _fields_ = [("level", C.c_int32), ("colour", C.c_int32), ("b", C.c_int64), ("n", C.c_int64),
                ("kp", C.c_int64), ("r", C.c_int64)] + [
        (nm, C.c_void_p) for nm in ("S", "R", "N", "T", "XRR", "LcS", "LcN", "UcS", "UcN")]


_lib = None


def lib():
    """Load librsrs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librsrs.so not built at {LIB_PATH}: run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        sig = {
            "rsrs_tree_build": [vp, i64, C.c_int, C.c_int, C.POINTER(vp)],
            "rsrs_tree_info": [vp, C.c_int, C.c_int, C.POINTER(TreeInfo)],
            "rsrs_tree_perm": [vp, vp],
            "rsrs_tree_schedule": [vp, C.c_int, C.c_int, vp],
            "rsrs_build": [vp, C.POINTER(Operator), C.c_int, C.c_int, C.POINTER(Options), vp, C.POINTER(vp)],
            "rsrs_build_batched": [C.c_int, C.POINTER(vp), C.POINTER(Operator), C.c_int, C.c_int, C.POINTER(Options),
                                   vp, C.POINTER(vp)],
            "rsrs_solve": [vp, vp, i64, i32, C.c_int, vp],
            "rsrs_refactor": [vp, C.c_uint64, vp],
            "rsrs_solve_noalloc": [vp, vp, i64, i32, C.c_int, vp],
            "rsrs_apply": [vp, vp, i64, i32, C.c_int, vp],
            "rsrs_refine": [vp, vp, vp, i64, i32, dbl, C.c_int, vp, C.POINTER(RefineReport)],
            "rsrs_gmres": [vp, vp, vp, i64, i32, dbl, C.c_int, C.c_int, vp, C.POINTER(RefineReport)],
            "rsrs_residual": [vp, vp, vp, vp, i64, i32, vp],
            "rsrs_matvec": [vp, vp, vp, i64, i32, vp],
            "rsrs_factor_stats": [vp, C.POINTER(Stats)],
            "rsrs_factor_box": [vp, i64, C.POINTER(BoxView)],
            "rsrs_factor_root": [vp, vp, vp, C.POINTER(i64)],
            "rsrs_factor_sketches": [vp, vp, vp, vp, vp],
            "rsrs_stencil7_create": [vp, C.c_int, C.POINTER(vp)],
            "rsrs_stencil7_matvec": [vp, C.c_int, i64, i32, vp, i64, vp, i64, vp],
            "rsrs_autotune": [C.c_int, C.POINTER(vp), C.POINTER(Operator), C.c_int, C.c_int, C.POINTER(Options),
                              C.c_int, C.c_char_p, vp, C.POINTER(Tune), C.POINTER(TuneReport)],
            "rsrs_wait_selftest": [i64, C.c_int, vp],
            "rsrs_grid_wait_selftest": [i64, C.c_int, vp],
            "rsrs_convert_selftest": [vp, i64, vp, vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.rsrs_tree_free.argtypes = [vp]
        L.rsrs_tree_free.restype = None
        L.rsrs_factor_free.argtypes = [vp]
        L.rsrs_factor_free.restype = None
        L.rsrs_stencil7_free.argtypes = [vp]
        L.rsrs_stencil7_free.restype = None
        L.rsrs_status_string.argtypes = [C.c_int]
        L.rsrs_status_string.restype = C.c_char_p
        L.rsrs_kernel_class_name.argtypes = [C.c_int]
        L.rsrs_kernel_class_name.restype = C.c_char_p
        L.rsrs_last_error.argtypes = []
        L.rsrs_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def wait_selftest(polls: int, arrive: bool, stream=None):
    """rsrs_wait_selftest: one CTA waits, through the kernels' bounded mbarrier wait (at most
    ``polls`` polls), for an arrival made only when ``arrive`` is true.  Raises RSRSError
    (RSRS_E_TIMEOUT) when the wait expired; returns None when it completed."""
    _check(lib().rsrs_wait_selftest(int(polls), int(bool(arrive)), _stream_ptr(stream)))


def grid_wait_selftest(polls: int, arrive: bool, stream=None):
    """rsrs_grid_wait_selftest: two CTAs meet at the fused sweeps' grid barrier (at most ``polls``
    polls), the second only when ``arrive`` is true.  Raises RSRSError (RSRS_E_TIMEOUT) when the
    wait expired; returns None when both arrived."""
    _check(lib().rsrs_grid_wait_selftest(int(polls), int(bool(arrive)), _stream_ptr(stream)))


def convert_selftest(x, stream=None):
    """rsrs_convert_selftest on a contiguous FP64 CUDA tensor: returns (f, g), the library's
    integer-pipe rounding of x to FP32 and its exact widening back to FP64."""
    import torch

    if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise ValueError("x must be a contiguous float64 CUDA tensor")
    f = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    g = torch.empty(x.shape, dtype=torch.float64, device=x.device)
    _check(lib().rsrs_convert_selftest(C.c_void_p(x.data_ptr()), x.numel(), C.c_void_p(f.data_ptr()),
                                       C.c_void_p(g.data_ptr()), _stream_ptr(stream)))
    return f, g


class RSRSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


def _check(st: int):
    if st != 0:
        raise RSRSError(st, lib().rsrs_last_error().decode())


def _stream_ptr(stream=None):
    """The given (or current) torch CUDA stream; NULL (legacy default stream) without a GPU, so that
    argument validation, which happens before any device work, can still run."""
    import torch
    if stream is None:
        if not torch.cuda.is_available():
            return C.c_void_p(0)
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _cm(t):
    """(ptr, ld, ncols) of a column-major N x nrhs float64 CUDA block given as a (nrhs, N) tensor."""
    import torch
    if t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError("expected a float64 CUDA tensor")
    if t.dim() == 1:
        t = t.unsqueeze(0)
    if not t.is_contiguous():
        raise ValueError("expected a contiguous (nrhs, N) tensor (column-major N x nrhs)")
    return C.c_void_p(t.data_ptr()), t.shape[1], t.shape[0]


class Tree:
    """rsrs_tree_build: quad/octree over host points (N x d float64)."""

    def __init__(self, points: np.ndarray, leaf_cap: int):
        pts = np.ascontiguousarray(points, dtype=np.float64)
        self.n, self.d = pts.shape
        h = C.c_void_p()
        _check(lib().rsrs_tree_build(pts.ctypes.data_as(C.c_void_p), self.n, self.d, leaf_cap, C.byref(h)))
        self._h = h

    def info(self, k: int, p: int = -1) -> TreeInfo:
        out = TreeInfo()
        _check(lib().rsrs_tree_info(self._h, k, p, C.byref(out)))
        return out

    def perm(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int64)
        _check(lib().rsrs_tree_perm(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    def schedule(self, k: int, p: int = -1) -> np.ndarray:
        n = self.info(k, p).n_compress
        out = np.empty((max(n, 1), 6), dtype=np.int64)
        _check(lib().rsrs_tree_schedule(self._h, k, p, out.ctypes.data_as(C.c_void_p)))
        return out[:n]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rsrs_tree_free(self._h)
            self._h = None


class Stencil7:
    """rsrs_stencil7: the 7-point variable-coefficient operator on an m^3 cell grid as a device
    matvec callback (pass it as ``matvec`` with ``kind=RSRS_OP_CALLBACK``)."""

    def __init__(self, coef: np.ndarray, m: int):
        b = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
        if b.size != m ** 3:
            raise ValueError("need m^3 coefficients")
        h = C.c_void_p()
        _check(lib().rsrs_stencil7_create(b.ctypes.data_as(C.c_void_p), m, C.byref(h)))
        self._h = h
        self.m = m
        self.n = m ** 3
        self.fn = C.cast(lib().rsrs_stencil7_matvec, MATVEC_FN)

    def matvec(self, X, Y, stream=None):
        """Y <- A X for (ncols, N) float64 CUDA tensors (column-major N x ncols)."""
        px, ld, nc = _cm(X)
        py, ldy, ncy = _cm(Y)
        rc = lib().rsrs_stencil7_matvec(self._h, 0, self.n, nc, px, ld, py, ldy, _stream_ptr(stream))
        if rc != 0:
            raise RSRSError(7, f"stencil matvec returned {rc}")
        return Y

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rsrs_stencil7_free(self._h)
            self._h = None


class Factor:
    """rsrs_build result: the invertible factorization of eq. (Afact)."""

    def __init__(self, tree: Tree, kind: int, k: int, s: int, shift: float = 1.0, scale: float = 0.0,
                 precision: int = RSRS_PREC_FP64, p: int = -1, omega: np.ndarray | None = None,
                 psi: np.ndarray | None = None, seed: int = 0, passes: int = 0, keep_sketches: bool = False,
                 matvec=None, stream=None, profile: bool = False,
                 sample_kernel: int = 0, mixed_cpqr: int = 0, residual_fp64: bool = False, residual=None,
                 mixed_gemm: int = 0, use_graph: bool = False, tune=None):
        self.tree = tree
        self.n = tree.n
        self._cb = None
        op = Operator(kind=kind, diag_shift=shift, scale=scale)
        if kind == RSRS_OP_CALLBACK:
            if matvec is None:
                raise ValueError("callback operator needs matvec")
            if isinstance(matvec, Stencil7):  # a library-side device matvec: no Python in the loop
                self._cb = matvec
                op.fn = matvec.fn
                op.ctx = matvec._h
            else:
                self._cb = MATVEC_FN(matvec)
                op.fn = self._cb
        opts = Options(precision=precision, p=p, proj_passes=passes, seed=seed,
                       keep_sketches=int(keep_sketches), profile=int(profile),
                       sample_kernel=sample_kernel,
                       mixed_cpqr=mixed_cpqr,
                       residual_fp64=int(residual_fp64) if residual is None else int(residual), mixed_gemm=mixed_gemm,
                       use_graph=int(use_graph), tune=_tune(tune))
        self._om = self._ps = None
        if omega is not None and hasattr(omega, "data_ptr"):  # device tensors (N, s), original order
            self._om, self._ps = omega, psi
            opts.omega_dev = C.c_void_p(omega.data_ptr())
            opts.psi_dev = C.c_void_p(psi.data_ptr())
        elif omega is not None:
            self._om = np.ascontiguousarray(omega, dtype=np.float64)
            self._ps = np.ascontiguousarray(psi, dtype=np.float64)
            assert self._om.shape == (self.n, s) and self._ps.shape == (self.n, s)
            opts.omega_host = self._om.ctypes.data_as(C.c_void_p)
            opts.psi_host = self._ps.ctypes.data_as(C.c_void_p)
        h = C.c_void_p()
        _check(lib().rsrs_build(tree._h, C.byref(op), k, s, C.byref(opts), _stream_ptr(stream), C.byref(h)))
        self._h = h
        self.s = s
        self.k = k

    def refactor(self, seed: int, stream=None):
        """rsrs_refactor: rebuild in place from new test matrices (key ``seed``) by replaying the
        build's captured graph (the factor must have been built with ``use_graph=True``)."""
        _check(lib().rsrs_refactor(self._h, seed, _stream_ptr(stream)))
        return self

    def solve(self, F, adjoint: bool = False, stream=None):
        """In place: F <- A_approx^-1 F, F a (nrhs, N) float64 CUDA tensor."""
        ptr, ld, nr = _cm(F)
        _check(lib().rsrs_solve(self._h, ptr, ld, nr, int(adjoint), _stream_ptr(stream)))
        return F

    def solve_noalloc(self, F, adjoint: bool = False, stream=None):
        """rsrs_solve_noalloc: as solve, staged in the library's static device buffer (no device
        allocation, no synchronisation; calls on one device must not overlap)."""
        ptr, ld, nr = _cm(F)
        _check(lib().rsrs_solve_noalloc(self._h, ptr, ld, nr, int(adjoint), _stream_ptr(stream)))
        return F

    def apply(self, F, adjoint: bool = False, stream=None):
        ptr, ld, nr = _cm(F)
        _check(lib().rsrs_apply(self._h, ptr, ld, nr, int(adjoint), _stream_ptr(stream)))
        return F

    def matvec(self, X, Y, stream=None):
        px, ld, nr = _cm(X)
        py, _, _ = _cm(Y)
        _check(lib().rsrs_matvec(self._h, px, py, ld, nr, _stream_ptr(stream)))
        return Y

    def residual(self, B, X, Rout, stream=None):
        """Rout <- B - A X in the refinement's residual arithmetic; (nrhs, N) float64 CUDA tensors."""
        pb, ld, nr = _cm(B)
        px, ldx, nrx = _cm(X)
        pr_, ldr, nrr = _cm(Rout)
        if (ldx, nrx) != (ld, nr) or (ldr, nrr) != (ld, nr):
            raise ValueError("B, X and Rout must have the same shape")
        _check(lib().rsrs_residual(self._h, pb, px, pr_, ld, nr, _stream_ptr(stream)))
        return Rout

    def gmres(self, B, X, rtol: float = 1e-12, restart: int = 30, maxit: int = 60, stream=None) -> RefineReport:
        """rsrs_gmres: X = A^-1 B by GMRES with this factor as right preconditioner."""
        pb, ld, nr = _cm(B)
        px, ldx, nrx = _cm(X)
        if (ldx, nrx) != (ld, nr):
            raise ValueError("B and X must have the same shape")
        rep = RefineReport()
        _check(lib().rsrs_gmres(self._h, pb, px, ld, nr, rtol, restart, maxit, _stream_ptr(stream), C.byref(rep)))
        return rep

    def refine(self, B, X, rtol: float = 1e-12, maxit: int = 20, stream=None) -> RefineReport:
        pb, ld, nr = _cm(B)
        px, _, _ = _cm(X)
        rep = RefineReport()
        _check(lib().rsrs_refine(self._h, pb, px, ld, nr, rtol, maxit, _stream_ptr(stream), C.byref(rep)))
        return rep

    def stats(self) -> Stats:
        out = Stats()
        _check(lib().rsrs_factor_stats(self._h, C.byref(out)))
        return out

    def class_stats(self) -> dict:
        """{class name: (ms, gflop, launches)} of the build (ms is 0 unless built with profile=True)."""
        st = self.stats()
        return {lib().rsrs_kernel_class_name(c).decode(): (st.class_ms[c], st.class_gflop[c], st.class_launches[c])
                for c in range(NCLASS)}

    def box(self, i: int) -> dict:
        v = BoxView()
        _check(lib().rsrs_factor_box(self._h, i, C.byref(v)))
        b, n, kp, r = v.b, v.n, v.kp, v.r
        arr = dict(S=np.empty(kp, np.int64), R=np.empty(r, np.int64), N=np.empty(n, np.int64),
                   T=np.empty((kp, r)), XRR=np.empty((r, r)), LcS=np.empty((kp, r)), LcN=np.empty((n, r)),
                   UcS=np.empty((r, kp)), UcN=np.empty((r, n)))
        for nm, a in arr.items():
            setattr(v, nm, a.ctypes.data_as(C.c_void_p))
        _check(lib().rsrs_factor_box(self._h, i, C.byref(v)))
        arr.update(level=v.level, colour=v.colour, b=b, n=n, kp=kp, r=r)
        return arr

    def root(self):
        size = C.c_int64()
        _check(lib().rsrs_factor_root(self._h, None, None, C.byref(size)))
        idx = np.empty(size.value, np.int64)
        a = np.empty((size.value, size.value))
        _check(lib().rsrs_factor_root(self._h, idx.ctypes.data_as(C.c_void_p), a.ctypes.data_as(C.c_void_p),
                                      C.byref(size)))
        return idx, a

    def sketches(self):
        out = [np.empty((self.n, self.s)) for _ in range(4)]
        _check(lib().rsrs_factor_sketches(self._h, *[o.ctypes.data_as(C.c_void_p) for o in out]))
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rsrs_factor_free(self._h)
            self._h = None


def build_batched(trees, kinds, k: int, s: int, shifts, scales, precision: int = RSRS_PREC_FP64, p: int = -1,
                  seed: int = 0, passes: int = 0, profile: bool = False, sample_kernel: int = 0,
                  keep_sketches: bool = False, mixed_cpqr: int = 0, residual_fp64: bool = False, residual=None,
                  mixed_gemm: int = 0, use_graph: bool = False, tune=None,
                  stream=None) -> list:
    """rsrs_build_batched: factors of independent problems built in one set of launches."""
    n = len(trees)
    ops = _operators(kinds, shifts, scales)
    handles = (C.c_void_p * n)(*[t._h for t in trees])
    outs = (C.c_void_p * n)()
    opts = Options(precision=precision, p=p, proj_passes=passes, seed=seed, profile=int(profile),
                   sample_kernel=sample_kernel,
                   keep_sketches=int(keep_sketches), mixed_cpqr=mixed_cpqr,
                   residual_fp64=int(residual_fp64) if residual is None else int(residual), mixed_gemm=mixed_gemm,
                   use_graph=int(use_graph),
                   tune=_tune(tune))
    _check(lib().rsrs_build_batched(n, handles, ops, k, s, C.byref(opts), _stream_ptr(stream), outs))
    res = []
    for i in range(n):
        f = Factor.__new__(Factor)
        f.tree, f.n, f._cb, f._om, f._ps = trees[i], trees[i].n, None, None, None
        f._h, f.s, f.k = C.c_void_p(outs[i]), s, k
        res.append(f)
    return res


def _operators(kinds, shifts, scales):
    n = len(kinds)
    ops = (Operator * n)()
    for i in range(n):
        ops[i].kind = kinds[i]
        ops[i].diag_shift = shifts[i]
        ops[i].scale = scales[i]
    return ops


def autotune(trees, kinds, k: int, s: int, shifts, scales, precision: int = RSRS_PREC_MIXED, p: int = -1,
             seed: int = 0, reps: int = 2, cache: str | None = None, stream=None, **options):
    """rsrs_autotune on built-in-kernel problems (one tree, or a list for a batched build): returns
    (tune dict, report dict).  options: the build options of Factor / build_batched."""
    if not isinstance(trees, (list, tuple)):
        trees, kinds, shifts, scales = [trees], [kinds], [shifts], [scales]
    n = len(trees)
    ops = _operators(kinds, shifts, scales)
    handles = (C.c_void_p * n)(*[t._h for t in trees])
    opts = Options(precision=precision, p=p, seed=seed,
                   proj_passes=options.pop("passes", 0), tune=_tune(options.pop("tune", None)))
    for key, val in options.items():
        setattr(opts, key, int(val))
    out, rep = Tune(), TuneReport()
    _check(lib().rsrs_autotune(n, handles, ops, k, s, C.byref(opts), reps,
                               cache.encode() if cache else None, _stream_ptr(stream), C.byref(out), C.byref(rep)))
    return out.as_dict(), {"candidates": rep.candidates, "from_cache": bool(rep.from_cache),
                           "default_ms": rep.default_ms, "tuned_ms": rep.tuned_ms}


def kind_of(kernel: str) -> int:
    return {"log2d": RSRS_OP_LOG2D, "invr3d": RSRS_OP_INVR3D}.get(kernel, RSRS_OP_CALLBACK)
