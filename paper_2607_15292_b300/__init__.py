"""Python binding of libgcqbem, the B300 (sm_103a) library for the
multi-frequency Laplace-domain operator of a 3D-ACA accelerated
convolution-quadrature BEM for 3-D elastodynamics (arXiv 2607.15292).

Argument marshalling only: every step of the computation runs in the CUDA
library behind the C ABI of ``include/gcqbem.h``.  Device buffers are
PyTorch tensors (their ``data_ptr()`` is passed); streams are PyTorch CUDA
streams.  Importing fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgcqbem.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libgcqbem.so not found at {LIB_PATH}: build it with "
        "`python paper_2607_15292_b300/build.py` (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)

BEM_OK, BEM_ERR_ARG, BEM_ERR_CUDA, BEM_ERR_OOM, BEM_ERR_MESH, BEM_ERR_NOT_CONVERGED, BEM_ERR_STATE = range(7)
BEM_FP64, BEM_MIXED = 0, 1
BEM_ROWS_CENTROIDS, BEM_ROWS_NODES = 0, 1
BEM_SL, BEM_DL = 0, 1
# wave-speed derivatives of the single layer, dV/dc_p and dV/dc_s (fixed density)
BEM_SL_DCP, BEM_SL_DCS = 2, 3
# and of the double layer C + K, d(C + K)/dc_p and d(C + K)/dc_s
BEM_DL_DCP, BEM_DL_DCS = 4, 5
BEM_APPLY_BATCHED, BEM_APPLY_CONTRACTED = 0, 1
# fault injection for tests (bem_debug_set)
BEM_DEBUG_FACE_WAIT_FAIL, BEM_DEBUG_ALLOC_CAP, BEM_DEBUG_FACE_ACA_FULL = 1, 2, 3

_STATUS = {0: "BEM_OK", 1: "BEM_ERR_ARG", 2: "BEM_ERR_CUDA", 3: "BEM_ERR_OOM", 4: "BEM_ERR_MESH",
           5: "BEM_ERR_NOT_CONVERGED", 6: "BEM_ERR_STATE"}


class bem_options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("eps_aca", ctypes.c_double), ("leaf", ctypes.c_int32),
                ("eta", ctypes.c_double), ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
                ("compress_faces", ctypes.c_int32)]


class bem_op_stats(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int64), ("n_far", ctypes.c_int64), ("n_aca", ctypes.c_int64),
                ("n_dense", ctypes.c_int64), ("n_rank0", ctypes.c_int64), ("rank_min", ctypes.c_int64),
                ("rank_max", ctypes.c_int64), ("rank_mean", ctypes.c_double),
                ("stored_bytes", ctypes.c_double), ("dense_bytes", ctypes.c_double),
                ("compression_rate", ctypes.c_double), ("entries_evaluated", ctypes.c_int64),
                ("t_entries_ms", ctypes.c_double), ("t_compress_ms", ctypes.c_double),
                ("apply_bytes", ctypes.c_int64), ("t_face_ms", ctypes.c_double),
                ("face_launches", ctypes.c_int64), ("face_alg_bytes", ctypes.c_double),
                ("launches", ctypes.c_int64), ("n_faces", ctypes.c_int64), ("n_faces_lowrank", ctypes.c_int64),
                ("face_rank_mean", ctypes.c_double), ("t_face_aca_ms", ctypes.c_double),
                ("apply_bk", ctypes.c_int64), ("apply_tune_ms", ctypes.c_double * 3),
                ("apply_kernel", ctypes.c_int64), ("apply_errors", ctypes.c_int64),
                ("apply_tensor_flops", ctypes.c_double)]


_vp, _i32, _i64, _dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_P = ctypes.POINTER
_SIGS = {
    "bem_options_default": (_i32, [_P(bem_options)]),
    "bem_ctx_create": (_i32, [_P(bem_options), _P(_vp)]),
    "bem_ctx_destroy": (None, [_vp]),
    "bem_last_error": (ctypes.c_char_p, [_vp]),
    "bem_ctx_options": (_i32, [_vp, _P(bem_options)]),
    "bem_material_set": (_i32, [_vp, _dbl, _dbl, _dbl, _P(_dbl), _P(_dbl)]),
    "bem_freqs_bdf2": (_i32, [_i32, _dbl, _i32, _P(_dbl)]),
    "bem_freqs_set": (_i32, [_vp, _P(_dbl), _i32]),
    "bem_mesh_create": (_i32, [_vp, _P(_dbl), _i64, _P(_i32), _i64, _P(_vp)]),
    "bem_mesh_destroy": (None, [_vp]),
    "bem_entries": (_i32, [_vp, _i32, _i32, _vp, _i64, _vp, _vp]),
    "bem_entries_noalloc": (_i32, [_vp, _i32, _i32, _vp, _i64, _vp, _vp]),
    "bem_tree_build": (_i32, [_vp, _i32, _i32, _P(_vp)]),
    "bem_tree_destroy": (None, [_vp]),
    "bem_tree_sizes": (_i32, [_vp, _P(_i64), _P(_i64), _P(_i64), _P(_i64)]),
    "bem_tree_export": (_i32, [_vp, _P(_i32), _P(_i32), _P(_i64)]),
    "bem_op_compress": (_i32, [_vp, _vp, _P(_vp)]),
    "bem_op_destroy": (None, [_vp]),
    "bem_op_apply": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
    "bem_op_dense": (_i32, [_vp, _vp, _vp]),
    "bem_op_stats_get": (_i32, [_vp, _P(bem_op_stats)]),
    "bem_op_blocks": (_i32, [_vp, _P(_i64)]),
    "bem_op_face_ranks": (_i32, [_vp, _P(_i32)]),
    "bem_op_solve": (_i32, [_vp, _vp, _vp, _dbl, _i32, _P(_i32), _P(_dbl), _vp]),
    "bem_op_inner": (_i32, [_vp, _i32, _vp, _vp, _P(_dbl), _vp]),
    "bem_op_solve_adjoint": (_i32, [_vp, _vp, _vp, _dbl, _i32, _P(_i32), _P(_dbl), _vp]),
    "bem_op_set_precond": (_i32, [_vp, _i32, _vp]),
    "bem_receiver_energy_grad": (_i32, [_vp, _vp, _P(_vp), _P(_vp), _i32, _i32, _dbl, _vp, _P(_i32), _i64, _dbl,
                                        _i32, _P(_dbl), _vp, _P(_dbl), _P(_i32), _vp]),
    "bem_op_compress_batch": (_i32, [_P(_vp), _i32, _i32, _P(_vp)]),
    "bem_op_set_apply_tile": (_i32, [_vp, _i32]),
    "bem_op_set_apply_kernel": (_i32, [_vp, _i32]),
    "bem_tc_selftest": (_i32, [_i32, _i32, _P(ctypes.c_float), _P(ctypes.c_float), _P(ctypes.c_float)]),
    "bem_measure_peaks": (_i32, [_i32, _P(_dbl)]),
    "bem_op_slot_stats": (_i32, [_vp, _i32, _P(_dbl), _P(_i64), _P(_i32)]),
    "bem_op_save": (_i32, [_vp, ctypes.c_char_p]),
    "bem_op_load": (_i32, [_vp, ctypes.c_char_p, _P(_vp)]),
    "bem_op_autotune": (_i32, [_vp, _vp, _P(_i32)]),
    "bem_batch_order": (_i32, [_P(_i64), _i32, _P(_i32)]),
    "bem_face_compress": (_i32, [_vp, _vp, _i64, _i64, _dbl, _P(_i32), _vp, _vp]),
    "bem_kernel_launches": (_i64, []),
    "bem_debug_set": (_i32, [_i32, _i64]),
    "bem_op_pivot_freqs": (_i32, [_vp, _P(_i32)]),
    "bem_freqs_radau2": (_i32, [_i32, _dbl, _P(_dbl), _P(_dbl)]),
    "bem_rkcq_apply": (_i32, [_vp, _i32, _dbl, _vp, _vp, _vp]),
    "bem_rkcq_solve": (_i32, [_vp, _i32, _dbl, _vp, _vp, _dbl, _i32, _P(_i32), _P(_dbl), _vp]),
    "bem_cq_forward": (_i32, [_i32, _i64, _vp, _vp, _vp]),
    "bem_cq_inverse": (_i32, [_i32, _i64, _vp, _vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class BemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st: int, ctx_ptr=None):
    if st != BEM_OK:
        msg = _lib.bem_last_error(ctx_ptr)
        raise BemError(st, msg.decode() if msg else "")


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _device_tensor(name, t, dtype, shape, device):
    """Refuses (ValueError, before any library call) a buffer the C ABI
    would misread: not a CUDA tensor on the context's device, another dtype,
    another shape, or not contiguous (the library writes by pointer and
    size, so any of these would read or write outside the buffer)."""
    if not hasattr(t, "data_ptr") or not hasattr(t, "is_cuda"):
        raise ValueError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor (it is on {t.device})")
    if device is not None and device >= 0 and t.device.index != device:
        raise ValueError(f"{name}: on cuda:{t.device.index}, the context is on cuda:{device}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if t.numel() and t.data_ptr() % 16:
        raise ValueError(f"{name}: must be 16-byte aligned")


def _cdtype(precision):
    import torch
    return torch.complex128 if precision == BEM_FP64 else torch.complex64


def options_default() -> bem_options:
    o = bem_options()
    _check(_lib.bem_options_default(ctypes.byref(o)))
    return o


def batch_order(cost) -> np.ndarray:
    """Work-list order of compress_batch: indices by decreasing cost."""
    c = np.ascontiguousarray(cost, dtype=np.int64)
    o = np.zeros(len(c), dtype=np.int32)
    _check(_lib.bem_batch_order(c.ctypes.data_as(_P(_i64)), len(c), o.ctypes.data_as(_P(_i32))))
    return o


def compress_batch(trees, n_streams: int = 4) -> list:
    """Compresses several trees (any meshes, kernels and frequency sets on
    one device) from one work list (bem_op_compress_batch)."""
    n = len(trees)
    arr = (_vp * n)(*[t._p.value for t in trees])
    out = (_vp * n)()
    st = _lib.bem_op_compress_batch(arr, n, int(n_streams), out)
    if st != BEM_OK:
        _check(st, trees[0].mesh.ctx.ptr)
    return [Operator._adopt(t, out[i]) for i, t in enumerate(trees)]


def debug_set(what: int, value: int):
    """Process-wide fault injection for tests (bem_debug_set): a failed
    staged-copy wait in the face kernel, or a cap on device allocations."""
    _check(_lib.bem_debug_set(int(what), int(value)))


def measure_peaks(device: int = 0) -> dict:
    """Measured unit throughputs on the device (bem_measure_peaks)."""
    out = np.zeros(7, dtype=np.float64)
    _check(_lib.bem_measure_peaks(int(device), out.ctypes.data_as(_P(_dbl))))
    keys = ("fp32_tflops", "fp64_tflops", "mufu_ex2_tops", "tf32_tflops_n128", "tf32_tflops_n256", "sm_mhz", "sms")
    return dict(zip(keys, out.tolist()))


def tc_selftest(A, B, device: int = 0, negate: bool = False):
    """D = A B^T, or -A B^T with negate (A 128 x 32, B 64 x 32 float32)
    through the tensor-core operand layout of the apply (bem_tc_selftest);
    returns D (128 x 64)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    if A.shape != (128, 32) or B.shape != (64, 32):
        raise ValueError("tc_selftest: A must be 128 x 32 and B 64 x 32")
    D = np.zeros((128, 64), dtype=np.float32)
    fp = _P(ctypes.c_float)
    _check(_lib.bem_tc_selftest(int(device), int(bool(negate)), A.ctypes.data_as(fp), B.ctypes.data_as(fp),
                                D.ctypes.data_as(fp)))
    return D


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(_lib.bem_kernel_launches())


def freqs_bdf2(N: int, dt: float, K: int) -> np.ndarray:
    """Frequencies of uniform BDF2 CQ (complex128, computed by the library)."""
    out = np.zeros(2 * K, dtype=np.float64)
    _check(_lib.bem_freqs_bdf2(N, dt, K, out.ctypes.data_as(_P(_dbl))))
    return out[0::2] + 1j * out[1::2]


def freqs_radau2(N: int, dt: float, half: bool = False):
    """Frequencies of constant-step 2-stage Radau IIA RK-CQ (2 (N + 1),
    complex128, k = 2 l + j; with half=True the first 2 (floor((N + 1) / 2)
    + 1) of them, the half set that real data needs) and the symbols
    (N + 1, 2, 2, 2) complex128: [l, 0] = P_l, [l, 1] = P_l^-1 with
    Delta(zeta_l) = P_l diag(mu_l) P_l^-1 (computed by the library)."""
    L = N + 1
    s = np.zeros(4 * L, dtype=np.float64)
    sym = np.zeros(16 * L, dtype=np.float64)
    _check(_lib.bem_freqs_radau2(N, dt, s.ctypes.data_as(_P(_dbl)), sym.ctypes.data_as(_P(_dbl))))
    freqs = s[0::2] + 1j * s[1::2]
    if half:
        freqs = freqs[:2 * (L // 2 + 1)]
    return freqs, (sym[0::2] + 1j * sym[1::2]).reshape(L, 2, 2, 2)


def rkcq_apply(op: "Operator", g, y, N: int, dt: float, stream=None):
    """y = RK-CQ (2-stage Radau IIA) convolution of op with the stage data g
    (bem_rkcq_apply): g real float64 device tensor (N + 1, 2, n_cols, 3),
    y (N + 1, 2, n_rows, 3); the context holds freqs_radau2(N, dt)[0]."""
    import torch
    _device_tensor("g", g, torch.float64, (N + 1, 2, op.tree.n_cols, 3), op.ctx.device)
    _device_tensor("y", y, torch.float64, (N + 1, 2, op.tree.n_rows, 3), op.ctx.device)
    _check(_lib.bem_rkcq_apply(op._p, int(N), float(dt), _dptr(g), _dptr(y), _stream_ptr(stream)), op.ctx.ptr)


def rkcq_solve(op: "Operator", b, x, N: int, dt: float, tol: float = 1e-8, max_iter: int = 300,
               stream=None, check: bool = True):
    """x = RK-CQ (2-stage Radau IIA) of op^-1 applied to the stage data b
    (bem_rkcq_solve): b, x real float64 device tensors (N + 1, 2, n, 3) of
    a square operator; returns (iterations, relative residuals) per
    frequency of the context (full or half set).  With check=False a
    frequency that did not converge is not an error."""
    import torch
    n = op.tree.n_rows
    if n != op.tree.n_cols:
        raise ValueError("rkcq_solve: the operator is not square")
    _device_tensor("b", b, torch.float64, (N + 1, 2, n, 3), op.ctx.device)
    _device_tensor("x", x, torch.float64, (N + 1, 2, n, 3), op.ctx.device)
    it = np.zeros(2 * (N + 1), dtype=np.int32)
    rr = np.zeros(2 * (N + 1), dtype=np.float64)
    st = _lib.bem_rkcq_solve(op._p, int(N), float(dt), _dptr(b), _dptr(x), float(tol), int(max_iter),
                             it.ctypes.data_as(_P(_i32)), rr.ctypes.data_as(_P(_dbl)), _stream_ptr(stream))
    if st != BEM_ERR_NOT_CONVERGED or check:
        _check(st, op.ctx.ptr)
    return it[:op.K], rr[:op.K]


def _cq_args(N, nvec, x, out):
    import torch
    for name, t in (("x", x), ("out", out)):
        _device_tensor(name, t, torch.complex128, (N + 1, nvec), None)
    if x.data_ptr() == out.data_ptr():
        raise ValueError("cq: in and out must not overlap")


def receiver_energy_grad(V: "Operator", A: "Operator", g, rec, N: int, dt: float, dV=(), dA=(),
                         tol: float = 1e-8, max_iter: int = 500, grad_g: bool = True, stream=None):
    """Receiver energy J of the traction-driven Neumann problem (V single
    layer, A = C + K double layer, node rows, the context holding the half
    set of the BDF2 frequencies of N, dt) and its adjoint gradient
    (bem_receiver_energy_grad).  g: real float64 device tensor
    (N + 1, n_tris, 3); rec: distinct node indices.  Returns (J, dJ/dg as a
    (N + 1, n_tris, 3) float64 device tensor or None, [dJ/dc_p, dJ/dc_s][:len(dV)],
    BiCGstab iterations of the forward and adjoint solves (2K))."""
    import torch
    ctx = V.ctx
    _device_tensor("g", g, torch.float64, (N + 1, V.tree.n_cols, 3), ctx.device)
    rec = np.ascontiguousarray(np.asarray(rec, dtype=np.int32))
    if len(dV) != len(dA) or len(dV) > 2:
        raise ValueError("receiver_energy_grad: dV and dA must be pairs, at most two")
    dg = torch.empty((N + 1, V.tree.n_cols, 3), dtype=torch.float64, device=g.device) if grad_g else None
    ns = len(dV)
    pv = (_vp * max(1, ns))(*[o._p for o in dV]) if ns else None
    pa = (_vp * max(1, ns))(*[o._p for o in dA]) if ns else None
    J = np.zeros(1, dtype=np.float64)
    dc = np.zeros(max(1, ns), dtype=np.float64)
    it = np.zeros(2 * V.K, dtype=np.int32)
    _check(_lib.bem_receiver_energy_grad(V._p, A._p, pv, pa, ns, int(N), float(dt), _dptr(g),
                                         rec.ctypes.data_as(_P(_i32)), len(rec), float(tol), int(max_iter),
                                         J.ctypes.data_as(_P(_dbl)), _dptr(dg) if dg is not None else None,
                                         dc.ctypes.data_as(_P(_dbl)), it.ctypes.data_as(_P(_i32)),
                                         _stream_ptr(stream)), ctx.ptr)
    return float(J[0]), dg, [float(x) for x in dc[:ns]], it


def cq_forward(N: int, nvec: int, x, out, stream=None):
    """Scaled DFT of N + 1 levels of nvec complex128 values (L x nvec)."""
    _cq_args(N, nvec, x, out)
    _check(_lib.bem_cq_forward(N, nvec, _dptr(x), _dptr(out), _stream_ptr(stream)))


def cq_inverse(N: int, nvec: int, x, out, stream=None):
    """Inverse of cq_forward (L x nvec complex128)."""
    _cq_args(N, nvec, x, out)
    _check(_lib.bem_cq_inverse(N, nvec, _dptr(x), _dptr(out), _stream_ptr(stream)))


class Context:
    """bem_ctx: options, material, frequencies (one CUDA device)."""

    def __init__(self, eps=1e-6, eps_aca=None, leaf=32, eta=2.0, precision=BEM_FP64, device=0,
                 compress_faces=1):
        o = options_default()
        o.eps = eps
        o.eps_aca = eps / 100.0 if eps_aca is None else eps_aca
        o.leaf, o.eta, o.precision, o.device, o.compress_faces = leaf, eta, precision, device, compress_faces
        self._p = ctypes.c_void_p()
        _check(_lib.bem_ctx_create(ctypes.byref(o), ctypes.byref(self._p)), None)
        self.precision = precision
        self.device = device
        self.K = 0

    @property
    def ptr(self):
        return self._p

    def close(self):
        if self._p:
            _lib.bem_ctx_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def material(self, rho, lam, mu):
        c1, c2 = _dbl(), _dbl()
        _check(_lib.bem_material_set(self._p, rho, lam, mu, ctypes.byref(c1), ctypes.byref(c2)), self._p)
        return c1.value, c2.value

    def freqs(self, s):
        s = np.asarray(s, dtype=np.complex128)
        buf = np.empty(2 * len(s))
        buf[0::2], buf[1::2] = s.real, s.imag
        _check(_lib.bem_freqs_set(self._p, buf.ctypes.data_as(_P(_dbl)), len(s)), self._p)
        self.K = len(s)

    def mesh(self, xyz, tri) -> "Mesh":
        return Mesh(self, xyz, tri)

    def face_compress(self, H, eps_face: float, out, stream=None) -> int:
        """Face ACA + QR/SVD recompression of one face H (device complex128,
        m x n x 3 x 3); out (device, >= 9 m n complex of the context's
        precision) receives U' (3m x k) then W' (3n x k) column-major.
        Returns k, or -1 when the face stays dense."""
        import torch
        m, n = int(H.shape[0]), int(H.shape[1])
        _device_tensor("H", H, torch.complex128, (m, n, 3, 3), self.device)
        if out.numel() < 9 * m * n:
            raise ValueError(f"out: needs at least {9 * m * n} complex values")
        _device_tensor("out", out, _cdtype(self.precision), tuple(out.shape), self.device)
        rk = ctypes.c_int32(-2)
        _check(_lib.bem_face_compress(self.ptr, _dptr(H), m, n, float(eps_face), ctypes.byref(rk), _dptr(out),
                                      _stream_ptr(stream)), self.ptr)
        return rk.value


class Mesh:
    def __init__(self, ctx: Context, xyz, tri):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.ctx = ctx
        self.n_nodes, self.n_tris = len(xyz), len(tri)
        self._p = ctypes.c_void_p()
        _check(_lib.bem_mesh_create(ctx.ptr, xyz.ctypes.data_as(_P(_dbl)), len(xyz),
                                    tri.ctypes.data_as(_P(_i32)), len(tri), ctypes.byref(self._p)), ctx.ptr)

    def __del__(self):
        try:
            if self._p:
                _lib.bem_mesh_destroy(self._p)
        except Exception:
            pass

    def _entry_args(self, req, out):
        import torch
        n = int(req.shape[0]) if hasattr(req, "shape") and len(req.shape) == 2 else -1
        if n < 0:
            raise ValueError("req: expected an (n, 3) int32 CUDA tensor")
        _device_tensor("req", req, torch.int32, (n, 3), self.ctx.device)
        _device_tensor("out", out, _cdtype(self.ctx.precision), (n, 3, 3), self.ctx.device)
        return n

    def entries(self, rows: int, kernel: int, req, out, stream=None):
        """req: int32 CUDA tensor (n, 3) of (row, col, k); out: complex CUDA
        tensor (n, 3, 3) (complex128 in FP64, complex64 in MIXED), both
        contiguous on the context's device (checked before the call)."""
        n = self._entry_args(req, out)
        _check(_lib.bem_entries(self._p, rows, kernel, _dptr(req), n, _dptr(out), _stream_ptr(stream)),
               self.ctx.ptr)

    def entries_noalloc(self, rows: int, kernel: int, req, out, stream=None):
        """As entries(), through bem_entries_noalloc: no device allocation in
        the call (static 1 KiB scratch, at most 16,777,216 requests)."""
        n = self._entry_args(req, out)
        _check(_lib.bem_entries_noalloc(self._p, rows, kernel, _dptr(req), n, _dptr(out), _stream_ptr(stream)),
               self.ctx.ptr)

    def tree(self, rows: int, kernel: int) -> "Tree":
        return Tree(self, rows, kernel)


class Tree:
    def __init__(self, mesh: Mesh, rows: int, kernel: int):
        self.mesh, self.rows, self.kernel = mesh, rows, kernel
        self._p = ctypes.c_void_p()
        _check(_lib.bem_tree_build(mesh._p, rows, kernel, ctypes.byref(self._p)), mesh.ctx.ptr)
        nb, nf, nr, nc = _i64(), _i64(), _i64(), _i64()
        _check(_lib.bem_tree_sizes(self._p, ctypes.byref(nb), ctypes.byref(nf), ctypes.byref(nr), ctypes.byref(nc)))
        self.n_blocks, self.n_far, self.n_rows, self.n_cols = nb.value, nf.value, nr.value, nc.value

    def __del__(self):
        try:
            if self._p:
                _lib.bem_tree_destroy(self._p)
        except Exception:
            pass

    def export(self):
        rp = np.zeros(self.n_rows, dtype=np.int32)
        cp = np.zeros(self.n_cols, dtype=np.int32)
        bl = np.zeros((self.n_blocks, 5), dtype=np.int64)
        _check(_lib.bem_tree_export(self._p, rp.ctypes.data_as(_P(_i32)), cp.ctypes.data_as(_P(_i32)),
                                    bl.ctypes.data_as(_P(_i64))))
        return rp, cp, bl

    def compress(self, stream=None) -> "Operator":
        return Operator(self, stream)


@dataclass
class Stats:
    n_blocks: int
    n_far: int
    n_aca: int
    n_dense: int
    n_rank0: int
    rank_min: int
    rank_max: int
    rank_mean: float
    stored_bytes: float
    dense_bytes: float
    compression_rate: float
    entries_evaluated: int
    t_entries_ms: float
    t_compress_ms: float
    apply_bytes: int
    t_face_ms: float
    face_launches: int
    face_alg_bytes: float
    launches: int
    n_faces: int
    n_faces_lowrank: int
    face_rank_mean: float
    t_face_aca_ms: float
    apply_bk: int
    apply_tune_ms: tuple
    apply_kernel: int
    apply_errors: int
    apply_tensor_flops: float


class Operator:
    """Compressed K-frequency tensor (bem_op)."""

    def __init__(self, tree: Tree, stream=None, _ptr=None):
        self.tree = tree
        self.ctx = tree.mesh.ctx
        self.K = self.ctx.K
        self._p = ctypes.c_void_p()
        if _ptr is not None:
            self._p = ctypes.c_void_p(_ptr)
            return
        _check(_lib.bem_op_compress(tree._p, _stream_ptr(stream), ctypes.byref(self._p)), self.ctx.ptr)

    @classmethod
    def _adopt(cls, tree: Tree, ptr) -> "Operator":
        """Wraps an operator the library already compressed (takes ownership)."""
        return cls(tree, _ptr=ptr)

    def __del__(self):
        try:
            if self._p:
                _lib.bem_op_destroy(self._p)
        except Exception:
            pass

    def _shapes(self, mode, transpose):
        """(input shape, output shape) of the apply in this mode."""
        K, nr, nc = self.K, self.tree.n_rows, self.tree.n_cols
        if mode not in (BEM_APPLY_BATCHED, BEM_APPLY_CONTRACTED):
            raise ValueError(f"mode: {mode} is neither BEM_APPLY_BATCHED nor BEM_APPLY_CONTRACTED")
        if not transpose:
            return (K, nc, 3), ((K, nr, 3) if mode == BEM_APPLY_BATCHED else (nr, 3))
        return ((K, nr, 3) if mode == BEM_APPLY_BATCHED else (nr, 3)), (K, nc, 3)

    def apply(self, X, Y, mode: int = BEM_APPLY_BATCHED, stream=None, transpose: int = 0):
        """transpose = 0: Y = C X; transpose = 1: Y = C^H X (X is then the
        row-side input, Y the column-side output).  Shapes, dtype (complex128
        in FP64, complex64 in MIXED), device and contiguity are checked first."""
        sin, sout = self._shapes(mode, transpose)
        cdt = _cdtype(self.ctx.precision)
        _device_tensor("input", X, cdt, sin, self.ctx.device)
        _device_tensor("output", Y, cdt, sout, self.ctx.device)
        _check(_lib.bem_op_apply(self._p, mode, transpose, _dptr(X), _dptr(Y), _stream_ptr(stream)), self.ctx.ptr)

    def solve(self, B, X, tol: float = 1e-8, max_iter: int = 200, stream=None, check: bool = True,
              adjoint: bool = False):
        """X_k = C(s_k)^{-1} B_k for all k (BiCGstab), or C(s_k)^{-H} B_k with
        adjoint=True; returns (iterations, relative residuals) per frequency.
        With check=False a frequency that did not converge is not an error
        (the residuals tell)."""
        if self.tree.n_rows != self.tree.n_cols:
            raise ValueError("solve: the operator is not square")
        cdt = _cdtype(self.ctx.precision)
        _device_tensor("B", B, cdt, (self.K, self.tree.n_rows, 3), self.ctx.device)
        _device_tensor("X", X, cdt, (self.K, self.tree.n_rows, 3), self.ctx.device)
        it = np.zeros(self.K, dtype=np.int32)
        rr = np.zeros(self.K, dtype=np.float64)
        fn = _lib.bem_op_solve_adjoint if adjoint else _lib.bem_op_solve
        st = fn(self._p, _dptr(B), _dptr(X), float(tol), int(max_iter),
                it.ctypes.data_as(_P(_i32)), rr.ctypes.data_as(_P(_dbl)), _stream_ptr(stream))
        if check or st != BEM_ERR_NOT_CONVERGED:
            _check(st, self.ctx.ptr)
        return it, rr

    def set_precond(self, kind: int, stream=None):
        """Preconditioner of solve(): 0 none, 1 block Jacobi (inverses of the
        3x3 diagonal blocks at every frequency; bem_op_set_precond)."""
        _check(_lib.bem_op_set_precond(self._p, int(kind), _stream_ptr(stream)), self.ctx.ptr)

    def apply_adjoint(self, Yin, Xout, mode: int = BEM_APPLY_BATCHED, stream=None):
        self.apply(Yin, Xout, mode, stream, transpose=1)

    def save(self, path: str):
        """Writes the compressed operator to a file (bem_op_save)."""
        _check(_lib.bem_op_save(self._p, os.fsencode(path)), self.ctx.ptr)

    @classmethod
    def load(cls, tree: "Tree", path: str) -> "Operator":
        """The operator of tree from a file written by save (bem_op_load)."""
        p = ctypes.c_void_p()
        _check(_lib.bem_op_load(tree._p, os.fsencode(path), ctypes.byref(p)), tree.mesh.ctx.ptr)
        return cls._adopt(tree, p.value)

    def set_apply_kernel(self, kind: int):
        """Batched-apply kernel of a MIXED operator: 1 tensor cores (default),
        0 SIMT (bem_op_set_apply_kernel)."""
        _check(_lib.bem_op_set_apply_kernel(self._p, int(kind)), self.ctx.ptr)

    def set_apply_tile(self, bk: int):
        """Frequency tile of the batched apply (16, 32 or 64)."""
        _check(_lib.bem_op_set_apply_tile(self._p, int(bk)), self.ctx.ptr)

    def autotune(self, stream=None) -> int:
        """Times the batched apply with each frequency tile on this operator
        and keeps the fastest; returns it."""
        bk = _i32(0)
        _check(_lib.bem_op_autotune(self._p, _stream_ptr(stream), ctypes.byref(bk)), self.ctx.ptr)
        return int(bk.value)

    def inner(self, G, X, mode: int = BEM_APPLY_BATCHED, stream=None) -> complex:
        """<G, C X> (bem_op_inner): sum of conj(G) times the apply of X."""
        sin, sout = self._shapes(mode, 0)
        cdt = _cdtype(self.ctx.precision)
        _device_tensor("G", G, cdt, sout, self.ctx.device)
        _device_tensor("X", X, cdt, sin, self.ctx.device)
        out = np.zeros(2, dtype=np.float64)
        _check(_lib.bem_op_inner(self._p, mode, _dptr(G), _dptr(X), out.ctypes.data_as(_P(_dbl)),
                                 _stream_ptr(stream)), self.ctx.ptr)
        return complex(out[0], out[1])

    def dense(self, out, stream=None):
        """Dense reconstruction into out (n_rows, n_cols, K, 3, 3)."""
        _device_tensor("out", out, _cdtype(self.ctx.precision),
                       (self.tree.n_rows, self.tree.n_cols, self.K, 3, 3), self.ctx.device)
        _check(_lib.bem_op_dense(self._p, _dptr(out), _stream_ptr(stream)), self.ctx.ptr)

    def stats(self) -> Stats:
        s = bem_op_stats()
        _check(_lib.bem_op_stats_get(self._p, ctypes.byref(s)))
        vals = [getattr(s, f) for f, _ in bem_op_stats._fields_]
        return Stats(*[tuple(v) if isinstance(v, ctypes.Array) else v for v in vals])

    def blocks(self) -> np.ndarray:
        out = np.zeros((self.tree.n_blocks, 4), dtype=np.int64)
        _check(_lib.bem_op_blocks(self._p, out.ctypes.data_as(_P(_i64))))
        return out

    def slot_stats(self):
        """Per 3D-ACA iteration: (face-kernel ms, active entries) arrays."""
        n = _i32(0)
        _check(_lib.bem_op_slot_stats(self._p, 0, None, None, ctypes.byref(n)))
        ms = np.zeros(n.value, dtype=np.float64)
        en = np.zeros(n.value, dtype=np.int64)
        _check(_lib.bem_op_slot_stats(self._p, n.value, ms.ctypes.data_as(_P(_dbl)), en.ctypes.data_as(_P(_i64)),
                                      ctypes.byref(n)))
        return ms, en

    def pivot_freqs(self) -> np.ndarray:
        """(n_blocks, K) int32: frequency index k_d of face d of each block
        (d < rank), -1 elsewhere and for dense and rank-0 blocks."""
        out = np.zeros((self.tree.n_blocks, self.K), dtype=np.int32)
        _check(_lib.bem_op_pivot_freqs(self._p, out.ctypes.data_as(_P(_i32))))
        return out

    def face_ranks(self) -> np.ndarray:
        """(K, n_blocks) int32: rank of each low-rank face, -1 dense face, -2 no face."""
        out = np.zeros((self.K, self.tree.n_blocks), dtype=np.int32)
        _check(_lib.bem_op_face_ranks(self._p, out.ctypes.data_as(_P(_i32))))
        return out
