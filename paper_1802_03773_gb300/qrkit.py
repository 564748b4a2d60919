"""Python binding of the C-ABI library libqrkit.so (argument marshalling only).

Every numerical step runs in the library's CUDA kernels; this module only checks tensor
dtypes/devices, passes raw device pointers and the CUDA stream, and turns status codes
into exceptions.  If the library is missing it raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqrkit.so")

FP64, FP32_REFINED, FP32 = 0, 1, 2
PRECISION = {"fp64": FP64, "fp32_refined": FP32_REFINED, "fp32": FP32}
STRUCT_BLOCKS, STRUCT_BANDED = 0, 1
BAND_AUTO, BAND_SWEEP, BAND_PARALLEL = 0, 1, 2
COUPLED_NONE, COUPLED_DENSE, COUPLED_WINDOW = 0, 1, 2
RESIDUAL_DOT2, RESIDUAL_FP64 = 0, 1

STATUS = {0: "QRKIT_OK", 1: "QRKIT_EINVAL", 2: "QRKIT_ENOMEM", 3: "QRKIT_ECUDA",
          4: "QRKIT_ESINGULAR", 5: "QRKIT_ENONFINITE", 6: "QRKIT_ETIMEOUT",
          7: "QRKIT_ENOTCONV", 8: "QRKIT_EUNSUPPORTED", 9: "QRKIT_ESTATE"}


class QRKitError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Structure(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("num_blocks", ctypes.c_int64),
        ("block_rows", ctypes.c_void_p),
        ("block_cols", ctypes.c_void_p),
        ("coupled_kind", ctypes.c_int32),
        ("shared_cols", ctypes.c_int64),
        ("window", ctypes.c_int32),
        ("window_start", ctypes.c_void_p),
        ("rows", ctypes.c_int64),
        ("cols", ctypes.c_int64),
        ("rows_per_col", ctypes.c_int32),
        ("band_window", ctypes.c_int32),
        ("instance_cols", ctypes.c_void_p),
        ("num_segments", ctypes.c_int64),
        ("segment_cols", ctypes.c_void_p),
        ("segment_blocks", ctypes.c_void_p),
        ("band_solver", ctypes.c_int32),
        ("band_row_start", ctypes.c_void_p),
        ("instance_rows", ctypes.c_void_p),
    ]


class LMProblem(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32),
        ("num_problems", ctypes.c_int64),
        ("num_points", ctypes.c_void_p),
        ("control_points", ctypes.c_void_p),
        ("data", ctypes.c_void_p),
    ]


class LMState(ctypes.Structure):
    _fields_ = [
        ("lambda_", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("cost", ctypes.c_double),
        ("cost_new", ctypes.c_double),
        ("pred", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("accepted", ctypes.c_int32),
        ("done", ctypes.c_int32),
        ("iteration", ctypes.c_int64),
    ]


class Metadata(ctypes.Structure):
    _fields_ = [
        ("damped", ctypes.c_int32),
        ("num_blocks", ctypes.c_int64),
        ("rows", ctypes.c_int64),
        ("cols", ctypes.c_int64),
        ("values", ctypes.c_int64),
        ("aug_rows", ctypes.c_int64),
        ("val_off", ctypes.c_void_p),
        ("row_off", ctypes.c_void_p),
        ("col_off", ctypes.c_void_p),
        ("row_order", ctypes.c_void_p),
        ("r_row_ptr", ctypes.c_void_p),
        ("r_col_idx", ctypes.c_void_p),
        ("r_capacity", ctypes.c_int64),
        ("r_nnz", ctypes.c_int64),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("refine_steps_max", ctypes.c_int32),
        ("refined_blocks", ctypes.c_int64),
        ("residual_norm", ctypes.c_double),
        ("optimality_norm", ctypes.c_double),
        ("optimality_scale", ctypes.c_double),
    ]


MODEL_CURVEFIT = 0
MLP_FEATURES, MLP_CLASSES, MLP_PARAMS = 16, 8, 5768
MLP_MULTIPLIERS = (1e-2, 1e-1, 1.0 / 3.0, 0.5, 1.0, 2.0, 4.0, 10.0)

_VP = ctypes.c_void_p
_SIGS = {
    "qrkit_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _VP, ctypes.c_int]),
    "qrkit_destroy": (None, [_VP]),
    "qrkit_last_error": (ctypes.c_char_p, [_VP]),
    "qrkit_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "qrkit_plan": (ctypes.c_int, [_VP, ctypes.POINTER(Structure)]),
    "qrkit_factor_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_double, _VP, _VP, ctypes.c_int]),
    "qrkit_get_factor": (ctypes.c_int, [_VP, _VP, _VP]),
    "qrkit_set_refinement": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int]),
    "qrkit_set_wait_limit": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "qrkit_more_solve": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, _VP]),
    "qrkit_more_trust_region": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_double), _VP, ctypes.POINTER(ctypes.c_int)]),
    "qrkit_column_sumsq": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "qrkit_norms_from_sumsq": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP]),
    "qrkit_get_reduced_r": (ctypes.c_int, [_VP, _VP]),
    "qrkit_solve_blocks": (ctypes.c_int, [_VP, _VP, _VP]),
    "qrkit_dense_lstsq": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_int64, _VP, _VP,
                                         ctypes.POINTER(ctypes.c_double)]),
    "qrkit_get_info": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.POINTER(Info)]),
    "qrkit_lm_trial": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_int, _VP,
                                      ctypes.POINTER(ctypes.c_double)]),
    "qrkit_peak_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "qrkit_host_link_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double)]),
    "qrkit_nielsen_update": (ctypes.c_int, [ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
    "qrkit_get_band_factor": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "qrkit_factor": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_double]),
    "qrkit_apply_qt": (ctypes.c_int, [_VP, _VP, _VP]),
    "qrkit_solve_r": (ctypes.c_int, [_VP, _VP, _VP]),
    "qrkit_solve": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int]),
    "qrkit_normal_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_double, _VP]),
    "qrkit_set_window_start": (ctypes.c_int, [_VP, _VP]),
    "qrkit_get_row_order": (ctypes.c_int, [_VP, _VP]),
    "qrkit_lm_plan": (ctypes.c_int, [_VP, ctypes.POINTER(LMProblem)]),
    "qrkit_lm_step": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int]),
    "qrkit_lm_run": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    "qrkit_mlp_init": (ctypes.c_int, [_VP, _VP]),
    "qrkit_mlp_params": (ctypes.c_int, [_VP, _VP]),
    "qrkit_mlp_forward": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP]),
    "qrkit_mlp_train_step": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_float, _VP, _VP]),
    "qrkit_lm_set_policy": (ctypes.c_int, [_VP, ctypes.c_int]),
    "qrkit_lm_residual": (ctypes.c_int, [_VP, _VP, _VP]),
    "qrkit_lm_linearize": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "qrkit_lm_features": (ctypes.c_int, [_VP, _VP]),
    "qrkit_autotune": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_char_p, ctypes.c_char_p,
                                       ctypes.c_int64]),
    "qrkit_apply_tuning": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "qrkit_sync_status": (ctypes.c_int, [_VP]),
    "qrkit_block_solve_noalloc": (ctypes.c_int, [ctypes.c_int, _VP, ctypes.c_int, ctypes.c_int64, _VP,
                                                 _VP, _VP, _VP, _VP, ctypes.c_int]),
    "qrkit_launch_count": (ctypes.c_int64, [_VP]),
    "qrkit_band_order": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, _VP, _VP, _VP, _VP, _VP, _VP]),
    "qrkit_structure_metadata": (ctypes.c_int, [ctypes.POINTER(Structure), ctypes.POINTER(Metadata)]),
    "qrkit_task_layout": (ctypes.c_int, [ctypes.c_int64, _VP, _VP, ctypes.c_int64, ctypes.c_int, _VP, _VP, _VP,
                                         ctypes.c_int64]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libqrkit.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libqrkit.so not found at {path}; build it first (the library has no "
                          "fallback implementation)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def block_solve_noalloc(n, m, J, b, p, precision="fp32_refined", refine_steps=2, stream=None):
    """qrkit_block_solve_noalloc: the batched block solve without any device allocation.

    n, m: host arrays of block shapes; J, b, p: CUDA tensors (inputs / output).  Blocks until
    the solve has finished and raises QRKitError on a non-zero status.
    """
    import torch
    lib = load()
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    n = np.ascontiguousarray(n, dtype=np.uint8)
    m = np.ascontiguousarray(m, dtype=np.uint8)
    dev = J.device.index if J.device.index is not None else torch.cuda.current_device()
    if stream is None:
        stream = torch.cuda.current_stream(J.device)
    st = lib.qrkit_block_solve_noalloc(dev, _VP(stream.cuda_stream), prec, n.shape[0],
                                       n.ctypes.data, m.ctypes.data, _ptr(J), _ptr(b), _ptr(p),
                                       int(refine_steps))
    if st != 0:
        raise QRKitError(st, "qrkit_block_solve_noalloc failed")


def task_layout(n, m, supertile=65536, key_major=False):
    """qrkit_task_layout: the warp tasks a block plan builds, computed on the host.

    n, m: host arrays of block shapes.  Returns (key (T,) int32, slots (T, 32, 4) int64): per
    task its shape key and, per slot, (block, first value, first row, first column), -1 where
    the slot is unused.  Raises QRKitError on a non-zero status.
    """
    lib = load()
    n = np.ascontiguousarray(n, dtype=np.uint8)
    m = np.ascontiguousarray(m, dtype=np.uint8)
    count = ctypes.c_int64(0)
    st = lib.qrkit_task_layout(n.shape[0], n.ctypes.data, m.ctypes.data, int(supertile), int(bool(key_major)),
                               ctypes.addressof(count), None, None, 0)
    if st != 0:
        raise QRKitError(st, "qrkit_task_layout failed")
    T = count.value
    key = np.empty(T, dtype=np.int32)
    slots = np.empty((T, 32, 4), dtype=np.int64)
    st = lib.qrkit_task_layout(n.shape[0], n.ctypes.data, m.ctypes.data, int(supertile), int(bool(key_major)),
                               ctypes.addressof(count), key.ctypes.data, slots.ctypes.data, T)
    if st != 0:
        raise QRKitError(st, "qrkit_task_layout failed")
    return key, slots


def peak_probe(device=0, kind="tf32"):
    """qrkit_peak_probe: TFLOP/s of "fp32" / "fp64" FMA or "tf32" tensor-core MMA on `device`."""
    lib = load()
    k = {"fp32": 0, "fp64": 1, "tf32": 2}[kind]
    v = ctypes.c_double(0.0)
    st = lib.qrkit_peak_probe(int(device), k, ctypes.byref(v))
    if st != 0:
        raise QRKitError(st, "qrkit_peak_probe failed")
    return v.value


def host_link_probe(device=0, nbytes=1 << 30):
    """qrkit_host_link_probe: (copy-engine GB/s, kernel zero-copy read GB/s) host -> device."""
    lib = load()
    c, k = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = lib.qrkit_host_link_probe(int(device), int(nbytes), ctypes.byref(c), ctypes.byref(k))
    if st != 0:
        raise QRKitError(st, "qrkit_host_link_probe failed")
    return c.value, k.value


def nielsen_update(rho, lam, nu):
    """qrkit_nielsen_update on the host: returns (lambda, nu, accepted)."""
    lib = load()
    l, v, a = ctypes.c_double(lam), ctypes.c_double(nu), ctypes.c_int32(0)
    st = lib.qrkit_nielsen_update(float(rho), ctypes.byref(l), ctypes.byref(v), ctypes.byref(a))
    if st != 0:
        raise QRKitError(st, "qrkit_nielsen_update failed")
    return l.value, v.value, bool(a.value)


def block_structure(n, m, coupled=COUPLED_NONE, shared_cols=0, window=0, window_start=None,
                    segment_cols=None, segment_blocks=None):
    """A QRKIT_STRUCT_BLOCKS descriptor and the arrays it points to (keep them alive)."""
    n = np.ascontiguousarray(n, dtype=np.uint8)
    m = np.ascontiguousarray(m, dtype=np.uint8)
    s = Structure()
    s.kind = STRUCT_BLOCKS
    s.num_blocks = n.shape[0]
    s.block_rows = n.ctypes.data
    s.block_cols = m.ctypes.data
    s.coupled_kind = int(coupled)
    s.shared_cols = int(shared_cols)
    s.window = int(window)
    keep = [n, m]
    if window_start is not None:
        ws = np.ascontiguousarray(window_start, dtype=np.int32)
        s.window_start = ws.ctypes.data
        keep.append(ws)
    if segment_cols is not None:
        sc = np.ascontiguousarray(segment_cols, dtype=np.int64)
        sb = np.ascontiguousarray(segment_blocks, dtype=np.int64)
        s.num_segments = sc.shape[0]
        s.segment_cols = sc.ctypes.data
        s.segment_blocks = sb.ctypes.data
        keep += [sc, sb]
    return s, keep


def structure_metadata(n, m, damped, **kw):
    """qrkit_structure_metadata: (val_off, row_off, col_off, row_order, r_row_ptr, r_col_idx)."""
    lib = load()
    s, keep = block_structure(n, m, **kw)
    md = Metadata()
    md.damped = 1 if damped else 0
    st = lib.qrkit_structure_metadata(ctypes.byref(s), ctypes.byref(md))
    if st != 0:
        raise QRKitError(st, "qrkit_structure_metadata failed")
    K, N = md.num_blocks, md.cols
    vo, ro, co = (np.empty(K + 1, dtype=np.int64) for _ in range(3))
    order = np.empty(max(md.aug_rows, 1), dtype=np.int64)
    ptr = np.empty(N + 1, dtype=np.int64)
    md.val_off, md.row_off, md.col_off = vo.ctypes.data, ro.ctypes.data, co.ctypes.data
    md.row_order, md.r_row_ptr = order.ctypes.data, ptr.ctypes.data
    st = lib.qrkit_structure_metadata(ctypes.byref(s), ctypes.byref(md))
    if st != 0:
        raise QRKitError(st, "qrkit_structure_metadata failed")
    idx = np.empty(max(md.r_nnz, 1), dtype=np.int32)
    md.r_col_idx, md.r_capacity = idx.ctypes.data, md.r_nnz
    st = lib.qrkit_structure_metadata(ctypes.byref(s), ctypes.byref(md))
    if st != 0:
        raise QRKitError(st, "qrkit_structure_metadata failed")
    del keep
    return vo, ro, co, order[:md.aug_rows], ptr, idx[:md.r_nnz]


def band_order(rows, cols, row_ptr, col_idx):
    """qrkit_band_order: P_c, P_r, row starts and band width exposing a banded structure.

    row_ptr (rows + 1), col_idx: the CSR pattern of A.  Returns (col_perm int32, row_perm
    int64, row_start int32, width).  Raises QRKitError on a non-zero status.
    """
    lib = load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    col_perm = np.empty(int(cols), dtype=np.int32)
    row_perm = np.empty(max(int(rows), 1), dtype=np.int64)
    row_start = np.empty(max(int(rows), 1), dtype=np.int32)
    width = ctypes.c_int32(0)
    st = lib.qrkit_band_order(int(rows), int(cols), row_ptr.ctypes.data, col_idx.ctypes.data if col_idx.size else None,
                              col_perm.ctypes.data, row_perm.ctypes.data, row_start.ctypes.data,
                              ctypes.addressof(width))
    if st != 0:
        raise QRKitError(st, "qrkit_band_order failed")
    return col_perm, row_perm[:int(rows)], row_start[:int(rows)], int(width.value)


def declared_symbols():
    return list(_SIGS)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """A qrkit context bound to one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None, precision="fp32_refined"):
        import torch
        self._torch = torch
        self.lib = load()
        self.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        self.dtype = torch.float64 if self.precision == FP64 else torch.float32
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = _VP()
        st = self.lib.qrkit_create(ctypes.byref(h), device, _VP(stream.cuda_stream), self.precision)
        if st != 0:
            raise QRKitError(st, "qrkit_create failed")
        self.h = h
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.qrkit_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise QRKitError(st, self.lib.qrkit_last_error(self.h).decode())

    def _t(self, t, name, allow_none=False):
        if t is None:
            if allow_none:
                return None
            raise ValueError(f"{name} is required")
        if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous {self.dtype} tensor on {self.device}")
        return _ptr(t)

    # ---- structure plan ----
    def plan_blocks(self, n, m, coupled=COUPLED_NONE, shared_cols=0, window=0, window_start=None,
                    segment_cols=None, segment_blocks=None):
        n = np.ascontiguousarray(n, dtype=np.uint8)
        m = np.ascontiguousarray(m, dtype=np.uint8)
        s = Structure()
        s.kind = STRUCT_BLOCKS
        s.num_blocks = n.shape[0]
        s.block_rows = n.ctypes.data
        s.block_cols = m.ctypes.data
        s.coupled_kind = int(coupled)
        s.shared_cols = int(shared_cols)
        s.window = int(window)
        ws = None
        if window_start is not None:
            ws = np.ascontiguousarray(window_start, dtype=np.int32)
            s.window_start = ws.ctypes.data
        sc = sb = None
        if segment_cols is not None:
            sc = np.ascontiguousarray(segment_cols, dtype=np.int64)
            sb = np.ascontiguousarray(segment_blocks, dtype=np.int64)
            s.num_segments = sc.shape[0]
            s.segment_cols = sc.ctypes.data
            s.segment_blocks = sb.ctypes.data
        self._check(self.lib.qrkit_plan(self.h, ctypes.byref(s)))
        self._keep = [n, m, ws, sc, sb]

    def set_window_start(self, start):
        """start: int32 CUDA tensor (one entry per block)."""
        import torch
        if start.device != self.device or start.dtype != torch.int32 or not start.is_contiguous():
            raise ValueError("start: expected a contiguous int32 tensor on the context's device")
        self._check(self.lib.qrkit_set_window_start(self.h, _ptr(start)))
        self._starts = start

    def get_row_order(self, order):
        """order: int64 CUDA tensor, one entry per reduced row."""
        self._check(self.lib.qrkit_get_row_order(self.h, _ptr(order)))

    def plan_banded(self, instance_cols, rows_per_col=4, window=8, solver=BAND_AUTO, row_start=None,
                    instance_rows=None):
        """row_start: optional explicit first column of every row (instances back to back, local
        columns, non-decreasing per instance); instance_rows: rows per instance with it."""
        cols = np.ascontiguousarray(np.atleast_1d(instance_cols), dtype=np.int64)
        s = Structure()
        s.kind = STRUCT_BANDED
        s.num_blocks = cols.shape[0]
        s.instance_cols = cols.ctypes.data
        s.cols = int(cols[0])
        s.rows_per_col = int(rows_per_col)
        s.band_window = int(window)
        s.band_solver = int(solver)
        rs = ir = None
        if row_start is not None:
            rs = np.ascontiguousarray(row_start, dtype=np.int32)
            s.band_row_start = rs.ctypes.data if rs.size else None
            s.rows = int(rs.shape[0])
            if instance_rows is not None:
                ir = np.ascontiguousarray(np.atleast_1d(instance_rows), dtype=np.int64)
                s.instance_rows = ir.ctypes.data
        self._check(self.lib.qrkit_plan(self.h, ctypes.byref(s)))
        self._keep = [cols, rs, ir]

    def get_band_factor(self, Rw=None, c=None, res2=None):
        """res2: a numpy float64 array (one entry per instance) or None."""
        rp = None if res2 is None else res2.ctypes.data_as(ctypes.c_void_p)
        self._check(self.lib.qrkit_get_band_factor(self.h, self._t(Rw, "Rw", True),
                                                   self._t(c, "c", True), rp))

    # ---- solves ----
    def factor_solve(self, J, b, p, qtb=None, D=None, lam=0.0, refine_steps=1):
        self._check(self.lib.qrkit_factor_solve(
            self.h, self._t(J, "J"), self._t(b, "b"), self._t(D, "D", True), float(lam),
            self._t(p, "p"), self._t(qtb, "qtb", True), int(refine_steps)))

    def set_refinement(self, select=2e-6, residual="dot2"):
        """Block refinement settings: selection threshold and residual precision ("dot2" or "fp64")."""
        mode = {"dot2": RESIDUAL_DOT2, "fp64": RESIDUAL_FP64}[residual] if isinstance(residual, str) else int(residual)
        self._check(self.lib.qrkit_set_refinement(self.h, float(select), mode))

    def lm_trial(self, J, S, b, p, D=None, lam=1e-3, refine_steps=1):
        """One LM trial step for the caller's own model: solve into p, return the predicted decrease."""
        pred = ctypes.c_double(0.0)
        self._check(self.lib.qrkit_lm_trial(self.h, self._t(J, "J"), self._t(S, "S", True), self._t(b, "b"),
                                            self._t(D, "D", True), float(lam), int(refine_steps), self._t(p, "p"),
                                            ctypes.byref(pred)))
        self._refs = (J, S, D)
        return pred.value

    def info(self, J, b, p, D=None, lam=0.0):
        """qrkit_get_info: dict of the solution's diagnostics (block-diagonal plans)."""
        out = Info()
        self._check(self.lib.qrkit_get_info(self.h, self._t(J, "J"), self._t(b, "b"), self._t(p, "p"),
                                            self._t(D, "D", True), float(lam), ctypes.byref(out)))
        return {k: getattr(out, k) for k, _ in Info._fields_}

    # ---- pieces of a dense-S solve split over several contexts ----
    def column_sumsq(self, J, S, sq):
        """sq: float64 CUDA tensor of N entries (squared column sums of J)."""
        self._check(self.lib.qrkit_column_sumsq(self.h, self._t(J, "J"), self._t(S, "S", True), _ptr(sq)))

    def norms_from_sumsq(self, sq, D):
        self._check(self.lib.qrkit_norms_from_sumsq(self.h, _ptr(sq), int(sq.numel()), self._t(D, "D")))

    def reduced_r(self, R):
        self._check(self.lib.qrkit_get_reduced_r(self.h, self._t(R, "R")))

    def solve_blocks(self, qtb, p):
        self._check(self.lib.qrkit_solve_blocks(self.h, self._t(qtb, "qtb"), self._t(p, "p")))

    def dense_lstsq(self, A, b, x):
        """A: (N, M) contiguous tensor viewed as M x N column-major (A.T of a row-major M x N)."""
        N, M = A.shape
        r2 = ctypes.c_double(0.0)
        self._check(self.lib.qrkit_dense_lstsq(self.h, int(M), int(N), self._t(A, "A"), int(M), self._t(b, "b"),
                                               self._t(x, "x"), ctypes.byref(r2)))
        return r2.value

    def more_solve(self, qtb, p, D=None, lam=0.0):
        """Moré's second factorization for the stored block factor (qtb from factor_solve)."""
        self._check(self.lib.qrkit_more_solve(self.h, self._t(qtb, "qtb"), self._t(D, "D", True), float(lam),
                                              self._t(p, "p")))

    def more_trust_region(self, qtb, p, delta, D=None, sigma=0.1, max_iter=30):
        """Moré's trust-region lambda for the stored block factor (qrkit_more_trust_region):
        returns (lambda, iterations); p receives the step."""
        lam = ctypes.c_double(0.0)
        it = ctypes.c_int(0)
        self._check(self.lib.qrkit_more_trust_region(self.h, self._t(qtb, "qtb"), self._t(D, "D", True), float(delta),
                                                     float(sigma), int(max_iter), ctypes.byref(lam),
                                                     self._t(p, "p"), ctypes.byref(it)))
        return lam.value, it.value

    def set_wait_limit(self, polls):
        """Poll limit of the bounded device waits (0 makes them run out: QRKIT_ETIMEOUT)."""
        self._check(self.lib.qrkit_set_wait_limit(self.h, int(polls)))

    def factor(self, J, S=None, D=None, lam=0.0):
        self._check(self.lib.qrkit_factor(self.h, self._t(J, "J"), self._t(S, "S", True),
                                          self._t(D, "D", True), float(lam)))
        self._refs = (J, S, D)   # the library reads J and S again during refinement

    def apply_qt(self, b, qtb):
        self._check(self.lib.qrkit_apply_qt(self.h, self._t(b, "b"), self._t(qtb, "qtb")))

    def solve_r(self, qtb, p):
        self._check(self.lib.qrkit_solve_r(self.h, self._t(qtb, "qtb"), self._t(p, "p")))

    def solve(self, b, p, refine_steps=1):
        self._check(self.lib.qrkit_solve(self.h, self._t(b, "b"), self._t(p, "p"), int(refine_steps)))

    def normal_solve(self, J, S, b, p, D=None, lam=0.0):
        """Normal equations by Cholesky (comparison path; no refinement)."""
        self._check(self.lib.qrkit_normal_solve(self.h, self._t(J, "J"), self._t(S, "S", True), self._t(b, "b"),
                                                self._t(D, "D", True), float(lam), self._t(p, "p")))

    def get_factor(self, factor=None, tau=None):
        self._check(self.lib.qrkit_get_factor(self.h, self._t(factor, "factor", True),
                                              self._t(tau, "tau", True)))

    # ---- Levenberg-Marquardt on the device ----
    def lm_plan(self, num_points, control_points, data):
        """data: float64 CUDA tensor (sum P_k, 2), kept alive by the context."""
        import torch
        if data.device != self.device or data.dtype != torch.float64 or not data.is_contiguous():
            raise ValueError("data: expected a contiguous float64 tensor on the context's device")
        npts = np.ascontiguousarray(np.atleast_1d(num_points), dtype=np.int64)
        kc = np.ascontiguousarray(np.atleast_1d(control_points), dtype=np.int32)
        pr = LMProblem()
        pr.model = MODEL_CURVEFIT
        pr.num_problems = npts.shape[0]
        pr.num_points = npts.ctypes.data
        pr.control_points = kc.ctypes.data
        pr.data = data.data_ptr()
        self._check(self.lib.qrkit_lm_plan(self.h, ctypes.byref(pr)))
        self._lm_data = data
        self._lm_B = int(npts.shape[0])

    def lm_states(self, lam=1e-3, nu=2.0):
        st = (LMState * self._lm_B)()
        lams = np.broadcast_to(np.asarray(lam, dtype=np.float64), (self._lm_B,))
        for k in range(self._lm_B):
            st[k].lambda_ = float(lams[k])
            st[k].nu = nu
        return st

    def _lm_x(self, x):
        import torch
        if x.device != self.device or x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("x: expected a contiguous float64 tensor on the context's device")
        return _ptr(x)

    def lm_step(self, x, states, refine_steps=1):
        self._check(self.lib.qrkit_lm_step(self.h, self._lm_x(x), ctypes.cast(states, _VP), int(refine_steps)))
        return states

    def lm_run(self, x, states, max_iter=100, ftol=1e-12, refine_steps=1, use_graph=True):
        self._check(self.lib.qrkit_lm_run(self.h, self._lm_x(x), ctypes.cast(states, _VP), int(max_iter),
                                          float(ftol), int(refine_steps), 1 if use_graph else 0))
        return states

    # ---- damping-policy MLP ----
    def mlp_init(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (MLP_PARAMS,):
            raise ValueError(f"params: expected {MLP_PARAMS} float32 values")
        self._check(self.lib.qrkit_mlp_init(self.h, p.ctypes.data))

    def mlp_params(self):
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        self._check(self.lib.qrkit_mlp_params(self.h, out.ctypes.data))
        return out

    def _f32(self, t, name, cols=None):
        import torch
        if t.device != self.device or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous float32 tensor on the context's device")
        return _ptr(t)

    def mlp_forward(self, X, logits):
        self._check(self.lib.qrkit_mlp_forward(self.h, self._f32(X, "X"), int(X.shape[0]), self._f32(logits, "logits")))

    def mlp_train_step(self, X, labels, lr, grad=None):
        import torch
        if labels.device != self.device or labels.dtype != torch.int32 or not labels.is_contiguous():
            raise ValueError("labels: expected a contiguous int32 tensor on the context's device")
        loss = ctypes.c_float(0.0)
        self._check(self.lib.qrkit_mlp_train_step(self.h, self._f32(X, "X"), _ptr(labels), int(X.shape[0]),
                                                  float(lr), ctypes.byref(loss),
                                                  None if grad is None else self._f32(grad, "grad")))
        return float(loss.value)

    def lm_residual(self, x, f):
        import torch
        if f.device != self.device or f.dtype != torch.float64 or not f.is_contiguous():
            raise ValueError("f: expected a contiguous float64 tensor on the context's device")
        self._check(self.lib.qrkit_lm_residual(self.h, self._lm_x(x), _ptr(f)))

    def lm_linearize(self, x, J=None, S=None, b=None, start=None):
        import torch
        if start is not None and (start.device != self.device or start.dtype != torch.int32):
            raise ValueError("start: expected an int32 tensor on the context's device")
        self._check(self.lib.qrkit_lm_linearize(self.h, self._lm_x(x), self._t(J, "J", True), self._t(S, "S", True),
                                                self._t(b, "b", True), _ptr(start)))

    def lm_set_policy(self, use_mlp):
        self._check(self.lib.qrkit_lm_set_policy(self.h, 1 if use_mlp else 0))

    def lm_features(self, out):
        self._check(self.lib.qrkit_lm_features(self.h, self._f32(out, "features")))

    def autotune(self, J, b, p, refine_steps=2, cache_path=None):
        """Time candidate launch configurations for the current plan; returns the choice."""
        buf = ctypes.create_string_buffer(256)
        path = None if cache_path is None else os.fsencode(cache_path)
        self._check(self.lib.qrkit_autotune(self.h, self._t(J, "J"), self._t(b, "b"), self._t(p, "p"),
                                            int(refine_steps), path, buf, 256))
        return buf.value.decode()

    def apply_tuning(self, choice):
        """Apply a configuration in the text form autotune returns, without timing."""
        self._check(self.lib.qrkit_apply_tuning(self.h, str(choice).encode()))

    def sync_status(self):
        self._check(self.lib.qrkit_sync_status(self.h))

    @property
    def launch_count(self):
        return int(self.lib.qrkit_launch_count(self.h))
