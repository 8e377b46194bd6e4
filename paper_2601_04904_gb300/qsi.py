"""ctypes binding of libqsi (include/qsi.h): argument marshalling only.

Every step of the solve runs in the CUDA library; this module converts dicts of
torch tensors (device) or numpy arrays (host) into the C structs and raises
``QsiError`` on a non-zero status.  Importing it loads ``libqsi.so`` and fails
loudly if the library has not been built (``__graft_entry__.build()``).

BTA containers are dicts with keys diag, upper, lower, arrow_r, arrow_b, tip
(see ``inputs.py``); device containers hold complex128 CUDA tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqsi.so")
KEYS = ("diag", "upper", "lower", "arrow_r", "arrow_b", "tip")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(LIB_PATH)

OK, ERR_ARG, ERR_OOM, ERR_SINGULAR, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY, ERR_STATE, ERR_UNSUPPORTED, ERR_ACCURACY = range(10)
FP64, FP64_EMU, MIXED, SPLIT3 = 0, 1, 2, 3
MAX_RHS = 4  # QSI_MAX_RHS
ASSUME_ANTIHERMITIAN_B = 1  # QSI_ASSUME_ANTIHERMITIAN_B
TWISTED_SPLIT = 2  # QSI_TWISTED_SPLIT
PRECISIONS = {"fp64": FP64, "fp64_emu": FP64_EMU, "mixed": MIXED, "split3": SPLIT3}
NOALLOC_MAX_B = 1024  # QSI_NOALLOC_MAX_B


class Shape(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int32), ("b", ctypes.c_int32), ("a", ctypes.c_int32)]


class BTA(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in KEYS]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("gemm_launches", ctypes.c_uint64),
                ("inv_launches", ctypes.c_uint64), ("gemm_flops", ctypes.c_double),
                ("gemm_ms", ctypes.c_double), ("inv_ms", ctypes.c_double), ("tc_launches", ctypes.c_uint64),
                ("tc_flops", ctypes.c_double), ("tc_ms", ctypes.c_double), ("panel_launches", ctypes.c_uint64),
                ("panel_flops", ctypes.c_double), ("panel_ms", ctypes.c_double),
                ("tc_aux_launches", ctypes.c_uint64), ("tc_aux_ms", ctypes.c_double),
                ("panel32_launches", ctypes.c_uint64), ("panel32_flops", ctypes.c_double),
                ("panel32_ms", ctypes.c_double), ("graph_launches", ctypes.c_uint64),
                ("partition_kappa", ctypes.c_double), ("partition_fallbacks", ctypes.c_uint64),
                ("tc_exp_ms", ctypes.c_double), ("tc_conv_ms", ctypes.c_double), ("tc_crt_ms", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("shape", Shape), ("precision", ctypes.c_int), ("A", ctypes.POINTER(BTA)), ("B", ctypes.POINTER(BTA)),
                ("GR", ctypes.POINTER(BTA)), ("GL", ctypes.POINTER(BTA))]


class Move(ctypes.Structure):
    """qsi_move: one block move of the partitioned solve's plan."""
    _fields_ = [("dst", ctypes.c_int32), ("ldd", ctypes.c_int32), ("rows", ctypes.c_int32), ("cols", ctypes.c_int32),
                ("fill", ctypes.c_int32), ("src", ctypes.c_int32 * 3), ("lds", ctypes.c_int32 * 3),
                ("cnt", ctypes.c_int32 * 3), ("dst_off", ctypes.c_int64), ("off", ctypes.c_int64 * 3),
                ("stride", ctypes.c_int64 * 3)]


PLAN_ARRAYS = 6 * 6 * (1 + MAX_RHS)  # QSI_PLAN_ARRAYS


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("slot", ctypes.c_int32), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("device_start_ms", ctypes.c_double),
                ("device_end_ms", ctypes.c_double)]


_P = ctypes.c_void_p
_S = ctypes.c_int
_sig = {
    "qsi_create": (_S, [ctypes.POINTER(_P), ctypes.c_int, _P]),
    "qsi_destroy": (_S, [_P]),
    "qsi_last_error": (ctypes.c_char_p, [_P]),
    "qsi_selftest_wait_timeout": (_S, [_P, ctypes.c_int32]),
    "qsi_set_flags": (_S, [_P, ctypes.c_uint32]),
    "qsi_batched_config": (_S, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
    "qsi_autotune_cache_store": (_S, [ctypes.c_char_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                      ctypes.c_double]),
    "qsi_autotune_cache_lookup": (_S, [ctypes.c_char_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int32)]),
    "qsi_synchronize": (_S, [_P]),
    "qsi_bta_assemble": (_S, [_P, Shape, ctypes.POINTER(BTA), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.POINTER(BTA)]),
    "qsi_bta_factor": (_S, [_P, Shape, ctypes.POINTER(BTA), ctypes.POINTER(BTA), ctypes.c_int, ctypes.POINTER(_P)]),
    "qsi_bta_selinv": (_S, [_P, _P, ctypes.POINTER(BTA)]),
    "qsi_bta_selquad": (_S, [_P, _P, ctypes.POINTER(BTA), ctypes.POINTER(BTA)]),
    "qsi_bta_factor_multi": (_S, [_P, Shape, ctypes.POINTER(BTA), ctypes.c_int, ctypes.POINTER(BTA), ctypes.c_int,
                                  ctypes.POINTER(_P)]),
    "qsi_bta_selquad_multi": (_S, [_P, _P, ctypes.POINTER(BTA), ctypes.c_int, ctypes.POINTER(BTA)]),
    "qsi_bta_solve": (_S, [_P, Shape, ctypes.POINTER(BTA), ctypes.c_int, ctypes.POINTER(BTA), ctypes.c_int,
                           ctypes.POINTER(BTA), ctypes.POINTER(BTA)]),
    "qsi_bta_solve_partitioned": (_S, [_P, Shape, ctypes.POINTER(BTA), ctypes.c_int, ctypes.POINTER(BTA), ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(BTA), ctypes.POINTER(BTA)]),
    "qsi_bta_solve_varsize": (_S, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                   ctypes.POINTER(BTA), ctypes.c_int, ctypes.POINTER(BTA), ctypes.c_int,
                                   ctypes.POINTER(BTA), ctypes.POINTER(BTA)]),
    "qsi_partition_plan": (ctypes.c_int64, [Shape, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Move),
                                            ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "qsi_factor_destroy": (_S, [_P]),
    "qsi_factor_bytes": (ctypes.c_size_t, [Shape, ctypes.c_int, ctypes.c_int]),
    "qsi_bta_selquad_batched": (_S, [_P, Shape, ctypes.POINTER(BTA), ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(BTA), ctypes.c_int,
                                     ctypes.POINTER(BTA), ctypes.POINTER(BTA)]),
    "qsi_block_inverse_noalloc": (_S, [_P, _P, ctypes.c_int32, _P, _P]),
    "qsi_zgemm": (_S, [_P, ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P,
                       ctypes.c_int64, ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                       ctypes.c_double, _P, ctypes.c_int64]),
    "qsi_request_bytes": (ctypes.c_size_t, [Shape, ctypes.c_int, ctypes.c_int]),
    "qsi_serve_create": (_S, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_size_t]),
    "qsi_serve_submit": (_S, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "qsi_serve_poll": (_S, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Result)]),
    "qsi_serve_destroy": (_S, [_P]),
    "qsi_stats_reset": (_S, [_P, ctypes.c_int]),
    "qsi_stats_read": (_S, [_P, ctypes.POINTER(Stats)]),
    "qsi_stats_timeline": (ctypes.c_int64, [_P, _P, _P, _P, _P, ctypes.c_int64]),
    "qsi_bta_selquad_host": (_S, [_P, Shape, ctypes.POINTER(BTA), ctypes.POINTER(BTA), ctypes.c_int,
                                  ctypes.POINTER(BTA), ctypes.POINTER(BTA)]),
}
for _name, (_res, _args) in _sig.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class QsiError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"qsi status {status}: {message}")
        self.status = status


def exported_symbols():
    return list(_sig)


def shape_of(m: dict) -> tuple[int, int, int]:
    """(n_blocks, b, a) of a single BTA container (the last three axes of diag, tip)."""
    n, b = int(m["diag"].shape[-3]), int(m["diag"].shape[-2])
    return n, b, int(m["tip"].shape[-1])


def _ptr(x) -> int | None:
    if hasattr(x, "data_ptr"):
        return x.data_ptr() if x.numel() else None
    return x.ctypes.data if x.size else None


def _bta(m: dict) -> BTA:
    """C struct of a BTA container; an output's "upper" / "lower" may be None
    (diagonal-only outputs)."""
    for k in KEYS:
        x = m[k]
        if x is None:
            if k not in ("upper", "lower"):
                raise ValueError(f"block array {k} is None")
            continue
        ok = x.is_contiguous() if hasattr(x, "is_contiguous") else x.flags["C_CONTIGUOUS"]
        if not ok:
            raise ValueError(f"block array {k} must be contiguous")
        if str(x.dtype) not in ("torch.complex128", "complex128"):
            raise ValueError(f"block array {k} must be complex128, got {x.dtype}")
    return BTA(*[_ptr(m[k]) if m[k] is not None else None for k in KEYS])


def factor_bytes(n: int, b: int, a: int, with_b: bool = True, precision: int = FP64) -> int:
    return int(_lib.qsi_factor_bytes(Shape(n, b, a), int(with_b), precision))


def device_zeros(n: int, b: int, a: int, device="cuda", off_diagonal: bool = True):
    """Zeroed device BTA container; off_diagonal=False leaves upper / lower None
    (a diagonal-only output)."""
    import torch

    shapes = {"diag": (n, b, b), "upper": (n - 1, b, b), "lower": (n - 1, b, b),
              "arrow_r": (n, b, a), "arrow_b": (n, a, b), "tip": (a, a)}
    return {k: (None if (not off_diagonal and k in ("upper", "lower")) else
                torch.zeros(s, dtype=torch.complex128, device=device)) for k, s in shapes.items()}


def batched_zeros(count: int, n: int, b: int, a: int, device="cuda", off_diagonal: bool = True):
    import torch

    shapes = {"diag": (n, b, b), "upper": (n - 1, b, b), "lower": (n - 1, b, b),
              "arrow_r": (n, b, a), "arrow_b": (n, a, b), "tip": (a, a)}
    return {k: (None if (not off_diagonal and k in ("upper", "lower")) else
                torch.zeros((count, *s), dtype=torch.complex128, device=device)) for k, s in shapes.items()}


def to_device(m: dict, device="cuda"):
    import torch

    return {k: torch.from_numpy(np.ascontiguousarray(m[k])).to(device) for k in KEYS}


def flat_zeros(sizes, a: int, device="cuda", off_diagonal: bool = True):
    """Zeroed device container of a non-uniform BTA matrix: one 1-D complex128
    tensor per key, blocks packed one after the other (qsi_bta_solve_varsize)."""
    import torch

    n = len(sizes)
    elems = {"diag": sum(s * s for s in sizes), "upper": sum(sizes[i] * sizes[i + 1] for i in range(n - 1)),
             "lower": sum(sizes[i] * sizes[i + 1] for i in range(n - 1)), "arrow_r": sum(sizes) * a,
             "arrow_b": sum(sizes) * a, "tip": a * a}
    return {k: (None if (not off_diagonal and k in ("upper", "lower")) else
                torch.zeros(e, dtype=torch.complex128, device=device)) for k, e in elems.items()}


def to_host(m: dict) -> dict:
    return {k: (m[k].cpu().numpy() if m[k] is not None else None) for k in KEYS}


class Factor:
    """Forward-pass result (S_A, S_B per right-hand side, updated arrows, tip) held on the device."""

    def __init__(self, ctx: "Context", handle: int, shape, quad: bool, nrhs: int | None = None):
        self._ctx = ctx
        self.handle = handle
        self.shape = shape
        self.quad = quad
        self.nrhs = (1 if quad else 0) if nrhs is None else nrhs

    def close(self):
        if self.handle:
            _lib.qsi_factor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A libqsi context bound to one device and one CUDA stream (default: torch's
    current stream on that device)."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.device = device
        self.stream = stream
        h = _P()
        st = _lib.qsi_create(ctypes.byref(h), device, _P(stream.cuda_stream))
        if st != OK:
            raise QsiError(st, "qsi_create failed")
        self.handle = h

    def _check(self, st: int):
        if st != OK:
            raise QsiError(st, _lib.qsi_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            _lib.qsi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synchronize(self):
        self._check(_lib.qsi_synchronize(self.handle))

    def batched_config(self) -> dict:
        """Points per wave and tensor-core launch knobs of the last batched call."""
        w, v, t = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        f = ctypes.c_double()
        self._check(_lib.qsi_batched_config(self.handle, ctypes.byref(w), ctypes.byref(v), ctypes.byref(f),
                                            ctypes.byref(t)))
        return {"wave": w.value, "crt_v": v.value, "cta_fill": f.value, "tuned": bool(t.value)}

    def set_flags(self, flags: int):
        """Context flags (qsi_set_flags): ASSUME_ANTIHERMITIAN_B, TWISTED_SPLIT (``solve`` and
        ``selquad_host`` through the twisted two-way split for n_blocks >= 3), or both."""
        self._check(_lib.qsi_set_flags(self.handle, int(flags)))

    def selftest_wait_timeout(self, limit_us: int):
        """Queue one bounded device wait that runs out (see qsi_selftest_wait_timeout)."""
        self._check(_lib.qsi_selftest_wait_timeout(self.handle, int(limit_us)))

    def stats_reset(self, time_kernels: bool = False):
        self._check(_lib.qsi_stats_reset(self.handle, int(time_kernels)))

    def stats_timeline(self) -> dict:
        """qsi_stats_timeline: per timed launch (after stats_reset(True)) its kernel
        family, stream index and start / end in ms."""
        n = int(_lib.qsi_stats_timeline(self.handle, None, None, None, None, 0))
        if n < 0:
            raise QsiError(ERR_CUDA, "qsi_stats_timeline failed")
        kind, strm = np.zeros(n, np.int32), np.zeros(n, np.int32)
        t0, t1 = np.zeros(n), np.zeros(n)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        got = int(_lib.qsi_stats_timeline(self.handle, p(kind), p(strm), p(t0), p(t1), n))
        if got < 0:
            raise QsiError(ERR_CUDA, "qsi_stats_timeline failed")
        return {"kind": kind, "stream": strm, "start_ms": t0, "end_ms": t1}

    def stats(self) -> dict:
        st = Stats()
        self._check(_lib.qsi_stats_read(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def zgemm(self, A, B, C, opA: int = 0, opB: int = 0, alpha: float = 1.0, beta: complex = 0.0,
              precision: int = FP64):
        """C <- alpha op(A) op(B) + beta C on device complex128 matrices (row-major)."""
        M = C.shape[0]
        N = C.shape[1]
        K = A.shape[1] if opA == 0 else A.shape[0]
        ptr = lambda t: _P(t.data_ptr()) if t.numel() else None
        self._check(_lib.qsi_zgemm(self.handle, precision, M, N, K, opA, ptr(A), A.stride(0), opB, ptr(B),
                                   B.stride(0), alpha, complex(beta).real, complex(beta).imag, ptr(C), C.stride(0)))
        return C

    def assemble(self, H: dict, energy: float, eta: float, gamma: float, out: dict | None = None) -> dict:
        n, b, a = shape_of(H)
        if out is None:
            out = device_zeros(n, b, a, H["diag"].device)
        self._check(_lib.qsi_bta_assemble(self.handle, Shape(n, b, a), ctypes.byref(_bta(H)), energy, eta, gamma,
                                          ctypes.byref(_bta(out))))
        return out

    def factor(self, A: dict, B: dict | None = None, precision: int = FP64) -> Factor:
        n, b, a = shape_of(A)
        h = _P()
        bb = ctypes.byref(_bta(B)) if B is not None else None
        self._check(_lib.qsi_bta_factor(self.handle, Shape(n, b, a), ctypes.byref(_bta(A)), bb, precision,
                                        ctypes.byref(h)))
        return Factor(self, h, (n, b, a), B is not None)

    def factor_multi(self, A: dict, Bs: list, precision: int = FP64) -> Factor:
        """Forward pass with several right-hand sides B_r (qsi_bta_factor_multi)."""
        n, b, a = shape_of(A)
        h = _P()
        arr = (BTA * max(1, len(Bs)))(*[_bta(Bk) for Bk in Bs])
        self._check(_lib.qsi_bta_factor_multi(self.handle, Shape(n, b, a), ctypes.byref(_bta(A)), len(Bs),
                                              arr if Bs else None, precision, ctypes.byref(h)))
        return Factor(self, h, (n, b, a), len(Bs) > 0, len(Bs))

    def selquad_multi(self, f: Factor, GR: dict | None = None, GX: list | None = None) -> tuple[dict, list]:
        """G^R and G_r = A^-1 B_r A^-H for every right-hand side of f (qsi_bta_selquad_multi)."""
        dev = f"cuda:{self.device}"
        if GR is None:
            GR = device_zeros(*f.shape, device=dev)
        if GX is None:
            GX = [device_zeros(*f.shape, device=dev) for _ in range(f.nrhs)]
        arr = (BTA * max(1, len(GX)))(*[_bta(G) for G in GX])
        self._check(_lib.qsi_bta_selquad_multi(self.handle, f.handle, ctypes.byref(_bta(GR)), len(GX), arr))
        return GR, GX

    def solve(self, A: dict, Bs: list, GR: dict | None = None, GX: list | None = None,
              precision: int = FP64) -> tuple[dict, list]:
        """The whole solve in one call (qsi_bta_solve): G^R and G_r = A^-1 B_r A^-H for every B_r;
        graph-cached on a non-default stream when the same buffers repeat."""
        n, b, a = shape_of(A)
        dev = f"cuda:{self.device}"
        if GR is None:
            GR = device_zeros(n, b, a, device=dev)
        if GX is None:
            GX = [device_zeros(n, b, a, device=dev) for _ in Bs]
        barr = (BTA * max(1, len(Bs)))(*[_bta(Bk) for Bk in Bs])
        garr = (BTA * max(1, len(GX)))(*[_bta(G) for G in GX])
        self._check(_lib.qsi_bta_solve(self.handle, Shape(n, b, a), ctypes.byref(_bta(A)), len(Bs),
                                       barr if Bs else None, precision, ctypes.byref(_bta(GR)),
                                       garr if GX else None))
        return GR, GX

    def solve_partitioned(self, A: dict, Bs: list, partitions: int, GR: dict | None = None,
                          GX: list | None = None, precision: int = FP64) -> tuple[dict, list]:
        """qsi_bta_solve_partitioned: the solve of ``solve`` with the chain cut into
        ``partitions`` partitions eliminated concurrently plus a reduced system.
        ``partitions = 2`` (and ``0``) is the twisted split (the top half eliminated
        from block 0 down, the bottom half from block n-1 up: the plain sweep's
        accuracy); ``partitions = -1`` takes round(sqrt(n)) general partitions
        while the device estimate of their pivots' conditioning allows
        (1e-13 kappa_F^2 <= 1e-10), else the twisted split (``stats()``:
        partition_kappa, partition_fallbacks)."""
        n, b, a = shape_of(A)
        dev = f"cuda:{self.device}"
        if GR is None:
            GR = device_zeros(n, b, a, device=dev)
        if GX is None:
            GX = [device_zeros(n, b, a, device=dev) for _ in Bs]
        barr = (BTA * max(1, len(Bs)))(*[_bta(Bk) for Bk in Bs])
        garr = (BTA * max(1, len(GX)))(*[_bta(G) for G in GX])
        self._check(_lib.qsi_bta_solve_partitioned(self.handle, Shape(n, b, a), ctypes.byref(_bta(A)), len(Bs),
                                                   barr if Bs else None, partitions, precision,
                                                   ctypes.byref(_bta(GR)), garr if GX else None))
        return GR, GX

    def solve_varsize(self, sizes, A: dict, Bs: list, GR: dict | None = None, GX: list | None = None,
                      precision: int = FP64) -> tuple[dict, list]:
        """qsi_bta_solve_varsize: non-uniform blocks (block i of size sizes[i]).
        A, B_r, GR, GX are packed device containers (``flat_zeros`` layout:
        one 1-D complex128 tensor per key, blocks one after the other)."""
        n = len(sizes)
        a = int(round(A["tip"].numel() ** 0.5))
        dev = f"cuda:{self.device}"
        if GR is None:
            GR = flat_zeros(sizes, a, device=dev)
        if GX is None:
            GX = [flat_zeros(sizes, a, device=dev) for _ in Bs]
        bs = (ctypes.c_int32 * n)(*[int(x) for x in sizes])
        barr = (BTA * max(1, len(Bs)))(*[_bta(Bk) for Bk in Bs])
        garr = (BTA * max(1, len(GX)))(*[_bta(G) for G in GX])
        self._check(_lib.qsi_bta_solve_varsize(self.handle, n, bs, a, ctypes.byref(_bta(A)), len(Bs),
                                               barr if Bs else None, precision, ctypes.byref(_bta(GR)),
                                               garr if GX else None))
        return GR, GX

    def selinv(self, f: Factor, GR: dict | None = None) -> dict:
        if GR is None:
            GR = device_zeros(*f.shape, device=f"cuda:{self.device}")
        self._check(_lib.qsi_bta_selinv(self.handle, f.handle, ctypes.byref(_bta(GR))))
        return GR

    def selquad(self, f: Factor, GR: dict | None = None, GL: dict | None = None) -> tuple[dict, dict]:
        if GR is None:
            GR = device_zeros(*f.shape, device=f"cuda:{self.device}")
        if GL is None:
            GL = device_zeros(*f.shape, device=f"cuda:{self.device}")
        self._check(_lib.qsi_bta_selquad(self.handle, f.handle, ctypes.byref(_bta(GR)), ctypes.byref(_bta(GL))))
        return GR, GL

    def selquad_batched(self, H: dict, energies, eta: float, gammas, B: dict, GR: dict | None = None,
                        GL: dict | None = None, precision: int = FP64):
        """Fused SI+SQ at every energy of ``energies`` for A_k = (E_k + i eta)I - H - Sigma_k.
        B, GR, GL are point-major device BTA containers (leading dimension n_E on every
        block array, e.g. GR["diag"] has shape (n_E, n, b, b))."""
        n, b, a = shape_of(H)
        e = np.ascontiguousarray(energies, dtype=np.float64)
        g = np.ascontiguousarray(gammas, dtype=np.float64)
        nE = int(e.shape[0])
        if g.shape[0] != nE:
            raise ValueError("energies and gammas differ in length")
        if GR is None:
            GR = batched_zeros(nE, n, b, a, device=f"cuda:{self.device}")
        if GL is None:
            GL = batched_zeros(nE, n, b, a, device=f"cuda:{self.device}")
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(_lib.qsi_bta_selquad_batched(self.handle, Shape(n, b, a), ctypes.byref(_bta(H)), nE,
                                                 e.ctypes.data_as(dp), eta, g.ctypes.data_as(dp),
                                                 ctypes.byref(_bta(B)), precision, ctypes.byref(_bta(GR)),
                                                 ctypes.byref(_bta(GL))))
        return GR, GL

    def selquad_host(self, A: dict, B: dict | None, GR: dict, GL: dict | None, precision: int = FP64):
        """End-to-end solve from host buffers (numpy arrays or pinned CPU tensors);
        results are written into GR / GL (host) and the call synchronises."""
        n, b, a = shape_of(A)
        bb = ctypes.byref(_bta(B)) if B is not None else None
        gl = ctypes.byref(_bta(GL)) if GL is not None else None
        self._check(_lib.qsi_bta_selquad_host(self.handle, Shape(n, b, a), ctypes.byref(_bta(A)), bb, precision,
                                              ctypes.byref(_bta(GR)), gl))
        return GR, GL


def partition_plan(n: int, b: int, a: int, partitions: int, n_rhs: int = 1, diag_only: bool = False):
    """The block moves of the partitioned solve (qsi_partition_plan; host only).
    Returns (moves: list of Move, sizes: int64[PLAN_ARRAYS], phase_end: 4 ints,
    meta: (P, m, arrow width, reduced blocks, diag stride, arrow stride)), or
    None for an invalid shape or partition count."""
    sizes = (ctypes.c_int64 * PLAN_ARRAYS)()
    pe = (ctypes.c_int64 * 4)()
    meta = (ctypes.c_int64 * 6)()
    cnt = _lib.qsi_partition_plan(Shape(n, b, a), n_rhs, partitions, int(diag_only), None, 0, sizes, pe, meta)
    if cnt < 0:
        return None
    moves = (Move * max(1, cnt))()
    _lib.qsi_partition_plan(Shape(n, b, a), n_rhs, partitions, int(diag_only), moves, cnt, sizes, pe, meta)
    return list(moves)[:cnt], np.array(sizes[:], dtype=np.int64), list(pe), tuple(meta)


def solve(A: dict, B: dict | None = None, precision: int = FP64, ctx: Context | None = None):
    """Convenience: fused SI+SQ (or SI if B is None) of device BTA matrices."""
    ctx = ctx or Context(A["diag"].device.index or 0)
    f = ctx.factor(A, B, precision)
    try:
        if B is None:
            return ctx.selinv(f), None
        return ctx.selquad(f)
    finally:
        f.close()


class Server:
    """Continuous-batching request server (qsi_serve_*).  Requests are dicts of
    device BTA containers; the containers must stay alive until the request is
    reported done (the server keeps references for that)."""

    def __init__(self, device: int = 0, slots: int = 4, hbm_budget: int = 0):
        h = _P()
        st = _lib.qsi_serve_create(ctypes.byref(h), device, slots, hbm_budget)
        if st != OK:
            raise QsiError(st, "qsi_serve_create failed")
        self.handle = h
        self._keep = {}

    def submit(self, A: dict, B: dict | None, GR: dict, GL: dict | None, precision: int = FP64) -> int:
        """Queue one solve.  The server's streams do not wait for the caller's,
        so the caller's current stream is synchronised first: the inputs (and
        any initialisation of the outputs) are complete on the device before
        the server can start the request."""
        import torch

        torch.cuda.current_stream().synchronize()
        n, b, a = shape_of(A)
        structs = [_bta(A), _bta(B) if B is not None else None, _bta(GR), _bta(GL) if GL is not None else None]
        req = Request(Shape(n, b, a), precision, ctypes.pointer(structs[0]),
                      ctypes.pointer(structs[1]) if structs[1] is not None else None,
                      ctypes.pointer(structs[2]), ctypes.pointer(structs[3]) if structs[3] is not None else None)
        t = ctypes.c_uint64()
        st = _lib.qsi_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t))
        if st != OK:
            raise QsiError(st, "qsi_serve_submit failed")
        self._keep[t.value] = (A, B, GR, GL, structs, req)
        return t.value

    def poll(self, ticket: int):
        """None while running, else a dict with status, slot, queue_ms, latency_ms and the
        request's device interval (device_start_ms, device_end_ms)."""
        done = ctypes.c_int()
        res = Result()
        st = _lib.qsi_serve_poll(self.handle, ticket, ctypes.byref(done), ctypes.byref(res))
        if st != OK:
            raise QsiError(st, "qsi_serve_poll failed")
        if not done.value:
            return None
        self._keep.pop(ticket, None)
        return {"status": res.status, "slot": res.slot, "queue_ms": res.queue_ms, "latency_ms": res.latency_ms,
                "device_start_ms": res.device_start_ms, "device_end_ms": res.device_end_ms}

    def close(self):
        if getattr(self, "handle", None):
            _lib.qsi_serve_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune_cache_store(path: str, n: int, b: int, a: int, precision: int, n_E: int, wave: int, crt_v: int,
                         cta_fill: float, ms_per_point: float) -> None:
    st = _lib.qsi_autotune_cache_store(path.encode(), n, b, a, precision, n_E, wave, crt_v, cta_fill, ms_per_point)
    if st != OK:
        raise QsiError(st, "qsi_autotune_cache_store failed")


def autotune_cache_lookup(path: str, n: int, b: int, a: int, precision: int, n_E: int):
    """(wave, crt_v, cta_fill) of the last matching line of the cache file, or None."""
    w, v, fnd = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    f = ctypes.c_double()
    st = _lib.qsi_autotune_cache_lookup(path.encode(), n, b, a, precision, n_E, ctypes.byref(w), ctypes.byref(v),
                                        ctypes.byref(f), ctypes.byref(fnd))
    if st != OK:
        raise QsiError(st, "qsi_autotune_cache_lookup failed")
    return (w.value, v.value, f.value) if fnd.value else None


def request_bytes(n: int, b: int, a: int, with_b: bool = True, precision: int = FP64) -> int:
    return int(_lib.qsi_request_bytes(Shape(n, b, a), int(with_b), precision))
