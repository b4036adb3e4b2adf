"""ctypes binding of libfbst.so (include/fbst.h): argument marshalling only.

Every step of the transform runs in the CUDA library. This module converts Python arguments to
the C structs, passes device pointers (torch tensors' data_ptr or plain integers) and the CUDA
stream through, and turns status codes into exceptions. There is no CPU or PyTorch fallback: if
the library is missing, importing the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfbst.so")

FBST_OK = 0
STATUS_NAMES = {0: "FBST_OK", -1: "FBST_ERR_INVALID", -2: "FBST_ERR_OOM", -3: "FBST_ERR_CUDA",
                -4: "FBST_ERR_UNSUPPORTED", -5: "FBST_ERR_TIMEOUT", -6: "FBST_ERR_NUMERIC"}
ULA, URA = 0, 1
STAGE2 = {"auto": 0, "gs": 1, "gs_ir1": 2, "dense_fp32": 3, "dense_bf16x3": 4, "dense_tf32": 5,
          "dense_tf32x3": 6, "dense_f16x3": 7}
STAGE2_NAMES = {v: k for k, v in STAGE2.items()}
GENERATOR_SOLVER = {"levinson": 0, "superfast": 1}


class FBSTError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        msg = f"{what} failed: {STATUS_NAMES.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class Geometry(C.Structure):
    _fields_ = [("kind", C.c_int), ("mx", C.c_int), ("my", C.c_int), ("bx", C.c_int), ("by", C.c_int)]


class Band(C.Structure):
    _fields_ = [("frac_bw", C.c_double), ("epsilon", C.c_double), ("gamma_num", C.c_int),
                ("gamma_den", C.c_int), ("delta", C.c_double), ("delta_relative", C.c_int),
                ("stage2", C.c_int), ("max_blocks", C.c_int), ("generator_solver", C.c_int)]


class Info(C.Structure):
    _fields_ = [("M", C.c_int), ("N", C.c_int), ("B", C.c_int), ("L", C.c_int),
                ("P_time", C.c_int), ("S_time", C.c_int), ("P_space_x", C.c_int), ("P_space_y", C.c_int),
                ("P_gs", C.c_int), ("P_rec", C.c_int), ("S_rec", C.c_int), ("stage2", C.c_int),
                ("delta", C.c_double), ("eps_num", C.c_int64), ("eps_den", C.c_int64),
                ("fb_num", C.c_int64), ("fb_den", C.c_int64), ("rho", C.c_double),
                ("snapshot_bound", C.c_double), ("gamma_bound", C.c_double),
                ("warn_snapshots", C.c_int), ("warn_gamma", C.c_int),
                ("table_bytes", C.c_size_t), ("workspace_bytes", C.c_size_t)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


# Every symbol include/fbst.h declares, with its ctypes signature.
_VP, _I = C.c_void_p, C.c_int
SIGNATURES = {
    "fbst_derive": (_I, [C.POINTER(Geometry), _I, _I, _I, C.POINTER(Band), C.POINTER(Info)]),
    "fbst_plan": (_I, [C.POINTER(_VP), C.POINTER(Geometry), _I, _I, _I, C.POINTER(Band), _VP, _VP, _VP, _VP]),
    "fbst_plan_positions": (_I, [C.POINTER(_VP), C.POINTER(Geometry), C.POINTER(C.c_double), _I, _I, _I,
                                 C.POINTER(Band), _VP, _VP, _VP, _VP]),
    "fbst_execute": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_execute_host": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_execute_noalloc": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_czt": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_czt_time": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_czt_space": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_toeplitz_apply": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_plan_info": (_I, [_VP, C.POINTER(Info)]),
    "fbst_sync_status": (_I, [_VP, _VP]),
    "fbst_plan_generators": (_I, [_VP, _VP]),
    "fbst_solve_generators": (_I, [_VP, _I, _VP, _VP]),
    "fbst_trace_stages": (_I, [_VP, _I]),
    "fbst_trace_read": (_I, [_VP, C.POINTER(C.c_float), _I]),
    "fbst_destroy": (_I, [_VP]),
    "fbst_status_string": (C.c_char_p, [_I]),
    "fbst_last_error": (C.c_char_p, []),
    "fbst_launch_count": (_I, [_VP, _I]),
    "fbst_batch_create": (_I, [C.POINTER(_VP), C.POINTER(_VP), _I]),
    "fbst_batch_execute": (_I, [_VP, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_I), _VP]),
    "fbst_batch_enqueue": (_I, [_VP, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_I), _VP]),
    "fbst_batch_launch_count": (_I, [_VP]),
    "fbst_batch_destroy": (_I, [_VP]),
    "fbst_autotune": (_I, [_VP, _I, _VP, C.POINTER(_I)]),
    "fbst_set_shapes": (_I, [_VP, _I, _I, _I, _I]),
    "fbst_get_shapes": (_I, [_VP, C.POINTER(_I)]),
    "fbst_null_create": (_I, [C.POINTER(_VP), _VP, C.POINTER(_I), _I, _I, _VP]),
    "fbst_null_create_directions": (_I, [C.POINTER(_VP), _VP, C.POINTER(C.c_double), _I, _I, _I, _VP]),
    "fbst_null_create_time": (_I, [C.POINTER(_VP), _VP, C.POINTER(_I), _I, _I, _VP]),
    "fbst_null_apply_time": (_I, [_VP, _VP, _VP, _VP, _I, _VP]),
    "fbst_null_apply": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_null_execute": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_null_launch_count": (_I, [_VP, _I]),
    "fbst_null_destroy": (_I, [_VP]),
    "fbst_fp32_fma_peak": (_I, [_VP, _I, C.POINTER(C.c_double), C.POINTER(C.c_double), _VP]),
    "fbst_set_wait_limit": (_I, [_VP, C.c_uint64]),
    "fbst_execute_stream": (_I, [_VP, _VP, C.c_longlong, _I, _VP, _I, _VP]),
    "fbst_offgrid_create": (_I, [C.POINTER(_VP), _VP, C.POINTER(C.c_double), _I, _I, _VP]),
    "fbst_offgrid_interpolate": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_offgrid_apply": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_offgrid_execute": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fbst_offgrid_destroy": (_I, [_VP]),
}
NULL_CONTRACTION = {"tf32x3": 0, "fp32": 1}

_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libfbst.so once (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2512_08887_gb300.build` "
                               "(the FBST has no CPU fallback)")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int, what: str) -> None:
    if status != FBST_OK:
        lib = load_library()
        detail = lib.fbst_last_error().decode() if status in (-2, -3) else ""
        raise FBSTError(status, what, detail)


def _ptr(x) -> int:
    """Device/host address of a torch tensor, a numpy array or a plain integer."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def make_geometry(kind: str, mx: int, my: int = 1, bx: int | None = None, by: int | None = None) -> Geometry:
    k = ULA if kind == "ula" else URA
    return Geometry(k, mx, my, mx if bx is None else bx, (my if k == URA else 1) if by is None else by)


def make_band(frac_bw: float, epsilon: float = 1.01, gamma=(2, 1), delta: float = 1e-3,
              delta_relative: bool = True, stage2: str = "auto", max_blocks: int = 64,
              generator_solver: str = "levinson") -> Band:
    return Band(float(frac_bw), float(epsilon), int(gamma[0]), int(gamma[1]), float(delta),
                int(bool(delta_relative)), STAGE2[stage2], int(max_blocks), GENERATOR_SOLVER[generator_solver])


def derive(geom: Geometry, N: int, band: Band) -> Info:
    """Host-only parameter derivation (fbst_derive); raises FBSTError on invalid input."""
    lib = load_library()
    info = Info()
    M, B = geom.mx * geom.my, geom.bx * geom.by
    _check(lib.fbst_derive(C.byref(geom), M, N, B, C.byref(band), C.byref(info)), "fbst_derive")
    return info


def fp32_fma_peak(iters: int = 4096, stream=None) -> tuple:
    """Measured FP32 FMA throughput of the current device (fbst_fp32_fma_peak): (TFLOP/s, ms)."""
    import torch
    lib = load_library()
    sink = torch.zeros(4, dtype=torch.float32, device="cuda")
    tf, ms = C.c_double(), C.c_double()
    _check(lib.fbst_fp32_fma_peak(sink.data_ptr(), int(iters), C.byref(tf), C.byref(ms), _stream(stream)),
           "fbst_fp32_fma_peak")
    return tf.value, ms.value


# fbst_alloc_fn / fbst_free_fn of include/fbst.h.
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator:
    """A device allocator for fbst_plan: `alloc(nbytes, stream) -> address` (0 when it has no
    memory) and `free(address, nbytes, stream)`, Python callables; `stream` is the cudaStream_t as an
    integer. Holds the ctypes callbacks, which must live as long as any plan that uses them."""

    def __init__(self, alloc, free):
        def _alloc(nbytes, stream, ctx):
            try:
                return int(alloc(int(nbytes), int(stream or 0))) or None
            except Exception:                   # an allocator failure is FBST_ERR_OOM, not a crash
                return None

        def _free(ptr, nbytes, stream, ctx):
            try:
                free(int(ptr), int(nbytes), int(stream or 0))
            except Exception:
                pass

        self.c_alloc, self.c_free = ALLOC_FN(_alloc), FREE_FN(_free)

    def pointers(self) -> tuple:
        return C.cast(self.c_alloc, C.c_void_p).value, C.cast(self.c_free, C.c_void_p).value


_torch_allocator = None


def torch_allocator() -> Allocator:
    """PyTorch's caching allocator (torch.cuda.caching_allocator_alloc / _delete), stream-ordered
    on the stream the plan was built on."""
    global _torch_allocator
    if _torch_allocator is None:
        import torch

        def alloc(nbytes, stream):
            return torch.cuda.caching_allocator_alloc(nbytes, stream=stream)

        def free(ptr, nbytes, stream):
            torch.cuda.caching_allocator_delete(ptr)

        _torch_allocator = Allocator(alloc, free)
    return _torch_allocator


class Plan:
    """An FBST plan on the current CUDA device (fbst_plan / fbst_destroy).

    `allocator`: "torch" (default) takes the plan's device memory from PyTorch's caching
    allocator; None lets the library use cudaMallocAsync; or an Allocator. Its memory is allocated
    and freed in stream order on `stream` (default: the current stream), which must outlive the plan.
    `positions` (M (x, y) pairs, half wavelengths): a linear or rectangular array off the grid
    (Sec. IX).
    """

    def __init__(self, geom: Geometry, N: int, band: Band, stream=None, allocator="torch", positions=None):
        self._lib = load_library()
        self.geom, self.band = geom, band
        self.M, self.B, self.N = geom.mx * geom.my, geom.bx * geom.by, N
        if isinstance(allocator, str):
            if allocator != "torch":
                raise ValueError(f"unknown allocator {allocator!r}")
            allocator = torch_allocator()
        self._allocator = allocator                 # keeps the callbacks alive with the plan
        self.nonuniform = positions is not None
        fa, ff = allocator.pointers() if allocator is not None else (None, None)
        h = C.c_void_p()
        if positions is None:
            _check(self._lib.fbst_plan(C.byref(h), C.byref(geom), self.M, N, self.B, C.byref(band),
                                       _stream(stream), fa, ff, None), "fbst_plan")
        else:
            # Element positions (M x 2, half wavelengths; a linear array has y = 0): Sec. IX.
            flat = [float(v) for pair in positions for v in (pair[0], pair[1])]
            if len(flat) != 2 * self.M:
                raise ValueError(f"positions must hold {self.M} (x, y) pairs")
            arr = (C.c_double * len(flat))(*flat)
            _check(self._lib.fbst_plan_positions(C.byref(h), C.byref(geom), arr, self.M, N, self.B, C.byref(band),
                                                 _stream(stream), fa, ff, None), "fbst_plan_positions")
        self._h = h
        self.info = Info()
        _check(self._lib.fbst_plan_info(self._h, C.byref(self.info)), "fbst_plan_info")
        self.L = self.info.L

    @property
    def handle(self) -> int:
        return self._h.value

    def _call(self, name: str, src, dst, nblk: int, stream) -> None:
        _check(getattr(self._lib, name)(self._h, _ptr(src), _ptr(dst), int(nblk), _stream(stream)), name)

    def execute(self, y, bhat, nblk: int, stream=None) -> None:
        """y [nblk][M][N] -> bhat [nblk][B][N], complex64 device buffers."""
        self._call("fbst_execute", y, bhat, nblk, stream)

    def execute_host(self, y, bhat, nblk: int, stream=None) -> None:
        """Same with host buffers (copies inside, synchronises the stream)."""
        self._call("fbst_execute_host", y, bhat, nblk, stream)

    def execute_noalloc(self, y, bhat, nblk: int, stream=None) -> None:
        """Same as execute, intermediates in the library's static device array (no allocation)."""
        self._call("fbst_execute_noalloc", y, bhat, nblk, stream)

    def execute_stream(self, record, T: int, hop: int, out, nblk: int, stream=None) -> None:
        """Continuous record [M][T] -> beam streams [B][nblk*hop] from blocks every `hop` samples,
        each contributing its central hop samples (fbst_execute_stream)."""
        _check(self._lib.fbst_execute_stream(self._h, _ptr(record), int(T), int(hop), _ptr(out), int(nblk),
                                             _stream(stream)), "fbst_execute_stream")

    def czt(self, y, w, nblk: int, stream=None) -> None:
        """Stage 1: y [nblk][M][N] -> w [nblk][B][L]."""
        self._call("fbst_czt", y, w, nblk, stream)

    def czt_time(self, y, yhat, nblk: int, stream=None) -> None:
        """Temporal chirp-z only: y [nblk][M][N] -> yhat [nblk][L][M]."""
        self._call("fbst_czt_time", y, yhat, nblk, stream)

    def czt_space(self, yhat, w, nblk: int, stream=None) -> None:
        """Spatial chirp-z only: yhat [nblk][L][M] -> w [nblk][B][L]."""
        self._call("fbst_czt_space", yhat, w, nblk, stream)

    def toeplitz_apply(self, w, bhat, nblk: int, stream=None) -> None:
        """Stage 2: w [nblk][B][L] -> bhat [nblk][B][N]."""
        self._call("fbst_toeplitz_apply", w, bhat, nblk, stream)

    def set_wait_limit(self, ns: int) -> None:
        """Limit of each pipeline wait of the tensor-core stage 2, ns (0 = default 1 s)."""
        _check(self._lib.fbst_set_wait_limit(self._h, int(ns)), "fbst_set_wait_limit")

    def sync_status(self, stream=None) -> int:
        """Synchronise the stream; return and clear the plan's device status word (0 = OK)."""
        return int(self._lib.fbst_sync_status(self._h, _stream(stream)))

    def launch_count(self, nblk: int) -> int:
        return int(self._lib.fbst_launch_count(self._h, int(nblk)))

    def autotune(self, nblk: int, stream=None) -> tuple:
        """Time every compiled stage-1 launch shape on nblk blocks; keep and return the fastest."""
        out = (C.c_int * 4)()
        _check(self._lib.fbst_autotune(self._h, int(nblk), _stream(stream), out), "fbst_autotune")
        return tuple(out)

    def set_shapes(self, time_E: int, time_G: int, space_E: int, space_G: int) -> None:
        _check(self._lib.fbst_set_shapes(self._h, time_E, time_G, space_E, space_G), "fbst_set_shapes")

    def shapes(self) -> tuple:
        out = (C.c_int * 4)()
        _check(self._lib.fbst_get_shapes(self._h, out), "fbst_get_shapes")
        return tuple(out)

    def generators(self):
        """First column of every A_b^{-1} from the plan's FP64 solve, numpy complex128 [B][L]."""
        import numpy as np
        out = np.empty((self.B, self.L), dtype=np.complex128)
        _check(self._lib.fbst_plan_generators(self._h, out.ctypes.data), "fbst_plan_generators")
        return out

    def trace_stages(self, capacity: int) -> None:
        """Record stage times of the next `capacity` execute calls (0 stops tracing)."""
        _check(self._lib.fbst_trace_stages(self._h, int(capacity)), "fbst_trace_stages")

    def trace_read(self, max_calls: int):
        """Per traced execute call, oldest first: (stage 1a, stage 1b, stage 2) device ms."""
        buf = (C.c_float * (3 * max(1, int(max_calls))))()
        n = self._lib.fbst_trace_read(self._h, buf, int(max_calls))
        if n < 0:
            _check(n, "fbst_trace_read")
        return [tuple(buf[3 * i:3 * i + 3]) for i in range(n)]

    def solve_generators(self, method: str, x, stream=None) -> None:
        """Solve again for every x_b = A_b^{-1} e_0 with `method` ("levinson" or "superfast") into
        x, a complex128 CUDA tensor [B][L], on `stream` (default: torch's current stream)."""
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.complex128
                and x.is_contiguous() and x.numel() == self.B * self.L):
            raise ValueError("x must be a contiguous complex128 CUDA tensor of B*L elements")
        _check(self._lib.fbst_solve_generators(self._h, GENERATOR_SOLVER[method], _ptr(x), _stream(stream)),
               "fbst_solve_generators")

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fbst_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Independent plans run together as grouped launches replayed from a CUDA graph."""

    def __init__(self, plans):
        self._lib = load_library()
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        h = C.c_void_p()
        _check(self._lib.fbst_batch_create(C.byref(h), arr, len(self.plans)), "fbst_batch_create")
        self._h = h

    def execute(self, ys, bhats, nblks, stream=None) -> None:
        n = len(self.plans)
        ya = (C.c_void_p * n)(*[_ptr(v) for v in ys])
        ba = (C.c_void_p * n)(*[_ptr(v) for v in bhats])
        na = (C.c_int * n)(*[int(v) for v in nblks])
        _check(self._lib.fbst_batch_execute(self._h, ya, ba, na, _stream(stream)), "fbst_batch_execute")

    def enqueue(self, ys, bhats, nblks, stream=None) -> None:
        """Grouped launches without graph capture (pointer sets that change every call)."""
        n = len(self.plans)
        ya = (C.c_void_p * n)(*[_ptr(v) for v in ys])
        ba = (C.c_void_p * n)(*[_ptr(v) for v in bhats])
        na = (C.c_int * n)(*[int(v) for v in nblks])
        _check(self._lib.fbst_batch_enqueue(self._h, ya, ba, na, _stream(stream)), "fbst_batch_enqueue")

    def launch_count(self) -> int:
        return int(self._lib.fbst_batch_launch_count(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fbst_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Nulling:
    """Beamspace interference nulling of grid beams `interferers` for `plan` (Eq. (14);
    fbst_null_create / fbst_null_destroy), or its time-domain form (Eq. (15), time_domain=True;
    fbst_null_create_time). The plan must outlive this object. `contraction`: "fp32"
    (CUDA cores, the accurate one: the correction is about ten times the nulled result at 20 dB, so
    its product rounding matters) or "tf32x3" (tensor cores, faster, coarser products)."""

    def __init__(self, plan: Plan, interferers=None, contraction: str = "fp32", stream=None, directions=None,
                 K: int = 8, time_domain: bool = False):
        self._lib = load_library()
        self.plan = plan
        self.time_domain = bool(time_domain)
        h = C.c_void_p()
        if time_domain:
            # The time-domain form of Eq. (15) (grid interferers).
            self.interferers = [int(p) for p in interferers]
            arr = (C.c_int * max(1, len(self.interferers)))(*self.interferers)
            _check(self._lib.fbst_null_create_time(C.byref(h), plan._h, arr, len(self.interferers),
                                                   NULL_CONTRACTION[contraction], _stream(stream)),
                   "fbst_null_create_time")
        elif directions is not None:
            # Off-grid interferers: (u, v) direction cosines, vectors interpolated from K grid beams.
            dirs = [(float(d[0]), float(d[1]) if len(d) > 1 else 0.0) for d in directions]
            self.interferers = dirs
            arr = (C.c_double * (2 * max(1, len(dirs))))(*[x for d in dirs for x in d])
            _check(self._lib.fbst_null_create_directions(C.byref(h), plan._h, arr, len(dirs), int(K),
                                                         NULL_CONTRACTION[contraction], _stream(stream)),
                   "fbst_null_create_directions")
        else:
            self.interferers = [int(p) for p in interferers]
            arr = (C.c_int * max(1, len(self.interferers)))(*self.interferers)
            _check(self._lib.fbst_null_create(C.byref(h), plan._h, arr, len(self.interferers),
                                              NULL_CONTRACTION[contraction], _stream(stream)), "fbst_null_create")
        self._h = h

    def apply(self, w, wt, nblk: int, stream=None) -> None:
        """The bracket of Eq. (14): w [nblk][B][L] -> wt [nblk][B][L] (wt may be w)."""
        _check(self._lib.fbst_null_apply(self._h, _ptr(w), _ptr(wt), int(nblk), _stream(stream)), "fbst_null_apply")

    def execute(self, y, bhat, nblk: int, stream=None) -> None:
        """Nulled transform: y [nblk][M][N] -> bhat [nblk][B][N], complex64 device buffers."""
        _check(self._lib.fbst_null_execute(self._h, _ptr(y), _ptr(bhat), int(nblk), _stream(stream)),
               "fbst_null_execute")

    def apply_time(self, y, y_int, out, nblk: int, stream=None) -> None:
        """Eq. (15) on time-domain beams (time_domain=True): y [nblk][B][N] plain beams, y_int
        [nblk][P][2L] the interferers' beams over the broader interval of 2L samples centred on the
        block -> out [nblk][B][N]."""
        _check(self._lib.fbst_null_apply_time(self._h, _ptr(y), _ptr(y_int), _ptr(out), int(nblk), _stream(stream)),
               "fbst_null_apply_time")

    def launch_count(self, nblk: int) -> int:
        return int(self._lib.fbst_null_launch_count(self._h, int(nblk)))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fbst_null_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class OffGrid:
    """Off-grid beams of `directions` ((u, v) direction cosines) by interpolation of the plan's grid
    beam vectors over K grid beams per axis (Sec. VIII-A; fbst_offgrid_create / _destroy). The plan
    must outlive this object."""

    def __init__(self, plan: Plan, directions, K: int = 8, stream=None):
        self._lib = load_library()
        self.plan = plan
        dirs = [(float(d[0]), float(d[1]) if len(d) > 1 else 0.0) for d in directions]
        self.ndir = len(dirs)
        arr = (C.c_double * (2 * max(1, self.ndir)))(*[x for d in dirs for x in d])
        h = C.c_void_p()
        _check(self._lib.fbst_offgrid_create(C.byref(h), plan._h, arr, self.ndir, int(K), _stream(stream)),
               "fbst_offgrid_create")
        self._h = h

    def _call(self, name, src, dst, nblk, stream):
        _check(getattr(self._lib, name)(self._h, _ptr(src), _ptr(dst), int(nblk), _stream(stream)), name)

    def interpolate(self, w, wstar, nblk: int, stream=None) -> None:
        """w [nblk][B][L] -> interpolated beam vectors [nblk][ndir][L]."""
        self._call("fbst_offgrid_interpolate", w, wstar, nblk, stream)

    def apply(self, w, bstar, nblk: int, stream=None) -> None:
        """w [nblk][B][L] -> off-grid beams [nblk][ndir][N]."""
        self._call("fbst_offgrid_apply", w, bstar, nblk, stream)

    def execute(self, y, bstar, nblk: int, stream=None) -> None:
        """y [nblk][M][N] -> off-grid beams [nblk][ndir][N]."""
        self._call("fbst_offgrid_execute", y, bstar, nblk, stream)

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fbst_offgrid_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
