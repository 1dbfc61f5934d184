"""Thin Python binding of the C ABI in ``include/mreg.h`` (ctypes).

Only argument marshalling lives here: every step of the registration runs in
the CUDA library ``lib/libmreg.so``.  There is no CPU fallback: if the
library is missing or fails to load, :func:`load` raises.

Host arrays are numpy arrays; device arrays are torch CUDA tensors (torch is
used for device memory and streams only).  ``stream`` arguments accept a
``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or ``None`` (torch's
current stream when torch is imported and CUDA is initialised, else the
legacy default stream).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmreg.so")

# mreg_status
MREG_OK = 0
MREG_ERR_INVALID_ARG = 1
MREG_ERR_BAD_MESH = 2
MREG_ERR_SIZE_MISMATCH = 3
MREG_ERR_NONFINITE = 4
MREG_ERR_CUDA = 5
MREG_ERR_OOM = 6
MREG_ERR_NOT_CONVERGED = 7
MREG_ERR_DEVICE_CHECK = 8
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "BAD_MESH", 3: "SIZE_MISMATCH", 4: "NONFINITE",
                5: "CUDA", 6: "OOM", 7: "NOT_CONVERGED", 8: "DEVICE_CHECK"}

MREG_MODE_EXPLICIT = 0
MREG_MODE_UMBRELLA_IMPLICIT = 1
MREG_MODE_FEM_IMPLICIT = 2
MREG_GRAD_MESH = 0
MREG_GRAD_SPLINE = 1
MREG_QUAD_NODES = 0
MREG_QUAD_EDGE_MIDPOINTS = 1

MREG_FIELD_U = 0
MREG_FIELD_FORCE = 1
MREG_FIELD_TE_NODES = 2
MREG_FIELD_RE_NODES = 3
MREG_FIELD_COEF_RE = 4
MREG_FIELD_COEF_TE = 5
MREG_FIELD_PIXEL_TRI = 6
MREG_FIELD_ENERGY = 7
MREG_FIELD_PCG_ITERS = 8
MREG_FIELD_PCG_RESID = 9
MREG_FIELD_COEF_TE_16 = 10
MREG_FIELD_U_PREV = 11

MODES = {"S0": MREG_MODE_EXPLICIT, "S1": MREG_MODE_UMBRELLA_IMPLICIT, "S2": MREG_MODE_FEM_IMPLICIT}
GRADS = {"G0": MREG_GRAD_MESH, "G1": MREG_GRAD_SPLINE}
QUADS = {"Q0": MREG_QUAD_NODES, "Q1": MREG_QUAD_EDGE_MIDPOINTS}
MREG_ENGINE_AUTO = 0
MREG_ENGINE_GRID = 1
ENGINES = {"auto": MREG_ENGINE_AUTO, "grid": MREG_ENGINE_GRID}
MREG_COEFF_FP32 = 0
MREG_COEFF_BF16 = 1
MREG_COEFF_FP16 = 2
COEFFS = {"fp32": MREG_COEFF_FP32, "bf16": MREG_COEFF_BF16, "fp16": MREG_COEFF_FP16}
MREG_SOLVER_AUTO = 0
MREG_SOLVER_CG = 1
MREG_SOLVER_CHEBYSHEV = 2
SOLVERS = {"auto": MREG_SOLVER_AUTO, "cg": MREG_SOLVER_CG, "chebyshev": MREG_SOLVER_CHEBYSHEV}


class mreg_mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_tris", C.c_int32),
                ("xy", C.POINTER(C.c_float)), ("tri", C.POINTER(C.c_int32))]


class mreg_image(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("row_stride", C.c_int64),
                ("data", C.c_void_p), ("on_device", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class mreg_options(C.Structure):
    _fields_ = [("mode", C.c_int32), ("grad", C.c_int32), ("quad", C.c_int32),
                ("pcg_maxit", C.c_int32), ("lambda_", C.c_double), ("pcg_rtol", C.c_double),
                ("block_size", C.c_int32), ("grid_blocks", C.c_int32), ("engine", C.c_int32),
                ("coeff_storage", C.c_int32), ("team_ctas", C.c_int32),
                ("smooth_passes", C.c_int32), ("host_topology", C.c_int32),
                ("team_blocks_per_sm", C.c_int32), ("node_lanes", C.c_int32),
                ("solver", C.c_int32), ("neighbour_sync", C.c_int32),
                ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p)]


class mreg_stats_t(C.Structure):
    _fields_ = [("iterations_done", C.c_int32), ("last_pcg_iters", C.c_int32),
                ("max_pcg_iters", C.c_int32), ("not_converged", C.c_int32),
                ("last_rel_resid", C.c_double), ("last_energy", C.c_double),
                ("grid_blocks", C.c_int32), ("block_size", C.c_int32),
                ("device_status", C.c_int32), ("engine", C.c_int32),
                ("node_lanes", C.c_int32), ("neighbour_sync", C.c_int32)]


EXPORTS = ["mreg_default_options", "mreg_create", "mreg_reset", "mreg_step", "mreg_warp",
           "mreg_msd", "mreg_energy", "mreg_energy_terms", "mreg_get_u", "mreg_set_u",
           "mreg_set_u_prev", "mreg_get_field",
           "mreg_stats", "mreg_destroy", "mreg_last_error", "mreg_version",
           "mreg_prefilter_noalloc", "mreg_warp_energy_grad", "mreg_unroll_grad",
           "mreg_test_barrier_timeout", "mreg_apply_operator", "mreg_batch_apply_operator",
           "mreg_unroll_grad_checkpointed",
           "mreg_batch_create", "mreg_batch_run", "mreg_batch_tune",
           "mreg_batch_shape", "mreg_batch_iterate_ms", "mreg_batch_msd", "mreg_batch_get_field",
           "mreg_batch_stats", "mreg_batch_destroy"]

NOALLOC_MAX_PIXELS = 1024 * 1024

_lib = None


class MregError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


def load(path: str | None = None) -> C.CDLL:
    """Load the CUDA library (once).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1411_2141_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "mreg_default_options": ([C.POINTER(mreg_options)], i32),
        "mreg_create": ([C.POINTER(mreg_mesh), C.POINTER(mreg_image), C.POINTER(mreg_image),
                         dbl, dbl, C.POINTER(mreg_options), vp, C.POINTER(vp)], i32),
        "mreg_reset": ([vp, vp], i32),
        "mreg_step": ([vp, i32, vp], i32),
        "mreg_warp": ([vp, vp, vp, vp], i32),
        "mreg_msd": ([vp, C.POINTER(dbl), vp], i32),
        "mreg_energy": ([vp, C.POINTER(dbl), vp], i32),
        "mreg_energy_terms": ([vp, C.POINTER(dbl), C.POINTER(dbl), vp], i32),
        "mreg_get_u": ([vp, vp, i32, vp], i32),
        "mreg_set_u": ([vp, vp, i32, vp], i32),
        "mreg_set_u_prev": ([vp, vp, i32, i32, vp], i32),
        "mreg_get_field": ([vp, i32, vp, i32, C.POINTER(i64), vp], i32),
        "mreg_stats": ([vp, C.POINTER(mreg_stats_t), vp], i32),
        "mreg_destroy": ([vp], None),
        "mreg_last_error": ([], C.c_char_p),
        "mreg_version": ([], i32),
        "mreg_prefilter_noalloc": ([vp, i64, vp, i32, i32, vp], i32),
        "mreg_warp_energy_grad": ([vp, vp, vp, vp, vp], i32),
        "mreg_unroll_grad": ([vp, vp, i32, vp, vp, vp], i32),
        "mreg_unroll_grad_checkpointed": ([vp, vp, i32, i32, vp, vp, vp], i32),
        "mreg_test_barrier_timeout": ([vp, i32, i32, i64], i32),
        "mreg_apply_operator": ([vp, vp, vp, vp], i32),
        "mreg_batch_apply_operator": ([vp, vp, vp, vp], i32),
        "mreg_batch_create": ([i32, C.POINTER(mreg_mesh), C.POINTER(mreg_image),
                               C.POINTER(mreg_image), dbl, dbl, C.POINTER(mreg_options), vp,
                               C.POINTER(vp)], i32),
        "mreg_batch_run": ([vp, i32, vp], i32),
        "mreg_batch_tune": ([vp, i32, vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                             C.POINTER(C.c_float)], i32),
        "mreg_batch_shape": ([vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                              C.POINTER(i32)], i32),
        "mreg_batch_iterate_ms": ([vp, C.POINTER(C.c_float)], i32),
        "mreg_batch_msd": ([vp, C.POINTER(dbl), vp], i32),
        "mreg_batch_get_field": ([vp, i32, i32, vp, i32, C.POINTER(i64), vp], i32),
        "mreg_batch_stats": ([vp, i32, C.POINTER(mreg_stats_t), vp], i32),
        "mreg_batch_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != MREG_OK:
        raise MregError(st, where, load().mreg_last_error().decode(errors="replace"))


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream or None
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _is_torch_cuda(x) -> bool:
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


def prefilter_noalloc(img, out, stream=None):
    """B-spline coefficients of a device image (2-D float32 CUDA tensor on the
    current device, unit column stride) into ``out`` (contiguous, same shape
    and device) without any device allocation; asynchronous on ``stream``."""
    if not (_is_torch_cuda(img) and _is_torch_cuda(out)):
        raise ValueError("img and out must be CUDA tensors")
    import torch
    dev = torch.cuda.current_device()
    if img.device.index != dev or out.device.index != dev:
        raise ValueError("img and out must be on the current CUDA device")
    if str(img.dtype) != "torch.float32" or img.dim() != 2 or img.stride(1) != 1:
        raise ValueError("img must be a 2-D float32 tensor with unit column stride")
    if tuple(out.shape) != tuple(img.shape) or not out.is_contiguous():
        raise ValueError("out must be contiguous with the image's shape")
    H, W = int(img.shape[0]), int(img.shape[1])
    _check(load().mreg_prefilter_noalloc(img.data_ptr(), int(img.stride(0)), out.data_ptr(), W, H,
                                         _stream_ptr(stream)), "mreg_prefilter_noalloc")
    return out


def default_options() -> mreg_options:
    o = mreg_options()
    _check(load().mreg_default_options(C.byref(o)), "mreg_default_options")
    return o


def make_options(mode="S0", grad="G0", quad="Q0", lam=None, pcg_rtol=None, pcg_maxit=None,
                 block_size=0, grid_blocks=0, engine="auto",
                 coeff_bf16=False, coeff="fp32", team_ctas=0, team_blocks_per_sm=0,
                 smooth_passes=0, host_topology=False, node_lanes=0, solver="auto",
                 neighbour_sync=False, allocator=None) -> mreg_options:
    o = default_options()
    o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    o.grad = GRADS[grad] if isinstance(grad, str) else int(grad)
    o.quad = QUADS[quad] if isinstance(quad, str) else int(quad)
    if lam is not None:
        o.lambda_ = float(lam)
    if pcg_rtol is not None:
        o.pcg_rtol = float(pcg_rtol)
    if pcg_maxit is not None:
        o.pcg_maxit = int(pcg_maxit)
    o.block_size = int(block_size)
    o.grid_blocks = int(grid_blocks)
    o.engine = ENGINES[engine] if isinstance(engine, str) else int(engine)
    # coeff: storage of Te's coefficients ("fp32", "bf16", "fp16");
    # coeff_bf16=True is the same as coeff="bf16"
    o.coeff_storage = MREG_COEFF_BF16 if coeff_bf16 else (COEFFS[coeff] if isinstance(coeff, str)
                                                          else int(coeff))
    o.team_ctas = int(team_ctas)
    o.team_blocks_per_sm = int(team_blocks_per_sm)
    o.node_lanes = int(node_lanes)
    o.solver = SOLVERS[solver] if isinstance(solver, str) else int(solver)
    o.neighbour_sync = int(bool(neighbour_sync)) if isinstance(neighbour_sync, bool) \
        else int(neighbour_sync)
    o.smooth_passes = int(smooth_passes)
    o.host_topology = int(bool(host_topology))
    if allocator is not None:
        o.alloc = allocator.alloc_fn
        o.free = allocator.free_fn
    return o


class TorchAllocator:
    """Device memory for handles from PyTorch's caching allocator (pass as
    ``allocator=`` to Registration or Batch).  Keep the object alive as long
    as the handles that use it; the wrappers below hold a reference."""

    def __init__(self):
        import torch

        def _alloc(nbytes, stream, ctx):
            try:
                s = torch.cuda.ExternalStream(stream) if stream else None
                return torch.cuda.caching_allocator_alloc(int(nbytes), stream=s)
            except Exception:   # reported to the library as an allocation failure
                return None

        def _free(ptr, stream, ctx):
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass
        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)


def _image(img, keep: list) -> mreg_image:
    im = mreg_image()
    if _is_torch_cuda(img):
        if str(img.dtype) != "torch.float32" or img.dim() != 2 or img.stride(1) != 1:
            raise ValueError("device images must be 2-D float32 tensors with unit column stride")
        im.height, im.width = int(img.shape[0]), int(img.shape[1])
        im.row_stride = int(img.stride(0))
        im.data = img.data_ptr()
        im.on_device = 1
        keep.append(img)
    else:
        a = np.ascontiguousarray(img, dtype=np.float32)
        if a.ndim != 2:
            raise ValueError("images must be 2-D")
        im.height, im.width = a.shape
        im.row_stride = a.shape[1]
        im.data = a.ctypes.data
        im.on_device = 0
        keep.append(a)
    return im


class Registration:
    """One registration problem on the current CUDA device (wraps a handle)."""

    def __init__(self, V, T, Re, Te, alpha: float, tau: float, options: mreg_options | None = None,
                 stream=None, **kw):
        lib = load()
        if options is None:
            options = make_options(**kw)
        self._allocator = kw.get("allocator")   # callbacks must outlive the handle
        keep: list = []
        Vh = np.ascontiguousarray(V, dtype=np.float32)
        Th = np.ascontiguousarray(T, dtype=np.int32)
        if Vh.ndim != 2 or Vh.shape[1] != 2 or Th.ndim != 2 or Th.shape[1] != 3:
            raise ValueError("V must be (n, 2) and T (m, 3)")
        mesh = mreg_mesh(Vh.shape[0], Th.shape[0], Vh.ctypes.data_as(C.POINTER(C.c_float)),
                         Th.ctypes.data_as(C.POINTER(C.c_int32)))
        re = _image(Re, keep)
        te = _image(Te, keep)
        h = C.c_void_p()
        self._h = None
        _check(lib.mreg_create(C.byref(mesh), C.byref(re), C.byref(te), float(alpha), float(tau),
                               C.byref(options), _stream_ptr(stream), C.byref(h)), "mreg_create")
        self._h = h
        self.n_nodes = int(Vh.shape[0])
        self.n_tris = int(Th.shape[0])
        self.height, self.width = int(re.height), int(re.width)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and _lib is not None:
            _lib.mreg_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def reset(self, stream=None):
        _check(load().mreg_reset(self._h, _stream_ptr(stream)), "mreg_reset")

    def step(self, n_iters: int, stream=None):
        _check(load().mreg_step(self._h, int(n_iters), _stream_ptr(stream)), "mreg_step")

    def apply_operator(self, x, y, stream=None):
        """y = A x with the semi-implicit system matrix (asynchronous); x, y:
        contiguous (n_nodes, 2) float32 device tensors."""
        for t in (x, y):
            if not _is_torch_cuda(t) or str(t.dtype) != "torch.float32" or not t.is_contiguous() \
                    or tuple(t.shape) != (self.n_nodes, 2):
                raise ValueError("x and y must be contiguous (n_nodes, 2) float32 device tensors")
        _check(load().mreg_apply_operator(self._h, x.data_ptr(), y.data_ptr(), _stream_ptr(stream)),
               "mreg_apply_operator")
        return y

    def test_barrier_timeout(self, block: int, barrier: int, timeout_ns: int):
        """Arm the next iteration launch to run out of one grid-barrier wait
        (a test of the failure path; see mreg_test_barrier_timeout)."""
        _check(load().mreg_test_barrier_timeout(self._h, int(block), int(barrier),
                                                int(timeout_ns)), "mreg_test_barrier_timeout")

    def warp(self, out=None, msd_out=None, stream=None):
        """Asynchronous warp into device tensors ``out`` (H x W float32) and
        ``msd_out`` (1 float64), either may be None."""
        po = out.data_ptr() if out is not None else None
        pm = msd_out.data_ptr() if msd_out is not None else None
        _check(load().mreg_warp(self._h, po, pm, _stream_ptr(stream)), "mreg_warp")

    def warp_energy_grad(self, u, energy=None, grad=None, stream=None):
        """Asynchronous E(u) into ``energy`` (1 float64 device tensor) and
        dE/du into ``grad`` (n x 2 float32 device tensor); either may be None.
        ``u``: n x 2 float32 contiguous device tensor."""
        if not _is_torch_cuda(u) or str(u.dtype) != "torch.float32" or not u.is_contiguous() \
                or tuple(u.shape) != (self.n_nodes, 2):
            raise ValueError("u must be a contiguous (n_nodes, 2) float32 device tensor")
        pe = energy.data_ptr() if energy is not None else None
        pg = grad.data_ptr() if grad is not None else None
        _check(load().mreg_warp_energy_grad(self._h, u.data_ptr(), pe, pg, _stream_ptr(stream)),
               "mreg_warp_energy_grad")

    def unroll_grad(self, u0, n_iters: int, energy=None, grad=None, stream=None,
                    checkpoint_every: int = 0):
        """Asynchronous E(u_K) after n_iters iterations from ``u0`` into
        ``energy`` and dE(u_K)/du0 into ``grad`` (device tensors, either may
        be None); explicit mode with the spline gradient only.  The handle's
        iterate is left at u_K.  checkpoint_every > 0 keeps only every
        c-th state and recomputes the segments (bitwise the same result)."""
        if not _is_torch_cuda(u0) or str(u0.dtype) != "torch.float32" or not u0.is_contiguous() \
                or tuple(u0.shape) != (self.n_nodes, 2):
            raise ValueError("u0 must be a contiguous (n_nodes, 2) float32 device tensor")
        pe = energy.data_ptr() if energy is not None else None
        pg = grad.data_ptr() if grad is not None else None
        _check(load().mreg_unroll_grad_checkpointed(self._h, u0.data_ptr(), int(n_iters),
                                                    int(checkpoint_every), pe, pg,
                                                    _stream_ptr(stream)),
               "mreg_unroll_grad_checkpointed")

    def msd(self, stream=None) -> float:
        v = C.c_double()
        _check(load().mreg_msd(self._h, C.byref(v), _stream_ptr(stream)), "mreg_msd")
        return v.value

    def energy(self, stream=None) -> float:
        """E = D + alpha S (Eq. 1) at the current u."""
        v = C.c_double()
        _check(load().mreg_energy(self._h, C.byref(v), _stream_ptr(stream)), "mreg_energy")
        return v.value

    def energy_terms(self, stream=None):
        """(D, S) at the current u: the data term and the regulariser."""
        d, sm = C.c_double(), C.c_double()
        _check(load().mreg_energy_terms(self._h, C.byref(d), C.byref(sm), _stream_ptr(stream)),
               "mreg_energy_terms")
        return d.value, sm.value

    def get_u(self, out=None, stream=None) -> np.ndarray:
        if out is not None and _is_torch_cuda(out):
            _check(load().mreg_get_u(self._h, out.data_ptr(), 1, _stream_ptr(stream)), "mreg_get_u")
            return out
        u = np.empty((self.n_nodes, 2), np.float32)
        _check(load().mreg_get_u(self._h, u.ctypes.data, 0, _stream_ptr(stream)), "mreg_get_u")
        return u

    def set_u(self, u, stream=None):
        if _is_torch_cuda(u):
            _check(load().mreg_set_u(self._h, u.data_ptr(), 1, _stream_ptr(stream)), "mreg_set_u")
            return
        a = np.ascontiguousarray(u, dtype=np.float32)
        if a.shape != (self.n_nodes, 2):
            raise ValueError("u must be (n_nodes, 2)")
        _check(load().mreg_set_u(self._h, a.ctypes.data, 0, _stream_ptr(stream)), "mreg_set_u")

    def set_u_prev(self, u_prev, stream=None):
        """The iterates before u for the Chebyshev solve's extrapolated guess,
        (n_prev, n_nodes, 2) newest first as get_field(MREG_FIELD_U_PREV)
        returns them (None or n_prev = 0 drops them); call after set_u."""
        if u_prev is None or u_prev.shape[0] == 0:
            _check(load().mreg_set_u_prev(self._h, None, 0, 0, _stream_ptr(stream)),
                   "mreg_set_u_prev")
            return
        if tuple(u_prev.shape[1:]) != (self.n_nodes, 2):
            raise ValueError("u_prev must be (n_prev, n_nodes, 2)")
        n_prev = int(u_prev.shape[0])
        if _is_torch_cuda(u_prev):
            if not u_prev.is_contiguous():
                raise ValueError("u_prev must be contiguous")
            _check(load().mreg_set_u_prev(self._h, u_prev.data_ptr(), n_prev, 1,
                                          _stream_ptr(stream)), "mreg_set_u_prev")
            return
        a = np.ascontiguousarray(u_prev, dtype=np.float32)
        _check(load().mreg_set_u_prev(self._h, a.ctypes.data, n_prev, 0, _stream_ptr(stream)),
               "mreg_set_u_prev")

    def get_field(self, field: int, stream=None) -> np.ndarray:
        lib = load()
        n = C.c_int64()
        _check(lib.mreg_get_field(self._h, field, None, 0, C.byref(n), _stream_ptr(stream)),
               "mreg_get_field")
        dtype = {MREG_FIELD_PIXEL_TRI: np.int32, MREG_FIELD_PCG_ITERS: np.int32,
                 MREG_FIELD_ENERGY: np.float64, MREG_FIELD_PCG_RESID: np.float64,
                 MREG_FIELD_COEF_TE_16: np.uint16}.get(field, np.float32)
        out = np.empty(n.value, dtype)
        if n.value:
            _check(lib.mreg_get_field(self._h, field, out.ctypes.data, 0, None, _stream_ptr(stream)),
                   "mreg_get_field")
        if field in (MREG_FIELD_U, MREG_FIELD_FORCE):
            out = out.reshape(-1, 2)
        elif field == MREG_FIELD_U_PREV:
            out = out.reshape(-1, self.n_nodes, 2)
        elif field in (MREG_FIELD_COEF_RE, MREG_FIELD_COEF_TE, MREG_FIELD_PIXEL_TRI) or (
                field == MREG_FIELD_COEF_TE_16 and n.value):
            out = out.reshape(self.height, self.width)
        return out

    def stats(self, stream=None, check: bool = True) -> dict:
        s = mreg_stats_t()
        st = load().mreg_stats(self._h, C.byref(s), _stream_ptr(stream))
        if check:
            _check(st, "mreg_stats")
        d = {k: getattr(s, k) for k, _ in mreg_stats_t._fields_}
        d["status"] = st
        return d


_FIELD_DTYPES = {MREG_FIELD_PIXEL_TRI: np.int32, MREG_FIELD_PCG_ITERS: np.int32,
                 MREG_FIELD_ENERGY: np.float64, MREG_FIELD_PCG_RESID: np.float64,
                 MREG_FIELD_COEF_TE_16: np.uint16}


class Batch:
    """Many registration problems registered together (the batched engine).

    ``pairs`` is a sequence of ``(V, T, Re, Te)``; every pair shares
    ``alpha``, ``tau`` and the options."""

    def __init__(self, pairs, alpha: float, tau: float, options: mreg_options | None = None,
                 stream=None, **kw):
        lib = load()
        if options is None:
            options = make_options(**kw)
        self._allocator = kw.get("allocator")   # callbacks must outlive the batch
        pairs = list(pairs)
        n = len(pairs)
        if n < 1:
            raise ValueError("need at least one pair")
        keep: list = []
        meshes = (mreg_mesh * n)()
        res = (mreg_image * n)()
        tes = (mreg_image * n)()
        self.n_nodes, self.shapes = [], []
        for k, (V, T, Re, Te) in enumerate(pairs):
            Vh = np.ascontiguousarray(V, dtype=np.float32)
            Th = np.ascontiguousarray(T, dtype=np.int32)
            if Vh.ndim != 2 or Vh.shape[1] != 2 or Th.ndim != 2 or Th.shape[1] != 3:
                raise ValueError(f"pair {k}: V must be (n, 2) and T (m, 3)")
            keep += [Vh, Th]
            meshes[k] = mreg_mesh(Vh.shape[0], Th.shape[0],
                                  Vh.ctypes.data_as(C.POINTER(C.c_float)),
                                  Th.ctypes.data_as(C.POINTER(C.c_int32)))
            res[k] = _image(Re, keep)
            tes[k] = _image(Te, keep)
            self.n_nodes.append(int(Vh.shape[0]))
            self.shapes.append((int(res[k].height), int(res[k].width)))
        h = C.c_void_p()
        self._h = None
        _check(lib.mreg_batch_create(n, meshes, res, tes, float(alpha), float(tau),
                                     C.byref(options), _stream_ptr(stream), C.byref(h)),
               "mreg_batch_create")
        self._h = h
        self.n_pairs = n

    def close(self):
        if self._h is not None and _lib is not None:
            _lib.mreg_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, n_iters: int, stream=None):
        _check(load().mreg_batch_run(self._h, int(n_iters), _stream_ptr(stream)), "mreg_batch_run")

    def apply_operator(self, x, y, stream=None):
        """y = A x for every pair (asynchronous); x, y: contiguous
        (sum of n_nodes, 2) float32 device tensors packed in pair order."""
        n = sum(self.n_nodes)
        for t in (x, y):
            if not _is_torch_cuda(t) or str(t.dtype) != "torch.float32" or not t.is_contiguous() \
                    or tuple(t.shape) != (n, 2):
                raise ValueError("x and y must be contiguous (total nodes, 2) float32 device tensors")
        _check(load().mreg_batch_apply_operator(self._h, x.data_ptr(), y.data_ptr(),
                                                _stream_ptr(stream)), "mreg_batch_apply_operator")
        return y

    def tune(self, n_iters: int, stream=None):
        """Autotune the team shape; returns ((team_ctas, block_size,
        blocks_per_sm), times) with times[(ctas, block, per_sm)] in ms (None
        where the shape is skipped)."""
        c, k, m = C.c_int32(), C.c_int32(), C.c_int32()
        t = (C.c_float * 30)()
        _check(load().mreg_batch_tune(self._h, int(n_iters), _stream_ptr(stream), C.byref(c),
                                      C.byref(k), C.byref(m), t), "mreg_batch_tune")
        times = {}
        for i, ctas in enumerate((1, 2, 4, 8, 16)):
            for j, blk in enumerate((128, 256, 512)):
                for q, per_sm in enumerate((1, 2)):
                    v = float(t[(i * 3 + j) * 2 + q])
                    times[(ctas, blk, per_sm)] = v if v >= 0 else None
        return (c.value, k.value, m.value), times

    def shape(self):
        """(team_ctas, block_size, blocks_per_sm, n_teams)."""
        c, k, m, n = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().mreg_batch_shape(self._h, C.byref(c), C.byref(k), C.byref(m), C.byref(n)),
               "mreg_batch_shape")
        return c.value, k.value, m.value, n.value

    def iterate_ms(self) -> float:
        """Device time of the iteration kernel in the last run (ms)."""
        v = C.c_float()
        _check(load().mreg_batch_iterate_ms(self._h, C.byref(v)), "mreg_batch_iterate_ms")
        return v.value

    def msd(self, stream=None) -> np.ndarray:
        out = np.empty(self.n_pairs, np.float64)
        _check(load().mreg_batch_msd(self._h, out.ctypes.data_as(C.POINTER(C.c_double)),
                                     _stream_ptr(stream)), "mreg_batch_msd")
        return out

    def get_field(self, pair: int, field: int, stream=None) -> np.ndarray:
        lib = load()
        n = C.c_int64()
        _check(lib.mreg_batch_get_field(self._h, int(pair), field, None, 0, C.byref(n),
                                        _stream_ptr(stream)), "mreg_batch_get_field")
        out = np.empty(n.value, _FIELD_DTYPES.get(field, np.float32))
        if n.value:
            _check(lib.mreg_batch_get_field(self._h, int(pair), field, out.ctypes.data, 0, None,
                                            _stream_ptr(stream)), "mreg_batch_get_field")
        if field in (MREG_FIELD_U, MREG_FIELD_FORCE):
            out = out.reshape(-1, 2)
        elif field in (MREG_FIELD_COEF_RE, MREG_FIELD_COEF_TE, MREG_FIELD_PIXEL_TRI) or (
                field == MREG_FIELD_COEF_TE_16 and n.value):
            out = out.reshape(self.shapes[pair])
        return out

    def get_u(self, pair: int, stream=None) -> np.ndarray:
        return self.get_field(pair, MREG_FIELD_U, stream)

    def stats(self, pair: int, stream=None, check: bool = True) -> dict:
        s = mreg_stats_t()
        st = load().mreg_batch_stats(self._h, int(pair), C.byref(s), _stream_ptr(stream))
        if check:
            _check(st, "mreg_batch_stats")
        d = {k: getattr(s, k) for k, _ in mreg_stats_t._fields_}
        d["status"] = st
        return d
