"""Python binding of libmemsynth (argument marshalling only).

The module-level functions carry the C ABI's names and arguments
(include/libmemsynth.h); every step of the computation runs in the CUDA
library.  Device buffers are torch CUDA tensors; the context is bound to the
torch stream current at creation.  Loading fails loudly when the library is
missing: there is no CPU path.

`Context` wraps one mem_ctx; `MemOperator` exposes the forward operator to
torch.autograd with the hand-written adjoint as its backward.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

PREC_FP64_DIRECT = 0
PREC_FP32_DIRECT = 1
PREC_BF16X3 = 2
PREC_FP16X3 = 3
PRECISIONS = {"fp64_direct": PREC_FP64_DIRECT, "fp32_direct": PREC_FP32_DIRECT, "bf16x3": PREC_BF16X3,
              "fp16x3": PREC_FP16X3}
IMAGES_PER_CHANNEL = 0
IMAGE_SHARED = 1

STATUS = {0: "MEM_OK", 1: "MEM_EINVAL", 2: "MEM_ENOMEM", 3: "MEM_ECUDA", 4: "MEM_ETIMEOUT",
          5: "MEM_ENUMERIC", 6: "MEM_ENOTSUP"}


class MemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class mem_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("n_channels", ctypes.c_int32), ("vis_offsets", ctypes.POINTER(ctypes.c_int64)),
                ("lambda_", ctypes.c_double), ("G", ctypes.c_double), ("precision", ctypes.c_int32),
                ("image_mode", ctypes.c_int32), ("spin_limit", ctypes.c_uint64)]


FWD_KERNELS = {"stream": 0, "resident": 1}


class mem_tiling_t(ctypes.Structure):
    _fields_ = [("fwd_kernel", ctypes.c_int32), ("fwd_cols", ctypes.c_int32),
                ("fwd_stages", ctypes.c_int32), ("adj_stages", ctypes.c_int32)]

    def as_tuple(self):
        kern = {v: k for k, v in FWD_KERNELS.items()}[self.fwd_kernel]
        return (kern, self.fwd_cols, self.fwd_stages, self.adj_stages)


def _tiling(kernel, cols, fwd_stages, adj_stages):
    return mem_tiling_t(FWD_KERNELS[kernel], int(cols), int(fwd_stages), int(adj_stages))


class mem_solve_report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("evaluations", ctypes.c_int32),
                ("status", ctypes.c_int32), ("stopped_early", ctypes.c_int32),
                ("phi", ctypes.c_double), ("chi2", ctypes.c_double), ("entropy", ctypes.c_double)]


_LIB = None
EXPORTS = ["mem_create", "mem_destroy", "mem_last_error", "mem_status_string", "mem_set_precision",
           "mem_num_vis", "mem_num_images", "mem_forward", "mem_adjoint", "mem_objective_grad",
           "mem_objective_grad_host", "mem_scalars_dev", "mem_solve", "mem_sync", "mem_launch_count",
           "mem_profile", "mem_profile_read", "mem_adjoint_noalloc", "mem_use_graphs", "mem_autotune",
           "mem_set_tiling", "mem_tiling", "mem_forward_gridded",
           "mem_dirty_image", "mem_residual_image", "mem_beam_fit", "mem_phase_rotate"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libmemsynth.so (building it first when allowed); raises if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"libmemsynth is not built ({path}); run python -m paper_1703_02920_gb300.build")
        _build.build()
    lib = ctypes.CDLL(path)
    P, D, I32, I64, V = ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    DP = ctypes.POINTER(ctypes.c_double)
    lib.mem_create.argtypes = [ctypes.POINTER(mem_config), P, P, P, P, P, V, ctypes.POINTER(ctypes.c_void_p)]
    lib.mem_create.restype = ctypes.c_int
    lib.mem_destroy.argtypes = [P]
    lib.mem_destroy.restype = None
    lib.mem_last_error.argtypes = [P]
    lib.mem_last_error.restype = ctypes.c_char_p
    lib.mem_status_string.argtypes = [ctypes.c_int]
    lib.mem_status_string.restype = ctypes.c_char_p
    lib.mem_set_precision.argtypes = [P, I32]
    lib.mem_set_precision.restype = ctypes.c_int
    lib.mem_num_vis.argtypes = [P]
    lib.mem_num_vis.restype = I64
    lib.mem_num_images.argtypes = [P]
    lib.mem_num_images.restype = I32
    lib.mem_forward.argtypes = [P, P, P]
    lib.mem_forward.restype = ctypes.c_int
    lib.mem_adjoint.argtypes = [P, P, P]
    lib.mem_adjoint.restype = ctypes.c_int
    lib.mem_objective_grad.argtypes = [P, P, P, I32, DP]
    lib.mem_objective_grad.restype = ctypes.c_int
    lib.mem_objective_grad_host.argtypes = [P, P, P, I32, DP]
    lib.mem_objective_grad_host.restype = ctypes.c_int
    lib.mem_scalars_dev.argtypes = [P]
    lib.mem_scalars_dev.restype = ctypes.c_void_p
    lib.mem_solve.argtypes = [P, P, I32, ctypes.POINTER(mem_solve_report), DP]
    lib.mem_solve.restype = ctypes.c_int
    lib.mem_sync.argtypes = [P]
    lib.mem_sync.restype = ctypes.c_int
    lib.mem_launch_count.argtypes = [P]
    lib.mem_launch_count.restype = I64
    lib.mem_profile.argtypes = [P, I32]
    lib.mem_profile.restype = ctypes.c_int
    lib.mem_profile_read.argtypes = [P, I32, ctypes.c_char_p, DP, ctypes.POINTER(ctypes.c_int64)]
    lib.mem_profile_read.restype = I32
    lib.mem_autotune.argtypes = [P, P, I32, ctypes.POINTER(mem_tiling_t)]
    lib.mem_autotune.restype = ctypes.c_int
    lib.mem_set_tiling.argtypes = [P, ctypes.POINTER(mem_tiling_t)]
    lib.mem_set_tiling.restype = ctypes.c_int
    lib.mem_tiling.argtypes = [P, ctypes.POINTER(mem_tiling_t)]
    lib.mem_tiling.restype = ctypes.c_int
    lib.mem_forward_gridded.argtypes = [P, P, I32, P]
    lib.mem_forward_gridded.restype = ctypes.c_int
    lib.mem_dirty_image.argtypes = [P, I32, P]
    lib.mem_dirty_image.restype = ctypes.c_int
    lib.mem_residual_image.argtypes = [P, P, P]
    lib.mem_residual_image.restype = ctypes.c_int
    lib.mem_beam_fit.argtypes = [P, I32, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.mem_beam_fit.restype = ctypes.c_int
    lib.mem_phase_rotate.argtypes = [ctypes.c_int64, P, P, ctypes.c_double, ctypes.c_double, P]
    lib.mem_phase_rotate.restype = ctypes.c_int
    lib.mem_use_graphs.argtypes = [P, I32]
    lib.mem_use_graphs.restype = ctypes.c_int
    lib.mem_adjoint_noalloc.argtypes = [I32, D, D, I64, P, P, P, P, P, V]
    lib.mem_adjoint_noalloc.restype = ctypes.c_int
    _LIB = lib
    return lib


def _check(status: int, ctx=None):
    if status != 0:
        msg = load().mem_last_error(ctx).decode(errors="replace")
        raise MemError(status, msg)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# the C ABI, one function per entry point
# ---------------------------------------------------------------------------
def mem_create(n, dx, dy, vis_offsets, lam, G, precision, image_mode, u, v, vis_obs, sigma, pb,
               stream=None, spin_limit: int = 0) -> int:
    """Create a context; host numpy inputs; returns the opaque handle (int)."""
    lib = load()
    offs = np.ascontiguousarray(vis_offsets, dtype=np.int64)
    cfg = mem_config(n=int(n), dx=float(dx), dy=float(dy), n_channels=len(offs) - 1,
                     vis_offsets=offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                     lambda_=float(lam), G=float(G), precision=int(precision),
                     image_mode=int(image_mode), spin_limit=int(spin_limit))
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    vo = np.asarray(vis_obs)
    if np.iscomplexobj(vo):
        vi = np.empty(2 * vo.size)
        vi[0::2], vi[1::2] = vo.real, vo.imag
    else:
        vi = np.ascontiguousarray(vo, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    beam = np.ascontiguousarray(pb, dtype=np.float32)
    handle = ctypes.c_void_p()
    st = ctypes.c_void_p(0 if stream is None else int(stream))
    _check(lib.mem_create(ctypes.byref(cfg), _np_ptr(u), _np_ptr(v), _np_ptr(vi), _np_ptr(sg),
                          _np_ptr(beam), st, ctypes.byref(handle)))
    return handle.value


def mem_destroy(ctx):
    load().mem_destroy(ctx)


def mem_set_precision(ctx, precision):
    _check(load().mem_set_precision(ctx, int(precision)), ctx)


def mem_forward(ctx, image_dev, vis_dev):
    _check(load().mem_forward(ctx, _ptr(image_dev), _ptr(vis_dev)), ctx)


def mem_adjoint(ctx, y_dev, img_dev):
    _check(load().mem_adjoint(ctx, _ptr(y_dev), _ptr(img_dev)), ctx)


def mem_objective_grad(ctx, image_dev, grad_dev, projected=0, want_scalars=True):
    out = (ctypes.c_double * 3)()
    _check(load().mem_objective_grad(ctx, _ptr(image_dev), _ptr(grad_dev), int(projected),
                                     out if want_scalars else None), ctx)
    return tuple(out) if want_scalars else None


def mem_objective_grad_host(ctx, image_host: np.ndarray, grad_host: np.ndarray | None, projected=0):
    out = (ctypes.c_double * 3)()
    _check(load().mem_objective_grad_host(ctx, _np_ptr(image_host),
                                          None if grad_host is None else _np_ptr(grad_host),
                                          int(projected), out), ctx)
    return tuple(out)


def mem_solve(ctx, image_dev, n_iter, n_images):
    rep = mem_solve_report()
    hist = np.zeros((n_images, n_iter + 1, 6))
    _check(load().mem_solve(ctx, _ptr(image_dev), int(n_iter), ctypes.byref(rep),
                            hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)
    return rep, hist


def mem_sync(ctx):
    _check(load().mem_sync(ctx), ctx)


def mem_launch_count(ctx) -> int:
    return int(load().mem_launch_count(ctx))


def mem_adjoint_noalloc(n, dx, dy, u_dev, v_dev, y_dev, pb_dev, img_dev, stream=None):
    """Allocation-free adjoint (see the C header): every argument a device tensor."""
    nv = 0 if u_dev is None else int(u_dev.numel())
    st = ctypes.c_void_p(0 if stream is None else int(stream))
    _check(load().mem_adjoint_noalloc(int(n), float(dx), float(dy), nv, _ptr(u_dev), _ptr(v_dev),
                                      _ptr(y_dev), _ptr(pb_dev), _ptr(img_dev), st))


def mem_autotune(ctx, image_dev, reps: int = 3):
    """Pick the tensor-core tiling on this context's data; returns
    (forward kernel, column block, forward stages, adjoint stages)."""
    out = mem_tiling_t()
    _check(load().mem_autotune(ctx, _ptr(image_dev), int(reps), ctypes.byref(out)), ctx)
    return out.as_tuple()


def mem_set_tiling(ctx, kernel: str, cols: int, fwd_stages: int, adj_stages: int):
    t = _tiling(kernel, cols, fwd_stages, adj_stages)
    _check(load().mem_set_tiling(ctx, ctypes.byref(t)), ctx)


def mem_tiling(ctx):
    out = mem_tiling_t()
    _check(load().mem_tiling(ctx, ctypes.byref(out)), ctx)
    return out.as_tuple()


def mem_forward_gridded(ctx, image_dev, pad, vis_dev):
    """The paper's gridded (FFT + bilinear) approximation of the forward."""
    _check(load().mem_forward_gridded(ctx, _ptr(image_dev), int(pad), _ptr(vis_dev)), ctx)


def mem_dirty_image(ctx, psf: bool, out_dev):
    _check(load().mem_dirty_image(ctx, int(bool(psf)), _ptr(out_dev)), ctx)


def mem_residual_image(ctx, image_dev, out_dev):
    _check(load().mem_residual_image(ctx, _ptr(image_dev), _ptr(out_dev)), ctx)


def mem_beam_fit(psf, dx: float, dy: float):
    """(BMAJ, BMIN, BPA, beam area in pixels) of a host PSF image (n x n float32)."""
    import numpy as np
    a = np.ascontiguousarray(psf, dtype=np.float32)
    out = (ctypes.c_double * 4)()
    _check(load().mem_beam_fit(a.ctypes.data, int(a.shape[0]), float(dx), float(dy), out), None)
    return tuple(out)


def mem_phase_rotate(u, v, vis, x_p: float, y_p: float):
    """Visibilities (complex array) rotated from a pointing's phase centre
    (x_p, y_p) to the image's: returns a new complex128 array."""
    import numpy as np
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    buf = np.ascontiguousarray(np.stack([np.real(vis), np.imag(vis)], 1), dtype=np.float64)
    _check(load().mem_phase_rotate(u.size, u.ctypes.data, v.ctypes.data, float(x_p), float(y_p), buf.ctypes.data), None)
    return buf[:, 0] + 1j * buf[:, 1]


def mem_use_graphs(ctx, enable: bool):
    _check(load().mem_use_graphs(ctx, int(bool(enable))), ctx)


def mem_profile(ctx, enable: bool):
    _check(load().mem_profile(ctx, int(bool(enable))), ctx)


def mem_profile_read(ctx, max_kernels: int = 32):
    """{kernel name: (total ms, launches)} since the last read."""
    names = ctypes.create_string_buffer(32 * max_kernels)
    ms = (ctypes.c_double * max_kernels)()
    cnt = (ctypes.c_int64 * max_kernels)()
    n = load().mem_profile_read(ctx, max_kernels, names, ms, cnt)
    if n < 0:
        raise MemError(3, "profile read failed")
    raw = names.raw
    out = {}
    for i in range(n):
        nm = raw[32 * i:32 * i + 32].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[i]), int(cnt[i]))
    return out


# ---------------------------------------------------------------------------
# convenience wrapper over torch tensors
# ---------------------------------------------------------------------------
class Context:
    """One libmemsynth context over a data set (synth.Dataset or equivalent)."""

    def __init__(self, ds, precision="bf16x3", lam=None, G=None, shared_image=None, stream=None,
                 spin_limit: int = 0):
        import torch
        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("libmemsynth needs a CUDA GPU (sm_103a); no CPU path exists")
        self.N = int(ds.N)
        self.shared = bool(ds.shared_image if shared_image is None else shared_image)
        self.offsets = np.asarray(ds.offsets, dtype=np.int64)
        self.C = len(self.offsets) - 1
        self.n_images = 1 if self.shared else self.C
        self.Z = int(self.offsets[-1])
        self.G = float(ds.G if G is None else G)
        self.lam = float(ds.lam if lam is None else lam)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self.handle = mem_create(self.N, ds.dx, ds.dy, self.offsets, self.lam, self.G, self.precision,
                                 IMAGE_SHARED if self.shared else IMAGES_PER_CHANNEL, ds.u, ds.v, ds.vo,
                                 ds.sigma, ds.pb, stream=self.stream.cuda_stream, spin_limit=spin_limit)

    def close(self):
        if self.handle:
            mem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def image_shape(self):
        return (self.n_images, self.N, self.N)

    def set_precision(self, precision):
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        mem_set_precision(self.handle, p)
        self.precision = p

    def _img(self, image):
        t = self.torch.as_tensor(image, dtype=self.torch.float32, device="cuda")
        return t.reshape(self.image_shape()).contiguous()

    def forward(self, image):
        """Model visibilities, float32 tensor (Z, 2)."""
        img = self._img(image)
        out = self.torch.empty((self.Z, 2), dtype=self.torch.float32, device="cuda")
        mem_forward(self.handle, img, out)
        return out

    def forward_gridded(self, image, pad: int = 2):
        """The paper's gridded approximation of the model visibilities, (Z, 2)."""
        img = self._img(image)
        out = self.torch.empty((self.Z, 2), dtype=self.torch.float32, device="cuda")
        mem_forward_gridded(self.handle, img, pad, out)
        return out

    def dirty_image(self, psf: bool = False):
        """Natural-weights dirty image (or PSF) per channel, (C, N, N) float32."""
        out = self.torch.empty((self.C, self.N, self.N), dtype=self.torch.float32, device="cuda")
        mem_dirty_image(self.handle, psf, out)
        return out

    def residual_image(self, image):
        """Natural-weights dirty image of V° - V(image) per channel, (C, N, N) float32."""
        out = self.torch.empty((self.C, self.N, self.N), dtype=self.torch.float32, device="cuda")
        mem_residual_image(self.handle, self._img(image), out)
        return out

    def adjoint(self, y):
        yt = self.torch.as_tensor(y, dtype=self.torch.float32, device="cuda").reshape(self.Z, 2).contiguous()
        out = self.torch.empty(self.image_shape(), dtype=self.torch.float32, device="cuda")
        mem_adjoint(self.handle, yt, out)
        return out

    def objective_grad(self, image, projected=False, want_grad=True):
        img = self._img(image)
        g = self.torch.empty_like(img) if want_grad else None
        phi, chi, S = mem_objective_grad(self.handle, img, g, int(projected))
        return phi, chi, S, g

    def objective_grad_host(self, image: np.ndarray, projected=False):
        img = np.ascontiguousarray(image, dtype=np.float32).reshape(self.image_shape())
        g = np.empty_like(img)
        phi, chi, S = mem_objective_grad_host(self.handle, img, g, int(projected))
        return phi, chi, S, g

    def solve(self, image, n_iter):
        img = self._img(image).clone()
        rep, hist = mem_solve(self.handle, img, n_iter, self.n_images)
        return img, rep, hist

    def sync(self):
        mem_sync(self.handle)

    def launches(self) -> int:
        return mem_launch_count(self.handle)

    def autotune(self, image, reps: int = 3):
        return mem_autotune(self.handle, self._img(image), reps)

    def set_tiling(self, kernel: str, cols: int, fwd_stages: int, adj_stages: int):
        mem_set_tiling(self.handle, kernel, cols, fwd_stages, adj_stages)

    def tiling(self):
        return mem_tiling(self.handle)

    def profile(self, enable: bool = True):
        mem_profile(self.handle, enable)

    def profile_read(self):
        return mem_profile_read(self.handle)


def _autograd():
    import torch

    class MemOperator(torch.autograd.Function):
        """V = F(A I) with backward grad_I = A Re(F^H grad_V) (the adjoint kernel).

        `MemOperator.apply(image, ctx)` with image (n_images, N, N) float32 on
        the GPU returns (Z, 2) float32 visibilities (re, im)."""

        @staticmethod
        def forward(fctx, image, op: Context):
            fctx.op = op
            return op.forward(image)

        @staticmethod
        def backward(fctx, grad_v):
            return fctx.op.adjoint(grad_v.contiguous()), None

    return MemOperator


_MEMOP = None


def MemOperator():
    global _MEMOP
    if _MEMOP is None:
        _MEMOP = _autograd()
    return _MEMOP
