"""Python binding of libcslsm, the GB300 PnP-ADMM light-sheet reconstruction.

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels of libcslsm.so (built in-tree for sm_103a by ``build.py``).  PyTorch
provides device memory and streams; tensors are passed to the C ABI as raw
device pointers together with the current CUDA stream.

There is no CPU path: importing the package works without a GPU, but every
call that computes raises if the shared library is missing or no CUDA device
is present.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcslsm.so")

TIKHONOV, TV, BM3D, WNNM = 0, 1, 2, 3
DENOISERS = {"tikhonov": TIKHONOV, "tv": TV, "bm3d": BM3D, "wnnm": WNNM}
MAX_R = 32
STORAGE = {"fp32": 0, "bf16": 1, "fp16": 2}
STORAGE_DTYPE = {"fp32": torch.float32, "bf16": torch.bfloat16, "fp16": torch.float16}

STATUS = {0: "CSLSM_OK", 1: "CSLSM_ERR_INVALID_ARG", 2: "CSLSM_ERR_CUDA",
          3: "CSLSM_ERR_TIMEOUT", 4: "CSLSM_ERR_UNSUPPORTED", 5: "CSLSM_ERR_OOM"}


class CslsmError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        self.status = status
        super().__init__(f"{func}: {STATUS.get(status, status)}: {msg}")


class AdmmParams(ctypes.Structure):
    """Mirror of cslsm_admm_params (include/cslsm.h)."""

    _fields_ = [("rho", ctypes.c_float), ("lambda_", ctypes.c_float),
                ("gamma", ctypes.c_float), ("iters", ctypes.c_int), ("tol", ctypes.c_float),
                ("check_every", ctypes.c_int), ("denoiser", ctypes.c_int),
                ("tv_inner", ctypes.c_int), ("tv_tau", ctypes.c_float),
                ("bm3d_sigma", ctypes.c_float), ("init_user", ctypes.c_int),
                ("storage", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    """Mirror of cslsm_batch_item."""

    _fields_ = [("plan", ctypes.c_void_p), ("b", ctypes.c_void_p), ("v_out", ctypes.c_void_p)]


class UnrolledParams(ctypes.Structure):
    """Mirror of cslsm_unrolled_params."""

    _fields_ = [("rho", ctypes.c_float), ("lambda_", ctypes.c_float), ("gamma", ctypes.c_float),
                ("iters", ctypes.c_int), ("tv_steps", ctypes.c_int), ("tv_tau", ctypes.c_float),
                ("huber_eps", ctypes.c_float), ("ckpt_every", ctypes.c_int),
                ("keep_duals", ctypes.c_int)]


class AdmmStats(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int), ("rel_change", ctypes.c_double)]


@dataclasses.dataclass
class Params:
    """Algorithm-1 parameters (see cslsm_admm_params in include/cslsm.h)."""

    rho: float = 1.0
    lam: float = 0.05
    gamma: float = 0.0
    iters: int = 50
    denoiser: str = "tv"
    tol: float = 0.0
    check_every: int = 1
    tv_inner: int = 20
    tv_tau: float = 0.125
    bm3d_sigma: float = 0.05
    storage: str = "fp32"

    def to_c(self, init_user: bool = False) -> AdmmParams:
        return AdmmParams(float(self.rho), float(self.lam), float(self.gamma), int(self.iters),
                          float(self.tol), int(self.check_every), DENOISERS[self.denoiser],
                          int(self.tv_inner), float(self.tv_tau), float(self.bm3d_sigma),
                          int(bool(init_user)), STORAGE[self.storage])


_lib = None


def lib() -> ctypes.CDLL:
    """Load libcslsm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libcslsm.so not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    sigs = {
        "cslsm_plan_create": [ctypes.POINTER(P), I, I, I, I, P, I, P],
        "cslsm_plan_set_masks": [P, P, I, P],
        "cslsm_plan_destroy": [P],
        "cslsm_forward": [P, P, P, P],
        "cslsm_adjoint": [P, P, P, P],
        "cslsm_admm_solve": [P, P, ctypes.POINTER(AdmmParams), P, P, P,
                             ctypes.POINTER(AdmmStats), P],
        "cslsm_denoise": [I, P, P, I, I, I, ctypes.POINTER(AdmmParams), P],
        "cslsm_psnr": [P, P, ctypes.c_size_t, P, P],
        "cslsm_ssim3d": [P, P, I, I, I, P, P],
        "cslsm_bm3d_match": [P, I, I, I, I, P, P, P],
        "cslsm_bm3d_stage": [I, P, P, P, I, I, I, F, P],
        "cslsm_bm3d_stage_groups": [I, P, P, P, I, I, I, F, P, P, P, P],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = I
    L.cslsm_status_string.argtypes = [I]
    L.cslsm_status_string.restype = ctypes.c_char_p
    L.cslsm_last_error.argtypes = []
    L.cslsm_last_error.restype = ctypes.c_char_p
    L.cslsm_abi_version.argtypes = []
    L.cslsm_abi_version.restype = I
    L.cslsm_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(BatchItem), I,
                                     ctypes.POINTER(AdmmParams), P]
    L.cslsm_batch_create.restype = I
    for name in ("cslsm_batch_run", "cslsm_batch_wait"):
        getattr(L, name).argtypes = [P, P]
        getattr(L, name).restype = I
    L.cslsm_batch_info.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I),
                                   ctypes.POINTER(ctypes.c_longlong)]
    L.cslsm_batch_info.restype = I
    L.cslsm_batch_set_wait_limit.argtypes = [P, ctypes.c_double, I]
    L.cslsm_batch_set_wait_limit.restype = I
    L.cslsm_batch_destroy.argtypes = [P]
    L.cslsm_batch_destroy.restype = I
    L.cslsm_unrolled_workspace_bytes.argtypes = [I, I, I, I, ctypes.POINTER(UnrolledParams)]
    L.cslsm_unrolled_workspace_bytes.restype = ctypes.c_size_t
    L.cslsm_unrolled_forward.argtypes = [P, P, I, I, I, I, ctypes.POINTER(UnrolledParams), P, P,
                                         P, P]
    L.cslsm_unrolled_forward.restype = I
    L.cslsm_unrolled_backward.argtypes = [P, P, I, I, I, I, ctypes.POINTER(UnrolledParams), P, P,
                                          P, P, P, P]
    L.cslsm_unrolled_backward.restype = I
    L.cslsm_bm3d_noalloc_capacity.argtypes = []
    L.cslsm_bm3d_noalloc_capacity.restype = ctypes.c_size_t
    L.cslsm_bm3d_scratch_bytes.argtypes = [I, I, I]
    L.cslsm_bm3d_scratch_bytes.restype = ctypes.c_size_t
    L.cslsm_denoise_bm3d_noalloc.argtypes = [P, P, I, I, I, F, P]
    L.cslsm_denoise_bm3d_noalloc.restype = I
    L.cslsm_tv_shape.argtypes = [I, I, I, I, P]
    L.cslsm_tv_shape.restype = I
    L.cslsm_set_autotune.argtypes = [I]
    L.cslsm_set_autotune.restype = I
    L.cslsm_set_batch_steps_per_phase.argtypes = [I]
    L.cslsm_set_batch_steps_per_phase.restype = I
    L.cslsm_set_tv_route.argtypes = [I]
    L.cslsm_set_tv_route.restype = I
    L.cslsm_zsweep_config.argtypes = [I, I, ctypes.c_double, I]
    L.cslsm_zsweep_config.restype = I
    L.cslsm_zsweep_num_tilings.argtypes = []
    L.cslsm_zsweep_num_tilings.restype = I
    L.cslsm_zsweep_shape.argtypes = [I, I, I, I, I, P]
    L.cslsm_zsweep_shape.restype = I
    L.cslsm_bm3d_num_refs.argtypes = [I, I]
    L.cslsm_bm3d_num_refs.restype = I
    L.cslsm_launch_count.argtypes = []
    L.cslsm_launch_count.restype = ctypes.c_ulonglong
    L.cslsm_timing_enable.argtypes = [I]
    L.cslsm_timing_enable.restype = I
    L.cslsm_timing_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_double), I]
    L.cslsm_timing_read.restype = I
    _lib = L
    return L


def _check(status: int, func: str) -> None:
    if status != 0:
        raise CslsmError(status, func, lib().cslsm_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, name: str, dtype: torch.dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """An acquisition geometry with its packed DMD patterns (cslsm_plan)."""

    def __init__(self, H: int, W: int, n_shots: int, R: int, masks: torch.Tensor,
                 per_slice: bool = True, stream=None):
        self.H, self.W, self.N, self.R = int(H), int(W), int(n_shots), int(R)
        self.Z = self.N * self.R
        self.per_slice = bool(per_slice)
        self._h = ctypes.c_void_p()
        mp = _dev(masks, "masks", torch.uint8,
                  (self.Z if per_slice else self.R, self.H, self.W))
        _check(lib().cslsm_plan_create(ctypes.byref(self._h), self.H, self.W, self.N, self.R,
                                       mp, int(self.per_slice), _stream(stream)),
               "cslsm_plan_create")

    @property
    def vol_shape(self):
        return (self.Z, self.H, self.W)

    @property
    def meas_shape(self):
        return (self.N, self.H, self.W)

    def set_masks(self, masks: torch.Tensor, stream=None) -> None:
        mp = _dev(masks, "masks", torch.uint8,
                  (self.Z if self.per_slice else self.R, self.H, self.W))
        _check(lib().cslsm_plan_set_masks(self._h, mp, int(self.per_slice), _stream(stream)),
               "cslsm_plan_set_masks")

    def forward(self, v: torch.Tensor, b: torch.Tensor | None = None, stream=None):
        if b is None:
            b = torch.empty(self.meas_shape, dtype=torch.float32, device=v.device)
        _check(lib().cslsm_forward(self._h, _dev(v, "v", torch.float32, self.vol_shape),
                                   _dev(b, "b", torch.float32, self.meas_shape),
                                   _stream(stream)), "cslsm_forward")
        return b

    def adjoint(self, b: torch.Tensor, v: torch.Tensor | None = None, stream=None):
        if v is None:
            v = torch.empty(self.vol_shape, dtype=torch.float32, device=b.device)
        _check(lib().cslsm_adjoint(self._h, _dev(b, "b", torch.float32, self.meas_shape),
                                   _dev(v, "v", torch.float32, self.vol_shape),
                                   _stream(stream)), "cslsm_adjoint")
        return v

    def solve(self, b: torch.Tensor, params: Params, v_out: torch.Tensor | None = None,
              u: torch.Tensor | None = None, d: torch.Tensor | None = None,
              init_user: bool = False, stream=None, stats: bool = False):
        """Algorithm 1; returns v^K (and the cslsm_admm_stats fields if stats).
        u, d (optional state) have the dtype of params.storage."""
        if v_out is None:
            v_out = torch.empty(self.vol_shape, dtype=torch.float32, device=b.device)
        sd = STORAGE_DTYPE[params.storage]
        up = _dev(u, "u", sd, self.vol_shape) if u is not None else None
        dp = _dev(d, "d", sd, self.vol_shape) if d is not None else None
        st = AdmmStats()
        cp = params.to_c(init_user)
        _check(lib().cslsm_admm_solve(self._h, _dev(b, "b", torch.float32, self.meas_shape),
                                      ctypes.byref(cp), _dev(v_out, "v_out", torch.float32,
                                                             self.vol_shape),
                                      up, dp, ctypes.byref(st), _stream(stream)),
               "cslsm_admm_solve")
        if stats:
            return v_out, {"iters_done": st.iters_done, "rel_change": st.rel_change}
        return v_out

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _check(lib().cslsm_plan_destroy(self._h), "cslsm_plan_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def denoise(x: torch.Tensor, params: Params, out: torch.Tensor | None = None, stream=None):
    """The u-step prior alone on each slice of x [Z,H,W] (cslsm_denoise)."""
    if x.dim() == 2:
        x = x[None]
    Z, H, W = x.shape
    if out is None:
        out = torch.empty_like(x)
    cp = params.to_c()
    _check(lib().cslsm_denoise(cp.denoiser, _dev(x, "x", torch.float32),
                               _dev(out, "out", torch.float32, (Z, H, W)), Z, H, W,
                               ctypes.byref(cp), _stream(stream)), "cslsm_denoise")
    return out


def psnr(x: torch.Tensor, ref: torch.Tensor, stream=None) -> torch.Tensor:
    """Volume PSNR (Sec. IV) as a 1-element float64 CUDA tensor."""
    if x.shape != ref.shape:
        raise ValueError("x and ref must have the same shape")
    out = torch.empty(1, dtype=torch.float64, device=x.device)
    _check(lib().cslsm_psnr(_dev(x, "x", torch.float32), _dev(ref, "ref", torch.float32),
                            x.numel(), ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "cslsm_psnr")
    return out


def ssim3d(x: torch.Tensor, ref: torch.Tensor, stream=None) -> torch.Tensor:
    """Volume SSIM of Sec. IV (cslsm_ssim3d) as a 0-dim float64 CUDA tensor."""
    if x.dim() == 2:
        x, ref = x[None], ref[None]
    Z, H, W = x.shape
    out = torch.empty((), dtype=torch.float64, device=x.device)
    _check(lib().cslsm_ssim3d(_dev(x, "x", torch.float32), _dev(ref, "ref", torch.float32,
                                                                (Z, H, W)),
                              Z, H, W, out.data_ptr(), _stream(stream)), "cslsm_ssim3d")
    return out


def launch_count() -> int:
    """Kernels launched by libcslsm in this process so far."""
    return int(lib().cslsm_launch_count())


def timing_enable(period: int) -> None:
    """Sample every period-th launch of each kernel with CUDA events (0: off)."""
    _check(lib().cslsm_timing_enable(int(period)), "cslsm_timing_enable")


def timing_read(kernel: str, reset: bool = False) -> tuple[int, float]:
    """(launches timed, summed device milliseconds) for one kernel name; reset
    clears the records of every kernel."""
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    _check(lib().cslsm_timing_read(kernel.encode(), ctypes.byref(n), ctypes.byref(ms),
                                   int(bool(reset))), "cslsm_timing_read")
    return int(n.value), float(ms.value)


def bm3d_match(img: torch.Tensor, stage: int, stream=None):
    """Block-matching groups of every reference of each slice of img [Z,H,W]:
    (lists int32 [Z,nref,16] of y*W+x positions, counts int32 [Z,nref])."""
    if img.dim() == 2:
        img = img[None]
    Z, H, W = img.shape
    nref = int(lib().cslsm_bm3d_num_refs(H, W))
    lists = torch.empty((Z, nref, 16), dtype=torch.int32, device=img.device)
    counts = torch.empty((Z, nref), dtype=torch.int32, device=img.device)
    _check(lib().cslsm_bm3d_match(_dev(img, "img", torch.float32), Z, H, W, int(stage),
                                  ctypes.c_void_p(lists.data_ptr()),
                                  ctypes.c_void_p(counts.data_ptr()), _stream(stream)),
           "cslsm_bm3d_match")
    return lists, counts


def bm3d_stage(stage: int, noisy: torch.Tensor, sigma: float, guide: torch.Tensor | None = None,
               out: torch.Tensor | None = None, stream=None):
    """One BM3D stage on each slice: 1 = hard threshold, 2 = Wiener guided by `guide`."""
    if noisy.dim() == 2:
        noisy = noisy[None]
        guide = guide[None] if guide is not None else None
    Z, H, W = noisy.shape
    if out is None:
        out = torch.empty_like(noisy)
    gp = _dev(guide, "guide", torch.float32, (Z, H, W)) if guide is not None else None
    _check(lib().cslsm_bm3d_stage(int(stage), _dev(noisy, "noisy", torch.float32), gp,
                                  _dev(out, "out", torch.float32, (Z, H, W)), Z, H, W,
                                  float(sigma), _stream(stream)), "cslsm_bm3d_stage")
    return out


def bm3d_stage_groups(stage: int, noisy: torch.Tensor, sigma: float,
                      guide: torch.Tensor | None = None, stream=None):
    """One BM3D stage on each slice with its decisions (cslsm_bm3d_stage_groups):
    (out [Z,H,W], lists int32 [Z,nref,16], counts int32 [Z,nref], stat float32
    [Z,nref]: kept coefficients per group (stage 1) or sum of squared Wiener factors)."""
    if noisy.dim() == 2:
        noisy = noisy[None]
        guide = guide[None] if guide is not None else None
    Z, H, W = noisy.shape
    nref = lib().cslsm_bm3d_num_refs(H, W)
    out = torch.empty_like(noisy)
    lists = torch.empty((Z, nref, 16), dtype=torch.int32, device=noisy.device)
    counts = torch.empty((Z, nref), dtype=torch.int32, device=noisy.device)
    stat = torch.empty((Z, nref), dtype=torch.float32, device=noisy.device)
    gp = _dev(guide, "guide", torch.float32, (Z, H, W)) if guide is not None else None
    _check(lib().cslsm_bm3d_stage_groups(int(stage), _dev(noisy, "noisy", torch.float32), gp,
                                         _dev(out, "out", torch.float32, (Z, H, W)), Z, H, W,
                                         float(sigma), ctypes.c_void_p(lists.data_ptr()),
                                         ctypes.c_void_p(counts.data_ptr()),
                                         ctypes.c_void_p(stat.data_ptr()), _stream(stream)),
           "cslsm_bm3d_stage_groups")
    return out, lists, counts, stat


def set_autotune(mode: int) -> None:
    """TV tile shapes: 0 cost model, 1 timed autotuning, 2..5 force a variant."""
    _check(lib().cslsm_set_autotune(int(mode)), "cslsm_set_autotune")


def set_tv_route(mode: int) -> None:
    """Slice-independent TV solves: 0 auto (a one-item persistent batch for large
    volumes), 1 per-launch tiles, 2 always the batch; the same bits either way."""
    _check(lib().cslsm_set_tv_route(int(mode)), "cslsm_set_tv_route")


def set_batch_steps_per_phase(k: int) -> None:
    """Chambolle steps per phase of batches created from now on: 0 the default
    (or the timed choice under set_autotune(1)), k >= 1 that many."""
    _check(lib().cslsm_set_batch_steps_per_phase(int(k)), "cslsm_set_batch_steps_per_phase")


def tv_shape(H: int, W: int, steps: int, nslices: int) -> dict:
    """The TV kernel variant and tile shape a launch of this geometry uses now."""
    buf = (ctypes.c_int * 4)()
    _check(lib().cslsm_tv_shape(int(H), int(W), int(steps), int(nslices), buf),
           "cslsm_tv_shape")
    return {"variant": buf[0], "tile_rows": buf[1], "tile_cols": buf[2], "region_rows": buf[3]}


def zsweep_config(enable: bool = True, tiling: int = -1, wait_limit_s: float = 2.0,
                  test_stall: bool = False) -> None:
    """Persistent z sweep of the TV u-step (gamma > 0): on/off, forced tiling
    (-1: chosen per geometry), device-side wait limit, timeout test hook."""
    _check(lib().cslsm_zsweep_config(int(bool(enable)), int(tiling), float(wait_limit_s),
                                     int(bool(test_stall))), "cslsm_zsweep_config")


def zsweep_num_tilings() -> int:
    return int(lib().cslsm_zsweep_num_tilings())


def zsweep_shape(H: int, W: int, Z: int, steps: int, storage: str = "fp32") -> dict:
    """The sweep tiling a solve of this geometry uses now."""
    buf = (ctypes.c_int * 8)()
    _check(lib().cslsm_zsweep_shape(int(H), int(W), int(Z), int(steps), STORAGE[storage], buf),
           "cslsm_zsweep_shape")
    keys = ("tiling", "steps_per_phase", "rows_per_warp", "warps", "tile_rows", "tile_cols",
            "region_rows", "tiles")
    return dict(zip(keys, list(buf)))


def denoise_bm3d_noalloc(x: torch.Tensor, sigma: float, out: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """BM3D of each slice of x [Z,H,W] using the library's fixed scratch array
    (cslsm_denoise_bm3d_noalloc: no device allocation by the library; `out`
    must be provided by callers that cannot let torch allocate either)."""
    if x.dim() == 2:
        x = x[None]
    Z, H, W = x.shape
    if out is None:
        out = torch.empty_like(x)
    with torch.cuda.device(x.device):  # the scratch array used is the current device's
        _check(lib().cslsm_denoise_bm3d_noalloc(_dev(x, "x", torch.float32),
                                                _dev(out, "out", torch.float32, (Z, H, W)), Z,
                                                H, W, float(sigma), _stream(stream)),
               "cslsm_denoise_bm3d_noalloc")
    return out


class Batch:
    """Many measurements solved by one persistent launch replayed from a CUDA graph
    (cslsm_batch_*).  items: list of (Plan, b, v_out) with device tensors."""

    def __init__(self, items, params: Params, stream=None):
        self._keep = list(items)  # the batch records these tensors' addresses
        arr = (BatchItem * len(items))()
        for k, (plan, b, v_out) in enumerate(items):
            arr[k] = BatchItem(plan._h, _dev(b, "b", torch.float32, plan.meas_shape),
                               _dev(v_out, "v_out", torch.float32, plan.vol_shape))
        self._h = ctypes.c_void_p()
        cp = params.to_c()
        _check(lib().cslsm_batch_create(ctypes.byref(self._h), arr, len(items), ctypes.byref(cp),
                                        _stream(stream)), "cslsm_batch_create")

    def run(self, stream=None) -> None:
        _check(lib().cslsm_batch_run(self._h, _stream(stream)), "cslsm_batch_run")

    def wait(self, stream=None) -> None:
        _check(lib().cslsm_batch_wait(self._h, _stream(stream)), "cslsm_batch_wait")

    def info(self) -> dict:
        """The schedule: Chambolle steps per phase, CTAs of the persistent
        launch, work units per ADMM iteration."""
        k, grid, units = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        _check(lib().cslsm_batch_info(self._h, ctypes.byref(k), ctypes.byref(grid),
                                      ctypes.byref(units)), "cslsm_batch_info")
        return {"steps_per_phase": k.value, "grid": grid.value, "units_per_iteration": units.value}

    def set_wait_limit(self, seconds: float, test_stall: bool = False) -> None:
        _check(lib().cslsm_batch_set_wait_limit(self._h, float(seconds), int(test_stall)),
               "cslsm_batch_set_wait_limit")

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _check(lib().cslsm_batch_destroy(self._h), "cslsm_batch_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _unrolled_params(rho, lam, gamma, cfg) -> UnrolledParams:
    return UnrolledParams(float(rho), float(lam), float(gamma), int(cfg["iters"]),
                          int(cfg["tv_steps"]), float(cfg["tv_tau"]), float(cfg["huber_eps"]),
                          int(cfg["ckpt_every"]), int(bool(cfg.get("keep_duals", False))))


class _UnrolledADMM(torch.autograd.Function):
    """v^K of the unrolled, relaxed PnP-ADMM (cslsm_unrolled_forward); its backward is
    the library's hand-written adjoint (cslsm_unrolled_backward)."""

    @staticmethod
    def forward(ctx, logits, b, rho, lam, gamma, cfg):
        B, Z, H, W = logits.shape
        cp = _unrolled_params(rho.item(), lam.item(), gamma.item(), cfg)
        nbytes = lib().cslsm_unrolled_workspace_bytes(B, Z, H, W, ctypes.byref(cp))
        if nbytes == 0:
            raise ValueError("invalid unrolled-solver parameters or sizes")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=logits.device)
        nck = -(-cfg["iters"] // cfg["ckpt_every"])
        ckpt = torch.empty((nck, 2, B, Z, H, W), dtype=torch.float32, device=logits.device)
        v = torch.empty_like(logits)
        _check(lib().cslsm_unrolled_forward(_dev(logits, "logits", torch.float32),
                                            _dev(b, "b", torch.float32, (B, H, W)), B, Z, H, W,
                                            ctypes.byref(cp), _dev(v, "v", torch.float32),
                                            _dev(ckpt, "ckpt", torch.float32),
                                            ctypes.c_void_p(ws.data_ptr()), _stream()),
               "cslsm_unrolled_forward")
        ctx.save_for_backward(logits, b, ckpt)
        ctx.ws, ctx.cp = ws, cp
        return v

    @staticmethod
    def backward(ctx, vbar):
        logits, b, ckpt = ctx.saved_tensors
        B, Z, H, W = logits.shape
        vbar = vbar.contiguous().float()
        lbar = torch.empty_like(logits)
        sbar = torch.empty(3, dtype=torch.float64, device=logits.device)
        _check(lib().cslsm_unrolled_backward(_dev(logits, "logits", torch.float32),
                                             _dev(b, "b", torch.float32), B, Z, H, W,
                                             ctypes.byref(ctx.cp), _dev(ckpt, "ckpt", torch.float32),
                                             _dev(vbar, "vbar", torch.float32),
                                             _dev(lbar, "lbar", torch.float32),
                                             ctypes.c_void_p(sbar.data_ptr()),
                                             ctypes.c_void_p(ctx.ws.data_ptr()), _stream()),
               "cslsm_unrolled_backward")
        s = sbar.to(torch.float32)
        return lbar, None, s[0], s[1], s[2], None


def unrolled_admm(logits: torch.Tensor, b: torch.Tensor, rho: torch.Tensor, lam: torch.Tensor,
                  gamma: torch.Tensor, iters: int = 30, tv_steps: int = 20, tv_tau: float = 0.125,
                  huber_eps: float = 1e-3, ckpt_every: int = 5,
                  keep_duals: bool = False) -> torch.Tensor:
    """Differentiable v^K of the unrolled PnP-ADMM with relaxed masks sigmoid(logits)
    [B,Z,H,W] and Huber-TV + z prior; b [B,H,W]; rho, lam, gamma 0-dim tensors.
    keep_duals: the backward keeps the dual iterates of a checkpoint segment
    instead of recomputing them per slice (more device memory, same gradients)."""
    cfg = dict(iters=iters, tv_steps=tv_steps, tv_tau=tv_tau, huber_eps=huber_eps,
               ckpt_every=ckpt_every, keep_duals=keep_duals)
    return _UnrolledADMM.apply(logits, b, rho, lam, gamma, cfg)
