"""PyTorch layers over the C ABI: Signal2SH, SH2Signal, LocalSphericalConvolution.

The classes mirror the paper's three layers (Sec. 2.2 and 2.3) and their
parameter names.  Torch supplies device memory, the current CUDA stream and
autograd; every arithmetic step runs in libdelimit's kernels.  Tensors are
feature-rows x voxel-columns (the paper's tensor with the voxel axes
flattened, Sec. 2.1); 5-D inputs [subjects, features, H, W, D] are accepted
and reshaped.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import _lib as L

_DT = {torch.float32: L.F32, torch.bfloat16: L.BF16}


def _code(t: torch.Tensor) -> int:
    if t.dtype not in _DT:
        raise TypeError(f"unsupported dtype {t.dtype}: float32 or bfloat16")
    return _DT[t.dtype]


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def padded_ld(n_vox: int) -> int:
    """Row stride (elements) that keeps every row 16-byte aligned for both dtypes."""
    return max(8, (int(n_vox) + 7) // 8 * 8)


def empty_act(rows: int, n_vox: int, dtype, device="cuda") -> torch.Tensor:
    """[rows, n_vox] view of a [rows, padded_ld] buffer (the library's activation layout)."""
    return torch.empty((rows, padded_ld(n_vox)), dtype=dtype, device=device)[:, :n_vox]


def as_act(x: torch.Tensor) -> torch.Tensor:
    """x as a 2-D activation with unit voxel stride and an aligned row stride (copies if needed)."""
    if x.dim() != 2:
        raise ValueError("activations are 2-D [features, voxels]")
    ok = x.stride(1) == 1 and (x.stride(0) * x.element_size()) % 16 == 0 and x.data_ptr() % 16 == 0 \
        and x.stride(0) >= x.shape[1]
    if ok:
        return x
    y = empty_act(x.shape[0], x.shape[1], x.dtype, x.device)
    y.copy_(x)
    return y


# ---------------------------------------------------------------------------
# raw calls (tensors in, tensors out)
# ---------------------------------------------------------------------------
_TRANSFORMS = {
    "signal2sh": "delimit_signal2sh",
    "sh2signal": "delimit_sh2signal",
    "signal2sh_backward": "delimit_signal2sh_backward",
    "sh2signal_backward": "delimit_sh2signal_backward",
}


def transform(kind: str, basis: L.SHBasis, x: torch.Tensor, channels: int, out_dtype=None,
              out: torch.Tensor | None = None) -> torch.Tensor:
    """One of the four transforms; output rows follow the library's row order."""
    x = as_act(x)
    n_vox = x.shape[1]
    to_sh = kind in ("signal2sh", "sh2signal_backward")
    rows_out = basis.n_shells * channels * basis.n_coef if to_sh else channels * basis.n_dirs
    rows_in = channels * basis.n_dirs if to_sh else basis.n_shells * channels * basis.n_coef
    if x.shape[0] != rows_in:
        raise ValueError(f"{kind}: expected {rows_in} input rows, got {x.shape[0]}")
    od = out_dtype or x.dtype
    if out is None:
        out = empty_act(rows_out, n_vox, od, x.device)
    fn = getattr(L.get(), _TRANSFORMS[kind])
    L.check(fn(basis.handle, x.data_ptr(), out.data_ptr(), n_vox, channels, x.stride(0), out.stride(0), _code(x),
               _code(out), _stream()), _TRANSFORMS[kind])
    return out


def signal2sh_gather(basis: L.SHBasis, dwi: torch.Tensor, index: torch.Tensor, n: int | None = None,
                     b0: torch.Tensor | None = None, channels: int = 1, out_dtype=None) -> torch.Tensor:
    """Signal2SH of the voxels ``index`` (int64, device) of the volume ``dwi``
    [channels x directions, n_src], divided by ``b0`` [n_src] (float32) first when
    given; returns SH rows [S*channels*N, n]."""
    if dwi.dim() != 2 or dwi.stride(1) != 1:
        raise ValueError("dwi is 2-D [rows, voxels] with unit voxel stride")
    n = int(index.numel()) if n is None else int(n)
    out = empty_act(basis.n_shells * channels * basis.n_coef, max(n, 1), out_dtype or dwi.dtype, dwi.device)[:, :n]
    b0p = None
    if b0 is not None:
        b0 = b0.contiguous().float()
        b0p = b0.data_ptr()
    index = index.contiguous()
    L.check(L.get().delimit_signal2sh_gather(basis.handle, dwi.data_ptr(), dwi.stride(0), dwi.shape[1], b0p,
                                             index.data_ptr(), n, out.data_ptr(), out.stride(0), channels,
                                             _code(dwi), _DT[out.dtype], _stream()), "delimit_signal2sh_gather")
    return out


def lsc_workspace(geom: L.LSCGeometry, n_vox: int, c_in: int, c_out: int, dtype, backward: bool, device="cuda"):
    """(keep-alive tensor, 256-byte aligned pointer, bytes) of an LSC workspace."""
    ws_n = geom.workspace_size(n_vox, c_in, c_out, _DT[dtype], backward)
    ws = torch.empty(ws_n + 256, dtype=torch.uint8, device=device)
    return ws, (ws.data_ptr() + 255) // 256 * 256, ws_n


def lsc_forward(geom: L.LSCGeometry, x: torch.Tensor, w: torch.Tensor, b: torch.Tensor | None, c_in: int,
                c_out: int, out: torch.Tensor | None = None, workspace=None) -> torch.Tensor:
    """``workspace``: optional (tensor, ptr, bytes) from lsc_workspace; a backward-sized
    workspace lets the following backward reuse the operator built here."""
    x = as_act(x)
    n_vox = x.shape[1]
    if out is None:
        out = empty_act(geom.s_out * c_out * geom.n_out, n_vox, x.dtype, x.device)
    _, wsp, ws_n = workspace if workspace is not None else lsc_workspace(geom, n_vox, c_in, c_out, x.dtype, False,
                                                                         x.device)
    w = w.detach().contiguous().float()
    bf = b.detach().contiguous().float() if b is not None else None  # lives until after the launch
    bp = bf.data_ptr() if bf is not None else None
    L.check(L.get().delimit_lsc_forward(geom.handle, x.data_ptr(), w.data_ptr(), bp, out.data_ptr(), n_vox, c_in,
                                        c_out, x.stride(0), out.stride(0), _code(x), 0, wsp, ws_n, _stream()),
            "delimit_lsc_forward")
    return out


def lsc_forward_sh2signal_supported(geom: L.LSCGeometry, n_vox: int, c_in: int, c_out: int, dtype) -> bool:
    """Whether the fused LSC forward + SH2Signal kernel takes these sizes (else run
    lsc_forward and transform("sh2signal", ...) one after the other)."""
    return L.get().delimit_lsc_forward_sh2signal_supported(geom.handle, n_vox, c_in, c_out, _DT[dtype]) == L.OK


def lsc_forward_sh2signal(geom: L.LSCGeometry, x: torch.Tensor, w: torch.Tensor, b: torch.Tensor | None, c_in: int,
                          c_out: int, out: torch.Tensor | None = None, workspace=None) -> torch.Tensor:
    """The LSC forward followed by SH2Signal on the geometry's output directions, one kernel:
    returns signal rows [c_out * total directions, n_vox] (the output SH never leaves the chip)."""
    x = as_act(x)
    n_vox = x.shape[1]
    if out is None:
        out = empty_act(c_out * geom.out_basis.n_dirs, n_vox, x.dtype, x.device)
    _, wsp, ws_n = workspace if workspace is not None else lsc_workspace(geom, n_vox, c_in, c_out, x.dtype, False,
                                                                         x.device)
    w = w.detach().contiguous().float()
    bf = b.detach().contiguous().float() if b is not None else None  # lives until after the launch
    L.check(L.get().delimit_lsc_forward_sh2signal(geom.handle, x.data_ptr(), w.data_ptr(),
                                                  bf.data_ptr() if bf is not None else None, out.data_ptr(), n_vox,
                                                  c_in, c_out, x.stride(0), out.stride(0), _code(x), 0, wsp, ws_n,
                                                  _stream()), "delimit_lsc_forward_sh2signal")
    return out


def lsc_backward(geom: L.LSCGeometry, x: torch.Tensor, w: torch.Tensor, d_out: torch.Tensor, c_in: int, c_out: int,
                 need_input: bool = True, need_weight: bool = True, need_bias: bool = True, workspace=None,
                 operator_ready: bool = False):
    """``workspace`` + ``operator_ready``: reuse the operator a forward built in this workspace."""
    x = as_act(x)
    d_out = as_act(d_out.to(x.dtype))
    n_vox = x.shape[1]
    d_in = empty_act(x.shape[0], n_vox, x.dtype, x.device) if need_input else None
    w = w.detach().contiguous().float()
    dw = torch.empty_like(w) if need_weight else None
    db = torch.empty((c_out, geom.s_out), dtype=torch.float32, device=x.device) if need_bias else None
    if workspace is None:
        workspace, operator_ready = lsc_workspace(geom, n_vox, c_in, c_out, x.dtype, True, x.device), False
    _, wsp, ws_n = workspace
    L.check(L.get().delimit_lsc_backward(
        geom.handle, x.data_ptr(), w.data_ptr(), d_out.data_ptr(), d_in.data_ptr() if d_in is not None else None,
        dw.data_ptr() if dw is not None else None, db.data_ptr() if db is not None else None, n_vox, c_in, c_out,
        x.stride(0), d_out.stride(0), _code(x), L.OPERATOR_READY if operator_ready else 0, wsp, ws_n, _stream()),
        "delimit_lsc_backward")
    return d_in, dw, db


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------
class _TransformFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, basis, kind, channels, out_dtype):
        ctx.basis, ctx.kind, ctx.channels, ctx.in_dtype = basis, kind, channels, x.dtype
        return transform(kind, basis, x, channels, out_dtype)

    @staticmethod
    def backward(ctx, g):
        adj = {"signal2sh": "signal2sh_backward", "sh2signal": "sh2signal_backward"}[ctx.kind]
        gx = transform(adj, ctx.basis, g, ctx.channels, ctx.in_dtype)
        return gx, None, None, None, None


class _LSCFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, b, geom, c_in, c_out):
        ctx.geom, ctx.c_in, ctx.c_out = geom, c_in, c_out
        ctx.has_b = b is not None
        ctx.save_for_backward(x, w)
        # a backward-sized workspace: the backward reuses the operator built here
        ws = lsc_workspace(geom, x.shape[1], c_in, c_out, x.dtype, True, x.device) \
            if any(ctx.needs_input_grad) else None
        ctx.ws = ws
        return lsc_forward(geom, x, w, b, c_in, c_out, workspace=ws)

    @staticmethod
    def backward(ctx, g):
        x, w = ctx.saved_tensors
        d_in, dw, db = lsc_backward(ctx.geom, x, w, g, ctx.c_in, ctx.c_out, need_input=ctx.needs_input_grad[0],
                                    need_weight=ctx.needs_input_grad[1],
                                    need_bias=ctx.has_b and ctx.needs_input_grad[2], workspace=ctx.ws,
                                    operator_ready=ctx.ws is not None)
        ctx.ws = None
        return d_in, dw, db, None, None, None


def leaky_relu(x: torch.Tensor, slope: float) -> torch.Tensor:
    x = as_act(x)
    y = empty_act(x.shape[0], x.shape[1], x.dtype, x.device)
    L.check(L.get().delimit_leaky_relu(x.data_ptr(), y.data_ptr(), x.shape[0], x.shape[1], x.stride(0), y.stride(0),
                                       float(slope), _code(x), _stream()), "delimit_leaky_relu")
    return y


class _LeakyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, slope):
        y = leaky_relu(x, slope)
        ctx.slope = slope
        ctx.save_for_backward(y)
        return y

    @staticmethod
    def backward(ctx, g):
        (y,) = ctx.saved_tensors
        g = as_act(g.to(y.dtype))
        dx = empty_act(y.shape[0], y.shape[1], y.dtype, y.device)
        L.check(L.get().delimit_leaky_relu_backward(y.data_ptr(), g.data_ptr(), dx.data_ptr(), y.shape[0], y.shape[1],
                                                    y.stride(0), g.stride(0), dx.stride(0), float(ctx.slope), _code(y),
                                                    _stream()), "delimit_leaky_relu_backward")
        return dx, None


class LeakyReLU(torch.nn.Module):
    """Leaky ReLU on SH activations, in the library's kernels."""

    def __init__(self, slope: float = 0.1):
        super().__init__()
        self.slope = float(slope)

    def forward(self, x):
        return _LeakyFn.apply(x, self.slope)


def _to_rows(x: torch.Tensor):
    """5-D [B, F, H, W, D] -> ([F, B*H*W*D], restore) ; 2-D passes through."""
    if x.dim() == 2:
        return x, lambda y: y
    if x.dim() != 5:
        raise ValueError("expected a 2-D [features, voxels] or 5-D [subjects, features, H, W, D] tensor")
    B, F, H, W, D = x.shape
    flat = x.reshape(B, F, H * W * D).permute(1, 0, 2).reshape(F, B * H * W * D)

    def restore(y):
        return y.reshape(y.shape[0], B, H, W, D).permute(1, 0, 2, 3, 4)
    return flat, restore


class Signal2SH(torch.nn.Module):
    """Signal -> SH per shell (Sec. 2.2): sh_order, gradients, lb_lambda; b-values optional (one shell)."""

    def __init__(self, sh_order: int, gradients, lb_lambda: float = 0.0, bvals=None, channels: int = 1,
                 out_dtype=None):
        super().__init__()
        g = np.asarray(gradients, np.float64).reshape(-1, 3)
        b = np.full(g.shape[0], 1000.0) if bvals is None else np.asarray(bvals, np.float64)
        self.basis = L.SHBasis(g, b, sh_order, lb_lambda)
        self.channels, self.out_dtype = channels, out_dtype

    def forward(self, signal):
        x, restore = _to_rows(signal)
        return restore(_TransformFn.apply(x, self.basis, "signal2sh", self.channels, self.out_dtype))


class SH2Signal(torch.nn.Module):
    """SH -> signal on the given (resampled) gradient directions (Sec. 2.2)."""

    def __init__(self, sh_order: int, gradients, bvals=None, channels: int = 1, out_dtype=None):
        super().__init__()
        g = np.asarray(gradients, np.float64).reshape(-1, 3)
        b = np.full(g.shape[0], 1000.0) if bvals is None else np.asarray(bvals, np.float64)
        self.basis = L.SHBasis(g, b, sh_order, 0.0, eval_only=True)
        self.channels, self.out_dtype = channels, out_dtype

    def forward(self, sh):
        x, restore = _to_rows(sh)
        return restore(_TransformFn.apply(x, self.basis, "sh2signal", self.channels, self.out_dtype))


class _RingExpandFn(torch.autograd.Function):
    """w_ring [.., rings + 1] -> per-point w [.., K] (ring-tied kernel); backward folds dw."""

    @staticmethod
    def forward(ctx, w_ring, geom, c_in, c_out):
        ctx.geom, ctx.c_in, ctx.c_out = geom, c_in, c_out
        w_ring = w_ring.detach().contiguous().float()
        w = torch.empty(w_ring.shape[:-1] + (geom.K,), dtype=torch.float32, device=w_ring.device)
        L.check(L.get().delimit_lsc_ring_expand(geom.handle, w_ring.data_ptr(), w.data_ptr(), c_in, c_out, _stream()),
                "delimit_lsc_ring_expand")
        return w

    @staticmethod
    def backward(ctx, dw):
        dw = dw.contiguous().float()
        g = ctx.geom
        dr = torch.empty(dw.shape[:-1] + (g.rings + 1,), dtype=torch.float32, device=dw.device)
        L.check(L.get().delimit_lsc_ring_reduce(g.handle, dw.data_ptr(), dr.data_ptr(), ctx.c_in, ctx.c_out,
                                                 _stream()), "delimit_lsc_ring_reduce")
        return dr, None, None, None


def ring_expand(geom: L.LSCGeometry, w_ring: torch.Tensor, c_in: int, c_out: int) -> torch.Tensor:
    """Per-point weights of a ring-tied kernel (differentiable)."""
    return _RingExpandFn.apply(w_ring, geom, c_in, c_out)


class LocalSphericalConvolution(torch.nn.Module):
    """Local spherical convolution (Sec. 2.3) with the paper's parameters.

    ``kernel_sizes`` lists the points of each ring (all rings equal here); the
    rings are spread evenly out to ``angular_distance``.  ``window`` selects
    which input shells feed each output shell.  Weights: ``weight``
    [channels_out, shells_out, channels_in, shells_in, K] and ``bias``
    [channels_out, shells_out], FP32 masters.  ``ring_tied``: one weight for the
    origin and one per ring ([.., rings + 1]), shared by the ring's points (the
    isotropic kernel; frame-independent when sectors exceed the input order).
    ``resample=False``: the kernel meets the acquired neighbours of every direction
    (each binned to its nearest kernel point, a point taking the mean of its
    neighbours) instead of the SH-resampled neighbourhood; input shell s' is then
    the sampled table's shell s'.
    """

    def __init__(self, shells_in: int, shells_out: int, sampled_gradients, sh_order_in: int, sh_order_out: int,
                 kernel_sizes, lb_lambda: float = 0.0, angular_distance: float = math.pi / 5, bvals=None,
                 channels_in: int = 1, channels_out: int = 1, window: str | None = None, bias: bool = True,
                 ring_tied: bool = False, resample: bool = True):
        super().__init__()
        ks = list(kernel_sizes)
        if len(set(ks)) != 1:
            raise ValueError("all rings must have the same number of points")
        g = np.asarray(sampled_gradients, np.float64).reshape(-1, 3)
        b = np.full(g.shape[0], 1000.0) if bvals is None else np.asarray(bvals, np.float64)
        self.out_basis = L.SHBasis(g, b, sh_order_out, lb_lambda)
        if self.out_basis.n_shells != shells_out:
            raise ValueError(f"sampled gradients have {self.out_basis.n_shells} shells, shells_out={shells_out}")
        if window is None:
            window = "same" if shells_in == shells_out else "all"
        self.geom = L.LSCGeometry(self.out_basis, sh_order_in, shells_in, angular_distance, len(ks), ks[0], window,
                                  neighbours=not resample)
        self.c_in, self.c_out = channels_in, channels_out
        self.ring_tied = bool(ring_tied)
        K = len(ks) + 1 if self.ring_tied else self.geom.K
        self.weight = torch.nn.Parameter(torch.zeros(channels_out, shells_out, channels_in, shells_in, K))
        self.bias = torch.nn.Parameter(torch.zeros(channels_out, shells_out)) if bias else None

    def point_weights(self) -> torch.Tensor:
        """Per-point kernel weights [.., K] (the ring weights expanded when ring-tied)."""
        return ring_expand(self.geom, self.weight, self.c_in, self.c_out) if self.ring_tied else self.weight

    def forward(self, sh):
        x, restore = _to_rows(sh)
        return restore(_LSCFn.apply(x, self.point_weights(), self.bias, self.geom, self.c_in, self.c_out))
