"""Signal2SH -> LSC -> SH2Signal, forward and backward, as one reusable step.

This is the metric path of the layers: a multi-shell signal with C_in channels
is fitted per shell (Signal2SH, Sec. 2.2), convolved by one LSC layer mixing
channels and shells (Sec. 2.3), and evaluated back on the table's directions
(SH2Signal); back-propagation runs the adjoints in reverse order and yields
the weight and bias gradients.  Each step issues six C-ABI calls on the
current CUDA stream with preallocated buffers and workspaces.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from . import layers


@dataclass
class ChainConfig:
    n_vox: int = 65536
    dirs_per_shell: tuple = (90, 90, 90)
    bvals: tuple = (1000, 2000, 3000)
    order: int = 8
    lam: float = 0.006
    c_in: int = 16
    c_out: int = 64
    radius_deg: float = 25.0
    rings: int = 4
    sectors: int = 12
    window: str = "adjacent"
    seed: int = 1808
    order_in: int | None = None  # SH order of the LSC input (Signal2SH); None = order
    resample: bool = True  # False: the LSC over acquired neighbours (no SH resampling)

    @property
    def l_in(self) -> int:
        return self.order if self.order_in is None else self.order_in

    def name(self) -> str:
        orders = f"L={self.order}" if self.l_in == self.order else f"L={self.l_in}->{self.order}"
        return (f"S2SH-LSC-SH2S fwd+bwd V={self.n_vox} {len(self.dirs_per_shell)}x{self.dirs_per_shell[0]} dirs "
                f"{orders} {self.c_in}->{self.c_out} ch {self.window} {self.radius_deg:g}deg "
                f"{self.rings}x{self.sectors}" + ("" if self.resample else " resampling-free"))


class Chain:
    """Preallocated buffers + handles for one configuration and activation dtype."""

    CALLS = ("signal2sh", "lsc_forward", "sh2signal", "sh2signal_backward", "lsc_backward", "signal2sh_backward")
    # with the LSC forward and SH2Signal fused into one kernel (BF16, where the kernel takes the sizes)
    CALLS_FUSED = ("signal2sh", "lsc_forward_sh2signal", "sh2signal_backward", "lsc_backward", "signal2sh_backward")

    def __init__(self, cfg: ChainConfig, dirs: np.ndarray, bvals: np.ndarray, dtype=torch.bfloat16, device="cuda",
                 fused: bool = False):
        self.cfg, self.dtype = cfg, dtype
        self.code = L.BF16 if dtype == torch.bfloat16 else L.F32
        self.basis = L.SHBasis(dirs, bvals, cfg.order, cfg.lam)  # output side (LSC projection, SH2Signal)
        self.basis_in = self.basis if cfg.l_in == cfg.order else L.SHBasis(dirs, bvals, cfg.l_in, cfg.lam)
        self.geom = L.LSCGeometry(self.basis, cfg.l_in, self.basis.n_shells, np.deg2rad(cfg.radius_deg), cfg.rings,
                                  cfg.sectors, cfg.window, neighbours=not cfg.resample)
        V, S = cfg.n_vox, self.basis.n_shells
        ci, co = cfg.c_in, cfg.c_out
        self.rows = self.row_counts(cfg, self.basis, self.basis_in)
        mk = lambda r: layers.empty_act(r, V, dtype, device)  # noqa: E731
        self.s_in, self.c_in_buf = mk(self.rows["s_in"]), mk(self.rows["c_in"])
        self.c_out_buf, self.s_out = mk(self.rows["c_out"]), mk(self.rows["s_out"])
        self.ds_out, self.dc_out = mk(self.rows["s_out"]), mk(self.rows["c_out"])
        self.dc_in, self.ds_in = mk(self.rows["c_in"]), mk(self.rows["s_in"])
        K = self.geom.K
        self.w = torch.zeros((co, S, ci, S, K), dtype=torch.float32, device=device)
        self.b = torch.zeros((co, S), dtype=torch.float32, device=device)
        self.dw = torch.empty_like(self.w)
        self.db = torch.empty_like(self.b)
        self.ws_f = self.geom.workspace_size(V, ci, co, self.code, False)
        self.ws_b = self.geom.workspace_size(V, ci, co, self.code, True)
        self._ws = torch.empty(max(self.ws_f, self.ws_b) + 256, dtype=torch.uint8, device=device)
        self.ws = (self._ws.data_ptr() + 255) // 256 * 256
        self.lib = L.get()
        # fused LSC forward + SH2Signal when asked for and the kernel takes the sizes (c_out is
        # then never written: c_out_buf stays unused).  Off by default: on the 3 x 90-direction,
        # 16 -> 64-channel workload the two unfused calls take 1.67 ms against 1.70 ms fused,
        # since the fused tile (four 48-row channel slots, N = 192) keeps the tensor pipe less
        # busy than the forward GEMM's N = 256 tile.
        self.fused = bool(fused) and layers.lsc_forward_sh2signal_supported(self.geom, V, ci, co, dtype)
        self.calls = self.CALLS_FUSED if self.fused else self.CALLS

    @staticmethod
    def row_counts(cfg: ChainConfig, basis, basis_in) -> dict:
        """Feature rows of the chain's activations: signals (channels x directions) and SH
        (shells x channels x coefficients), input and output side."""
        S, nd = basis.n_shells, basis.n_dirs
        return dict(s_in=cfg.c_in * nd, c_in=S * cfg.c_in * basis_in.n_coef, c_out=S * cfg.c_out * basis.n_coef,
                    s_out=cfg.c_out * nd)

    def set_inputs(self, s_in: torch.Tensor, ds_out: torch.Tensor, w: torch.Tensor, b: torch.Tensor):
        self.s_in.copy_(s_in)
        self.ds_out.copy_(ds_out)
        self.w.copy_(w)
        self.b.copy_(b)

    def step(self, stream: int | None = None, events=None):
        """One forward + backward pass.  ``events``: optional list of len(self.calls) + 1 CUDA
        events recorded between the calls (per-call timing on the launch stream)."""
        lib, cfg, V = self.lib, self.cfg, self.cfg.n_vox
        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        bh, gh, t, ci, co, ws = self.basis.handle, self.geom.handle, self.code, cfg.c_in, cfg.c_out, self.ws
        bih = self.basis_in.handle
        rec = (lambda i: events[i].record()) if events is not None else (lambda i: None)
        rec(0)
        L.check(lib.delimit_signal2sh(bih, self.s_in.data_ptr(), self.c_in_buf.data_ptr(), V, ci, self.s_in.stride(0),
                                      self.c_in_buf.stride(0), t, t, st), "delimit_signal2sh")
        n = 1
        rec(n)
        if self.fused:
            L.check(lib.delimit_lsc_forward_sh2signal(gh, self.c_in_buf.data_ptr(), self.w.data_ptr(),
                                                      self.b.data_ptr(), self.s_out.data_ptr(), V, ci, co,
                                                      self.c_in_buf.stride(0), self.s_out.stride(0), t, 0, ws,
                                                      self.ws_b, st), "delimit_lsc_forward_sh2signal")
        else:
            L.check(lib.delimit_lsc_forward(gh, self.c_in_buf.data_ptr(), self.w.data_ptr(), self.b.data_ptr(),
                                            self.c_out_buf.data_ptr(), V, ci, co, self.c_in_buf.stride(0),
                                            self.c_out_buf.stride(0), t, 0, ws, self.ws_b, st), "delimit_lsc_forward")
            n += 1
            rec(n)
            L.check(lib.delimit_sh2signal(bh, self.c_out_buf.data_ptr(), self.s_out.data_ptr(), V, co,
                                          self.c_out_buf.stride(0), self.s_out.stride(0), t, t, st),
                    "delimit_sh2signal")
        n += 1
        rec(n)
        L.check(lib.delimit_sh2signal_backward(bh, self.ds_out.data_ptr(), self.dc_out.data_ptr(), V, co,
                                               self.ds_out.stride(0), self.dc_out.stride(0), t, t, st),
                "delimit_sh2signal_backward")
        n += 1
        rec(n)
        L.check(lib.delimit_lsc_backward(gh, self.c_in_buf.data_ptr(), self.w.data_ptr(), self.dc_out.data_ptr(),
                                         self.dc_in.data_ptr(), self.dw.data_ptr(), self.db.data_ptr(), V, ci, co,
                                         self.c_in_buf.stride(0), self.dc_out.stride(0), t, L.OPERATOR_READY, ws,
                                         self.ws_b, st),
                "delimit_lsc_backward")
        n += 1
        rec(n)
        L.check(lib.delimit_signal2sh_backward(bih, self.dc_in.data_ptr(), self.ds_in.data_ptr(), V, ci,
                                               self.dc_in.stride(0), self.ds_in.stride(0), t, t, st),
                "delimit_signal2sh_backward")
        n += 1
        rec(n)

    # algorithmic work per step (used for roofline figures)
    def _pairs(self) -> int:
        S, w = self.basis.n_shells, self.cfg.window
        return int(sum(abs(s - p) <= 1 if w == "adjacent" else (s == p if w == "same" else True)
                       for s in range(S) for p in range(S)))

    def flops(self, per_call: bool = True) -> dict:
        """Algorithmic FLOPs per call (per_call=False: the six steps of the unfused chain)."""
        cfg, b = self.cfg, self.basis
        V, N, N_in, ci, co, K = cfg.n_vox, b.n_coef, self.basis_in.n_coef, cfg.c_in, cfg.c_out, self.geom.K
        pairs = self._pairs()
        lsc_gemm = 2.0 * pairs * (co * N) * (ci * N_in) * V  # one of fwd / dgrad / wgrad
        build_w = 2.0 * pairs * co * ci * N * N_in * K
        s2sh = 2.0 * ci * b.n_dirs * N_in * V
        sh2s = 2.0 * co * b.n_dirs * N * V
        out = dict(signal2sh=s2sh, lsc_forward=lsc_gemm + build_w, sh2signal=sh2s, sh2signal_backward=sh2s,
                   lsc_backward=2 * lsc_gemm + build_w + 2.0 * pairs * co * ci * N * N * K, signal2sh_backward=s2sh)
        if self.fused and per_call:
            out["lsc_forward_sh2signal"] = out.pop("lsc_forward") + out.pop("sh2signal")
        return out

    def kernel_work(self) -> dict:
        """Algorithmic work per launch of each traced kernel group: (flops, compulsory HBM bytes)."""
        cfg, b = self.cfg, self.basis
        V, N, N_in, ci, co, K = cfg.n_vox, b.n_coef, self.basis_in.n_coef, cfg.c_in, cfg.c_out, self.geom.K
        e = 2 if self.dtype == torch.bfloat16 else 4
        pairs = self._pairs()
        r = self.rows
        gemm = 2.0 * pairs * (co * N) * (ci * N_in) * V
        build = 2.0 * pairs * co * ci * N * N_in * K
        wbytes = 2.0 * e * r["c_out"] * r["c_in"]
        fl = self.flops(per_call=False)
        by = self.bytes(per_call=False)
        out = {
            "lsc_fwd_gemm": (gemm, e * V * (r["c_in"] + r["c_out"])),
            "lsc_dgrad_gemm": (gemm, e * V * (r["c_out"] + r["c_in"])),
            "lsc_wgrad_gemm": (gemm, e * V * (r["c_out"] + r["c_in"])),
            "lsc_build_w": (build, wbytes),
            "lsc_build_w_tc": (build, wbytes),
            "lsc_reduce_dw": (build, 4.0 * r["c_out"] * r["c_in"]),
            "lsc_rowsum": (1.0 * r["c_out"] * V, e * V * r["c_out"]),
            "signal2sh_tc": (fl["signal2sh"], by["signal2sh"]),
            "sh2signal_tc": (fl["sh2signal"], by["sh2signal"]),
            "sh2signal_bwd_tc": (fl["sh2signal_backward"], by["sh2signal_backward"]),
            "signal2sh_bwd_tc": (fl["signal2sh_backward"], by["signal2sh_backward"]),
            "split_bf16x3": (0.0, 0.0),
            # fused LSC forward + SH2Signal: both products, the LSC input read and the signal written
            "lsc_fwd_sh2signal": (gemm + 2.0 * co * b.n_dirs * N * V, e * V * (r["c_in"] + r["s_out"])),
        }
        # FP32 activations: the same algorithmic work through the split-operand kernels
        for k in ("lsc_fwd_gemm", "lsc_dgrad_gemm", "lsc_wgrad_gemm", "signal2sh_tc", "sh2signal_tc",
                  "sh2signal_bwd_tc", "signal2sh_bwd_tc"):
            out[k + "_f32"] = out[k]
        return out

    def bytes(self, per_call: bool = True) -> dict:
        """Compulsory HBM bytes per call (activations read + written once; per_call=False: the
        six steps of the unfused chain)."""
        e = 2 if self.dtype == torch.bfloat16 else 4
        V, r = self.cfg.n_vox, self.rows
        out = dict(signal2sh=e * V * (r["s_in"] + r["c_in"]), lsc_forward=e * V * (r["c_in"] + r["c_out"]),
                   sh2signal=e * V * (r["c_out"] + r["s_out"]), sh2signal_backward=e * V * (r["s_out"] + r["c_out"]),
                   lsc_backward=e * V * (r["c_out"] + 2 * r["c_in"]),
                   signal2sh_backward=e * V * (r["c_in"] + r["s_in"]))
        if self.fused and per_call:
            out.pop("lsc_forward"), out.pop("sh2signal")
            out["lsc_forward_sh2signal"] = e * V * (r["c_in"] + r["s_out"])
        return out


class HostPipeline:
    """Runs the chain on inputs in pinned host memory and returns every step's outputs
    to pinned host memory, overlapping the copies with the compute.

    Two Chain instances (same tables, separate buffers) alternate between steps.
    Stream ``h2d`` copies step i's inputs, ``comp`` runs step i, ``d2h`` copies its
    outputs back; events order the three so that a chain's buffers are refilled only
    after its previous step's compute and copy-back are done.
    """

    def __init__(self, chains):
        assert len(chains) == 2
        self.chains = chains
        self.h2d, self.comp, self.d2h = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev = lambda: torch.cuda.Event()  # noqa: E731
        self.in_ready = [ev(), ev()]
        self.comp_done = [ev(), ev()]
        self.out_done = [ev(), ev()]
        self.started = [False, False]

    @staticmethod
    def host_buffers(chain, outputs=("dw", "db")):
        """Pinned host buffers for the step's inputs and for the outputs read back each
        step (default: the weight and bias gradients, the step's result for a weight
        update; add "s_out", "ds_in" to bring the activation outputs back too)."""
        pin = lambda t: torch.empty(t.shape, dtype=t.dtype, pin_memory=True)  # noqa: E731
        return {"s_in": pin(chain.s_in), "ds_out": pin(chain.ds_out)}, {k: pin(getattr(chain, k)) for k in outputs}

    def step(self, i: int, host_in: dict, host_out: dict):
        j = i % 2
        ch = self.chains[j]
        with torch.cuda.stream(self.h2d):
            if self.started[j]:
                self.h2d.wait_event(self.comp_done[j])  # the previous step on this chain has read its inputs
            ch.s_in.copy_(host_in["s_in"], non_blocking=True)
            ch.ds_out.copy_(host_in["ds_out"], non_blocking=True)
            self.in_ready[j].record(self.h2d)
        with torch.cuda.stream(self.comp):
            self.comp.wait_event(self.in_ready[j])
            if self.started[j]:
                self.comp.wait_event(self.out_done[j])  # outputs of the previous step on this chain are copied out
            ch.step(stream=self.comp.cuda_stream)
            self.comp_done[j].record(self.comp)
        with torch.cuda.stream(self.d2h):
            self.d2h.wait_event(self.comp_done[j])
            for k, h in host_out.items():
                h.copy_(getattr(ch, k), non_blocking=True)
            self.out_done[j].record(self.d2h)
        self.started[j] = True

    def synchronize(self):
        for s in (self.h2d, self.comp, self.d2h):
            s.synchronize()
