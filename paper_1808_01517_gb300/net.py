"""A small LSC network that predicts a dense multi-shell signal from a sparse
single-shell acquisition, built from the library's layers (the use the paper
motivates for the LSC in Sec. 1 and 2.3: gradient-neighbourhood information
and multi-shell prediction inside a network).

Architecture (reading of the learned-part configuration):
  Signal2SH(30 b=1000 directions, order 4, lambda 0.006)          -> 15 coefficients
  LSC(1 -> 64 channels, 1 input shell -> 3 output shells, order 4 -> 8,
      sampled on the 3 x 90 target directions, all input shells)   -> 3 x 64 x 45
  LeakyReLU(0.1) on the SH coefficients
  LSC(64 -> 64, adjacent shells) + LeakyReLU, twice
  LSC(64 -> 1, adjacent shells)                                    -> 3 x 45
  SH2Signal onto each shell's 90 target directions                -> 270 values
All LSCs use radius 25 deg with 4 rings x 12 sectors.  Activations are BF16,
master weights FP32 (torch Adam).  The comparison is plain SH least-squares
interpolation: an order-8 fit of the 30 input values (lambda 0.006),
evaluated on the 90 b=1000 targets and extrapolated to b = 2000, 3000 by
S_b = S_1000^(b/1000).
"""
from __future__ import annotations

import math
import os
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L
from . import layers, synth


@dataclass
class NetConfig:
    hidden: int = 64
    n_lsc: int = 4
    order_in: int = 4
    order: int = 8
    lam_in: float = 0.006
    lam: float = 0.006
    radius_deg: float = 25.0
    rings: int = 4
    sectors: int = 12
    slope: float = 0.1
    n_in_dirs: int = 30
    dirs_per_shell: tuple = (90, 90, 90)
    bvals: tuple = (1000, 2000, 3000)
    seed: int = 1808


def tables(cfg: NetConfig):
    """Target table (3 x 90, shell-grouped) and the input subset (30 of the b=1000 directions)."""
    dirs, bvals = synth.multishell_table(list(cfg.dirs_per_shell), list(cfg.bvals), seed=cfg.seed)
    sel = np.sort(synth.rng(cfg.seed, "subset", 7).choice(cfg.dirs_per_shell[0], cfg.n_in_dirs, replace=False))
    return dirs, bvals, sel


class SphericalNet(torch.nn.Module):
    def __init__(self, cfg: NetConfig, in_dirs: np.ndarray, target_dirs: np.ndarray, target_bvals: np.ndarray,
                 dtype=torch.bfloat16):
        super().__init__()
        self.cfg, self.dtype = cfg, dtype
        S = len(cfg.dirs_per_shell)
        rad = math.radians(cfg.radius_deg)
        ks = [cfg.sectors] * cfg.rings
        self.s2sh = layers.Signal2SH(cfg.order_in, in_dirs, cfg.lam_in, bvals=np.full(len(in_dirs), 1000.0))
        self.lscs = torch.nn.ModuleList()
        chans = [1] + [cfg.hidden] * (cfg.n_lsc - 1) + [1]
        for i in range(cfg.n_lsc):
            first = i == 0
            lsc = layers.LocalSphericalConvolution(
                shells_in=1 if first else S, shells_out=S, sampled_gradients=target_dirs,
                sh_order_in=cfg.order_in if first else cfg.order, sh_order_out=cfg.order, kernel_sizes=ks,
                lb_lambda=cfg.lam, angular_distance=rad, bvals=target_bvals, channels_in=chans[i],
                channels_out=chans[i + 1], window="all" if first else "adjacent")
            K = lsc.geom.K
            fan = chans[i] * (1 if first else 3) * K
            gain = math.sqrt(2.0) if i < cfg.n_lsc - 1 else 1.0
            with torch.no_grad():
                g = torch.Generator().manual_seed(cfg.seed + 17 * i)
                lsc.weight.copy_(torch.randn(lsc.weight.shape, generator=g) * (gain / math.sqrt(fan)))
                # weights outside the shell window are unused: keep them zero
                if not first:
                    m = torch.zeros(S, S, dtype=torch.bool)
                    for s in range(S):
                        m[s] = torch.from_numpy(lsc.geom.tables(s)["window"]).bool()
                    lsc.weight.mul_(m[None, :, None, :, None].float())
            self.lscs.append(lsc)
        self.act = layers.LeakyReLU(cfg.slope)
        self.sh2s = layers.SH2Signal(cfg.order, target_dirs, bvals=target_bvals)

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """x [n_in_dirs, V] (b0-normalised) -> [270, V] in the target table's row order."""
        return self.forward_sh(self.s2sh(x.to(self.dtype)))

    def forward_sh(self, h: torch.Tensor) -> torch.Tensor:
        """From the input's SH coefficients (the Signal2SH output, e.g. of a gathered,
        b0-normalised load) to the [270, V] prediction."""
        for i, lsc in enumerate(self.lscs):
            h = lsc(h)
            if i < len(self.lscs) - 1:
                h = self.act(h)
        return self.sh2s(h)


class Fallback:
    """Order-8 SH least squares on the 30 inputs, mono-exponential extrapolation to higher b."""

    def __init__(self, cfg: NetConfig, in_dirs, target_dirs, target_bvals):
        self.cfg = cfg
        m0 = cfg.dirs_per_shell[0]
        self.fit = layers.Signal2SH(cfg.order, in_dirs, cfg.lam, bvals=np.full(len(in_dirs), 1000.0))
        self.eval1000 = layers.SH2Signal(cfg.order, target_dirs[:m0], bvals=np.full(m0, 1000.0))
        self.ratios = [b / cfg.bvals[0] for b in cfg.bvals]

    @torch.no_grad()
    def __call__(self, x: torch.Tensor) -> torch.Tensor:
        s1 = self.eval1000(self.fit(x.float().contiguous()))  # [90, V] fp32
        s1 = s1.clamp_min(1e-4)
        return torch.cat([s1 ** r for r in self.ratios], 0)


@dataclass
class Data:
    x: torch.Tensor       # [30, N] noisy input
    y: torch.Tensor       # [270, N] noisy dense target
    clean: torch.Tensor   # [270, N] noise-free dense signal


def make_data(cfg: NetConfig, n: int, seed: int, dtype=torch.bfloat16, chunk: int = 1 << 20) -> Data:
    """Seeded fibre-model voxels (1-3 fibres, SNR 15-40) drawn on the device."""
    dirs, bvals, sel = tables(cfg)
    xs, ys, cs = [], [], []
    for i, v0 in enumerate(range(0, n, chunk)):
        m = min(chunk, n - v0)
        noisy, clean = synth.fibre_signal_torch(dirs, bvals, m, seed=seed, sub=i, max_fibres=3, min_fibres=1,
                                                snr=(15.0, 40.0), return_clean=True)
        xs.append(noisy[torch.as_tensor(sel, device=noisy.device)].to(dtype))
        ys.append(noisy.to(dtype))
        cs.append(clean.to(dtype))
    return Data(torch.cat(xs, 1), torch.cat(ys, 1), torch.cat(cs, 1))


def rel_l2(pred: torch.Tensor, ref: torch.Tensor) -> float:
    p, r = pred.float(), ref.float()
    return float(torch.linalg.vector_norm(p - r) / torch.linalg.vector_norm(r))


@dataclass
class TrainLog:
    losses: list = field(default_factory=list)
    seconds: float = 0.0
    steps: int = 0
    batch: int = 0
    device_error_checks: int = 0  # clean reads of the device error word during the run


def save_checkpoint(path: str, net: torch.nn.Module, opt, sched, gen: torch.Generator, next_step: int):
    """What a resumed run needs to continue bit for bit: the weights, the optimizer's
    moments, the learning-rate schedule, the batch sampler's generator state and the
    next step.  Written to a temporary file and renamed, so a crash mid-write leaves the
    previous checkpoint intact."""
    state = {"net": net.state_dict(), "opt": opt.state_dict(), "sched": sched.state_dict(),
             "gen": gen.get_state(), "next_step": int(next_step)}
    tmp = path + ".tmp"
    torch.save(state, tmp)
    os.replace(tmp, path)


def load_checkpoint(path: str, net: torch.nn.Module, opt, sched, gen: torch.Generator) -> int:
    """Restores what save_checkpoint wrote into freshly built objects; returns the next step."""
    state = torch.load(path, map_location="cpu", weights_only=True)
    net.load_state_dict(state["net"])
    opt.load_state_dict(state["opt"])
    sched.load_state_dict(state["sched"])
    gen.set_state(state["gen"])
    return int(state["next_step"])


def train(net: SphericalNet, data: Data, steps: int, batch: int, lr: float = 2e-3, seed: int = 0,
          log_every: int = 100, checkpoint: str = "", checkpoint_every: int = 0, resume: str = "") -> TrainLog:
    """Adam with a cosine schedule on random batches of ``data``.  checkpoint /
    checkpoint_every: write a checkpoint every that many steps; resume: continue from
    one (the same steps, batch and lr as the run that wrote it)."""
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=max(1, steps))
    gen = torch.Generator(device=data.x.device)
    gen.manual_seed(seed)
    start = load_checkpoint(resume, net, opt, sched, gen) if resume else 0
    n = data.x.shape[1]
    log = TrainLog(steps=steps - start, batch=batch)  # the steps this call runs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for step in range(start, steps):
        idx = torch.randint(0, n, (batch,), generator=gen, device=data.x.device)
        pred = net(data.x[:, idx])
        loss = torch.mean((pred.float() - data.y[:, idx].float()) ** 2)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        sched.step()
        if step % log_every == 0 or step == steps - 1:
            log.losses.append((step, float(loss.detach())))
            # the loss read has synchronised already; a kernel that gave up leaves partial
            # outputs, so training stops here instead of going on with them
            L.check_device_error(f"training step {step}")
            log.device_error_checks += 1
        if checkpoint and checkpoint_every > 0 and (step + 1) % checkpoint_every == 0:
            save_checkpoint(checkpoint, net, opt, sched, gen, step + 1)
    torch.cuda.synchronize()
    log.seconds = time.perf_counter() - t0
    L.check_device_error("end of training")
    log.device_error_checks += 1
    return log


@torch.no_grad()
def predict(model, x: torch.Tensor, chunk: int = 1 << 18) -> torch.Tensor:
    outs = [model(x[:, i:i + chunk]).float() for i in range(0, x.shape[1], chunk)]
    return torch.cat(outs, 1)


def evaluate(net: SphericalNet, fb: Fallback, data: Data) -> dict:
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p_net = predict(net, data.x)
    torch.cuda.synchronize()
    t_net = time.perf_counter() - t0
    p_fb = predict(fb, data.x)
    L.check_device_error("evaluation")
    m = net.cfg.dirs_per_shell[0]
    out = {"rel_l2_net": rel_l2(p_net, data.clean), "rel_l2_fallback": rel_l2(p_fb, data.clean),
           "voxels": int(data.x.shape[1]), "net_inference_voxels_per_s": data.x.shape[1] / t_net}
    for s, b in enumerate(net.cfg.bvals):
        sl = slice(s * m, (s + 1) * m)
        out[f"b{b}_net"] = rel_l2(p_net[sl], data.clean[sl])
        out[f"b{b}_fallback"] = rel_l2(p_fb[sl], data.clean[sl])
    return out


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Train the LSC network and compare it with SH least-squares interpolation")
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--train-voxels", type=int, default=10_000_000)
    ap.add_argument("--test-voxels", type=int, default=1_000_000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--save", default="")
    ap.add_argument("--checkpoint", default="", help="checkpoint file written during training")
    ap.add_argument("--checkpoint-every", type=int, default=0)
    ap.add_argument("--resume", default="", help="continue from this checkpoint")
    args = ap.parse_args()
    cfg = NetConfig()
    dirs, bvals, sel = tables(cfg)
    net = SphericalNet(cfg, dirs[sel], dirs, bvals).cuda()
    fb = Fallback(cfg, dirs[sel], dirs, bvals)
    tr = make_data(cfg, args.train_voxels, seed=cfg.seed)
    te = make_data(cfg, args.test_voxels, seed=cfg.seed + 1)
    log = train(net, tr, args.steps, args.batch, args.lr, checkpoint=args.checkpoint,
                checkpoint_every=args.checkpoint_every, resume=args.resume)
    res = evaluate(net, fb, te)
    res.update({"steps": args.steps, "batch": args.batch, "train_seconds": log.seconds,
                "train_voxels_per_s": log.steps * args.batch / max(log.seconds, 1e-9),
                "loss_first_last": [log.losses[0], log.losses[-1]] if log.losses else [],
                "device_error_word": f"clean at {log.device_error_checks} checks and after evaluation"})
    if args.save:
        torch.save({"state": net.state_dict(), "cfg": cfg.__dict__, "result": res}, args.save)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
