"""Whole-volume inference with per-subject gradient tables.

Each synthetic subject is a 145 x 174 x 145 volume of a 30-direction b=1000
acquisition inside an ellipsoid brain mask (about 900,000 voxels), with its own
gradient table: the base 3 x 90 table rotated by a seeded rotation of at most
5 deg plus per-direction jitter of at most 2 deg (the distorted gradient
directions the paper names as the reason for a uniform SH representation,
Sec. 1).  Every subject gets its own FP64 pseudo-inverses and LSC geometries;
the trained network's weights are shared.  The acquisition is stored raw: the
normalised signal times a smooth S0 field (b = 0 image, with noise), so the
normalisation the paper asks for before fitting (Sec. 2.2) happens on the device.
For all subjects, in one launch sequence: mask compaction (table T5), Signal2SH
of the masked voxels with the division by b0 fused into its load (no separate
gather or normalisation pass), the rest of the network in BF16, scatter of the
dense 270-direction prediction into the output volume.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import _lib as L
from . import layers, synth
from .net import NetConfig, SphericalNet, tables

SHAPE = (145, 174, 145)


class Subject:
    def __init__(self, idx: int, cfg: NetConfig, state: dict, shape=SHAPE, mask_voxels: int = 900_000,
                 seed: int = 1808):
        base_dirs, bvals, sel = tables(cfg)
        self.idx, self.cfg = idx, cfg
        self.dirs = synth.perturbed_table(base_dirs, math.radians(5.0), math.radians(2.0), seed, sub=idx)
        self.bvals, self.sel = bvals, sel
        self.mask = synth.ellipsoid_mask(shape, mask_voxels, seed=seed, sub=idx)
        self.n = int(np.prod(shape))
        t0 = time.perf_counter()
        self.net = SphericalNet(cfg, self.dirs[sel], self.dirs, bvals).cuda()
        self.net.load_state_dict(state)
        self.table_seconds = time.perf_counter() - t0
        self.net.eval()
        # the acquisition: noisy 30-direction signal inside the mask, zero outside, times S0
        n_mask = int(self.mask.sum())
        sig = synth.fibre_signal_torch(self.dirs[sel], np.full(len(sel), 1000.0), n_mask, seed=seed + 7, sub=idx,
                                       max_fibres=3, snr=(15.0, 40.0))
        midx = torch.from_numpy(np.flatnonzero(self.mask.reshape(-1))).cuda()
        self.b0 = self.s0_field(shape, seed, idx)  # float32 [n]
        self.volume = layers.empty_act(len(sel), self.n, torch.bfloat16)
        self.volume.zero_()
        self.volume[:, midx] = (sig * self.b0[midx]).to(torch.bfloat16)
        self.mask_dev = torch.from_numpy(self.mask.reshape(-1).astype(np.uint8)).cuda()
        self.midx = midx
        self._seed = seed

    def clean_signal(self) -> torch.Tensor:
        """The noise-free dense signal [270, mask voxels] of this subject's masked voxels on its
        own 3 x 90 table: the same fibres as the acquisition (the generator draws the fibres
        before the directions and the noise)."""
        _, clean = synth.fibre_signal_torch(self.dirs, self.bvals, int(self.midx.numel()), seed=self._seed + 7,
                                            sub=self.idx, max_fibres=3, snr=(15.0, 40.0), return_clean=True)
        return clean

    @staticmethod
    def s0_field(shape, seed, sub):
        """A smooth positive S0 (b = 0) image with 1 % noise, float32 on the device."""
        g = torch.Generator(device="cuda")
        g.manual_seed(seed * 1000 + sub)
        axes = [torch.linspace(-1.0, 1.0, n, device="cuda") for n in shape]
        zz, yy, xx = torch.meshgrid(*axes, indexing="ij")
        field = 1000.0 * (1.0 + 0.3 * torch.cos(2.0 * zz) * torch.cos(1.5 * yy) - 0.2 * xx * xx)
        noise = 1.0 + 0.01 * torch.randn(field.shape, generator=g, device="cuda")
        return (field * noise).reshape(-1).float().contiguous()


def run(subjects, chunk: int = 1 << 18):
    """Infer every subject in one launch sequence; returns (outputs, seconds, voxels)."""
    lib = L.get()
    st = torch.cuda.current_stream().cuda_stream
    n_dirs = subjects[0].dirs.shape[0]
    outs, idxs, cnts = [], [], []
    for sb in subjects:
        idx = torch.empty(sb.n, dtype=torch.int64, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        ws_n = lib.delimit_mask_compact_workspace_size(sb.n)
        ws = torch.empty(ws_n, dtype=torch.uint8, device="cuda")
        idxs.append((idx, cnt, ws, ws_n))
        out = layers.empty_act(n_dirs, sb.n, torch.bfloat16)
        out.zero_()
        outs.append(out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # mask compaction for all subjects first: the voxel counts size the gathers
    e0.record()
    for sb, (idx, cnt, ws, ws_n) in zip(subjects, idxs):
        L.check(lib.delimit_mask_compact(sb.mask_dev.data_ptr(), sb.n, idx.data_ptr(), cnt.data_ptr(), ws.data_ptr(),
                                         ws_n, st), "delimit_mask_compact")
    cnts = [int(c.item()) for (_, c, _, _) in idxs]  # one host read of the counts
    total = 0
    with torch.no_grad():
        for sb, (idx, _, _, _), k, out in zip(subjects, idxs, cnts, outs):
            total += k
            for v0 in range(0, k, chunk):
                m = min(chunk, k - v0)
                # Signal2SH of the chunk's masked voxels, divided by b0 in the load
                h = layers.signal2sh_gather(sb.net.s2sh.basis, sb.volume, idx[v0:], m, b0=sb.b0, channels=1,
                                            out_dtype=torch.bfloat16)
                y = sb.net.forward_sh(h)
                L.check(lib.delimit_scatter_voxels(y.data_ptr(), y.stride(0), n_dirs, idx[v0:].data_ptr(), m,
                                                   out.data_ptr(), out.stride(0), sb.n, L.BF16, st),
                        "delimit_scatter_voxels")
    e1.record()
    torch.cuda.synchronize()
    # outside the timed region: a kernel that gave up (or a gather index out of range)
    # leaves partial outputs, so the run fails here instead of returning them
    L.check_device_error("volume inference")
    return outs, e0.elapsed_time(e1) * 1e-3, total


@torch.no_grad()
def evaluate(subjects, outs) -> dict:
    """Relative L2 error, over every subject's masked voxels, of the network's dense 3 x 90
    prediction and of the SH least-squares fallback (order 8 on the 30 inputs, each subject's
    own table, the same b0-normalised input) against the noise-free signal."""
    from .net import Fallback
    num_net = num_fb = den = 0.0
    for sb, out in zip(subjects, outs):
        clean = sb.clean_signal()
        pred = out[:, sb.midx].float()
        x = (sb.volume[:, sb.midx].float() / sb.b0[sb.midx][None, :]).contiguous()
        fb = Fallback(sb.cfg, sb.dirs[sb.sel], sb.dirs, sb.bvals)(x)
        num_net += float(torch.sum((pred - clean) ** 2))
        num_fb += float(torch.sum((fb - clean) ** 2))
        den += float(torch.sum(clean ** 2))
    L.check_device_error("volume evaluation")
    return {"rel_l2_net": math.sqrt(num_net / den), "rel_l2_fallback": math.sqrt(num_fb / den),
            "against": "noise-free 3 x 90 signal inside every mask"}


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Whole-volume inference with per-subject gradient tables")
    ap.add_argument("--model", help="state saved by paper_1808_01517_gb300.net --save")
    ap.add_argument("--random-init", action="store_true",
                    help="seeded untrained weights (throughput only; the prediction is meaningless)")
    ap.add_argument("--subjects", type=int, default=16)
    ap.add_argument("--mask-voxels", type=int, default=900_000)
    args = ap.parse_args()
    if args.random_init:
        from .net import tables
        cfg = NetConfig()
        d, b, sel = tables(cfg)
        ck = {"state": SphericalNet(cfg, d[sel], d, b).state_dict()}
    elif args.model:
        ck = torch.load(args.model, map_location="cuda")
        cfg = NetConfig(**{k: (tuple(v) if isinstance(v, list) else v) for k, v in ck["cfg"].items()})
    else:
        ap.error("give --model or --random-init")
    t0 = time.perf_counter()
    subs = [Subject(i, cfg, ck["state"], mask_voxels=args.mask_voxels) for i in range(args.subjects)]
    setup = time.perf_counter() - t0
    outs, secs, vox = run(subs)
    # check: prediction inside the mask is finite, outside stays zero, b=1000 values plausible
    o = outs[0].float()
    m = torch.from_numpy(subs[0].mask.reshape(-1)).cuda()
    res = {"subjects": len(subs), "voxels": vox, "seconds": secs, "voxels_per_s": vox / secs,
           "weights": "random-init" if args.random_init else args.model,
           "table_seconds_total": sum(s.table_seconds for s in subs), "setup_seconds": setup,
           "finite": bool(torch.isfinite(o[:, m]).all()), "outside_zero": bool((o[:, ~m] == 0).all()),
           "mean_b1000_inside": float(o[:90, m].mean()), "device_error_word": "clean after the run"}
    if not args.random_init:
        res["accuracy"] = evaluate(subs, outs)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
