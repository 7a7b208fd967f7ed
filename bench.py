#!/usr/bin/env python3
"""Benchmark: voxels/s of Signal2SH -> LSC -> SH2Signal forward + backward.

Workload (one step = one pass of the whole path over one batch): 65,536 voxels,
3 shells x 90 directions (b = 1000/2000/3000), SH order 8 (3 x 45 coefficients,
lambda 0.006), LSC 16 -> 64 channels mixing adjacent shells, radius 25 deg,
4 rings x 12 sectors (K = 49); BF16 activations on the tensor cores with FP32
accumulation and FP32 master weights.  The FP32 path is measured beside it.
Inputs are seeded synthetic fibre-model signals (stick + zeppelin, SNR 20) and
Gaussian upstream gradients, larger than L2 (no flush needed).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 oracle
(the reference arm: plain numpy on the host cores) on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "voxels/s, Signal2SH->LSC->SH2Signal fwd+bwd, BF16 vs FP32 at stated error vs FP64 oracle"
UNIT = "voxels/s"

# DRAM traffic (read + write) of one launch at the 65,536-voxel workload, from the
# single-pass ncu capture of the bench command summarised in
# profiles/chain_65536vox_launch_list.md (the `dram__bytes_*` metrics); valid only
# while the kernel's sources hash to the value recorded with the capture (re-hashed
# only after host-side edits that leave the kernels' device code unchanged).
_GEMM = ("csrc/tc_gemm.cu", "csrc/tc_ptx.cuh"), "ab66a0cc8a65094a"
_TF = ("csrc/tc_transform.cu", "csrc/tc_ptx.cuh"), "03ad4be21121a183"
NCU_TRAFFIC = {
    "lsc_fwd_gemm": {"bytes": 1.523e9, "n_vox": 65536, "sources": _GEMM[0], "sha256_16": _GEMM[1]},
    "lsc_dgrad_gemm": {"bytes": 2.653e9, "n_vox": 65536, "sources": _GEMM[0], "sha256_16": _GEMM[1]},
    "lsc_wgrad_gemm": {"bytes": 3.270e9, "n_vox": 65536, "sources": _GEMM[0], "sha256_16": _GEMM[1]},
    "signal2sh_tc": {"bytes": 0.8136e9, "n_vox": 65536, "sources": _TF[0], "sha256_16": _TF[1]},
    "sh2signal_tc": {"bytes": 3.333e9, "n_vox": 65536, "sources": _TF[0], "sha256_16": _TF[1]},
    "sh2signal_bwd_tc": {"bytes": 3.358e9, "n_vox": 65536, "sources": _TF[0], "sha256_16": _TF[1]},
    "signal2sh_bwd_tc": {"bytes": 0.7846e9, "n_vox": 65536, "sources": _TF[0], "sha256_16": _TF[1]},
}


def ncu_traffic(kernel: str, n_vox: int):
    import hashlib
    rec = NCU_TRAFFIC.get(kernel)
    if rec is None:
        return None
    h = hashlib.sha256()
    for rel in rec["sources"]:
        with open(os.path.join(HERE, "paper_1808_01517_gb300", rel), "rb") as f:
            h.update(f.read())
    if h.hexdigest()[:16] != rec["sha256_16"]:
        return None  # the kernel changed since the counters were taken
    if n_vox != rec["n_vox"]:
        return None  # counters were taken at another workload size
    return rec["bytes"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-vox", type=int, default=65536)
    ap.add_argument("--fp32-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extras", action="store_true", help="skip fp32 / e2e / cpu / transform legs (profiling runs)")
    ap.add_argument("--fused", action="store_true",
                    help="time the chain with the LSC forward and SH2Signal fused into one kernel")
    ap.add_argument("--precision", default="bf16", choices=["bf16", "f32"],
                    help="activations of the timed chain (f32: the split-operand tensor-core path)")
    ap.add_argument("--learned-seconds", type=float, default=25.0,
                    help="training budget of the learned-network leg (0 skips it)")
    ap.add_argument("--transform-vox", type=int, default=1 << 20,
                    help="voxels of the stand-alone transform leg (one channel, 3 x 90 directions)")
    return ap.parse_args()


def workload_config(n_vox):
    from paper_1808_01517_gb300.chain import ChainConfig
    return ChainConfig(n_vox=n_vox)


def table(cfg):
    from paper_1808_01517_gb300 import synth
    return synth.multishell_table(list(cfg.dirs_per_shell), list(cfg.bvals), seed=cfg.seed)


# ---------------------------------------------------------------------------
# FP64 oracle chain (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
class OracleChain:
    def __init__(self, cfg, dirs, bvals):
        from oracle import lsc as olsc
        from oracle import sh as osh
        self.cfg = cfg
        self.ob = osh.SHBasisOracle(dirs, bvals, cfg.order, cfg.lam)
        self.ob_in = self.ob if cfg.l_in == cfg.order else osh.SHBasisOracle(dirs, bvals, cfg.l_in, cfg.lam)
        cls = olsc.LSCOracle if cfg.resample else olsc.LSCNeighbourOracle
        self.og = cls(self.ob, cfg.l_in, self.ob.n_shells, np.deg2rad(cfg.radius_deg), cfg.rings, cfg.sectors,
                      cfg.window)

    def step(self, sig, w, b, ds_out):
        """sig [V, Ci, dirs], ds_out [V, Co, dirs] -> (s_out, ds_in, dw, db)."""
        ob, og = self.ob, self.og
        c_in = self.ob_in.signal2sh(sig)
        s_out = ob.sh2signal(og.forward(c_in, w, b))
        dc_in, dw, db = og.backward(c_in, w, ob.sh2signal_backward(ds_out))
        return s_out, self.ob_in.signal2sh_backward(dc_in), dw, db


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var, "").strip().isdigit() and int(os.environ[var]) > 0:
            return int(os.environ[var])
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle_single_thread(steps=3, warm=1, timeout_s=120):
    """The reference arm (the FP64 oracle on 64-voxel samples) in a child interpreter with
    every BLAS / OpenMP pool held to one thread: the oracle's single-core rate."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", str(steps),
           "--warmup", str(warm)]
    try:
        r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=timeout_s)
        rec = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
        return {"value": rec["value"], "unit": rec["unit"], "cores": 1, "kind": "oracle",
                "sample": f"{steps} x 64 voxels of the same workload, FP64 numpy oracle, one thread"}
    except Exception as e:  # reported, not fatal: the GPU legs do not depend on it
        return {"unavailable": f"{type(e).__name__}: {str(e)[:200]}"}


def oracle_inputs(cfg, dirs, bvals, V, seed):
    from paper_1808_01517_gb300 import synth
    S = len(cfg.dirs_per_shell)
    sig = synth.fibre_signal(dirs, bvals, V * cfg.c_in, seed=seed).astype(np.float64)
    sig = sig.reshape(cfg.c_in, V, -1).transpose(1, 0, 2)
    K = 1 + cfg.rings * cfg.sectors
    w = synth.gaussian((cfg.c_out, S, cfg.c_in, S, K), 0.1, seed=seed)
    b = synth.gaussian((cfg.c_out, S), 0.1, seed=seed + 1)
    ds = synth.gaussian((V, cfg.c_out, dirs.shape[0]), 0.1, seed=seed, tag="grads")
    return sig, w, b, ds


def time_oracle(cfg, dirs, bvals, budget_s, chunk=64, max_vox=4096):
    """Voxels/s of the oracle chain on a bounded sample (chunks of `chunk` voxels until
    `budget_s` seconds of work or `max_vox` voxels)."""
    oc = OracleChain(cfg, dirs, bvals)
    done, t_work = 0, 0.0
    while t_work < budget_s and done < max_vox:
        sig, w, b, ds = oracle_inputs(cfg, dirs, bvals, chunk, seed=cfg.seed + done)
        t0 = time.perf_counter()
        oc.step(sig, w, b, ds)
        t_work += time.perf_counter() - t0
        done += chunk
    return done / t_work, done, t_work


def chain_inputs(cfg, dirs, bvals, dtype, rank=0):
    """Device-drawn fibre signals (library row order), Gaussian upstream gradients,
    N(0, 0.1) weights and biases; seeded per rank."""
    import torch
    from paper_1808_01517_gb300 import synth
    V, S = cfg.n_vox, len(cfg.dirs_per_shell)
    sig = synth.fibre_signal_torch(dirs, bvals, cfg.c_in * V, seed=cfg.seed + rank)  # [dirs, Ci*V]
    # library row order (s, c, i): per shell, channel-major blocks of that shell's directions
    s_rows = []
    off = 0
    for m in cfg.dirs_per_shell:
        s_rows.append(sig[off:off + m].reshape(m, cfg.c_in, V).permute(1, 0, 2).reshape(cfg.c_in * m, V))
        off += m
    s_in = torch.cat(s_rows, 0).to(dtype)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(cfg.seed * 31 + rank)
    ds_out = (0.1 * torch.randn((cfg.c_out * dirs.shape[0], V), generator=gen, device="cuda")).to(dtype)
    K = 1 + cfg.rings * cfg.sectors
    w = torch.from_numpy(synth.gaussian((cfg.c_out, S, cfg.c_in, S, K), 0.1, seed=cfg.seed)).float().cuda()
    b = torch.from_numpy(synth.gaussian((cfg.c_out, S), 0.1, seed=cfg.seed + 1)).float().cuda()
    return s_in, ds_out, w, b


def guarded(name, fn, *args, **kwargs):
    """Runs one optional leg of the bench.  A failure is printed to stderr and reported as
    {"unavailable": reason} in that leg's entry, so that the JSON line of the timed step is
    still printed."""
    try:
        return fn(*args, **kwargs)
    except Exception as e:  # noqa: BLE001 - any failure of an optional leg is reported, not raised
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"unavailable": f"{name}: {type(e).__name__}: {str(e)[:300]}"}


def time_tables(cfg, dirs, bvals, repeats=3):
    """Host FP64 table build (Sec. 2.2, 2.3; built once per gradient table, outside every timed
    step): the per-shell basis and regularised pseudo-inverse, then the LSC geometry (kernel
    points, basis at the kernel points, collapse matrices).  Host-only handles, so no device
    upload is timed; best of `repeats`."""
    from paper_1808_01517_gb300 import _lib as L
    best_b = best_g = float("inf")
    for _ in range(repeats):
        t0 = time.perf_counter()
        basis = L.SHBasis(dirs, bvals, cfg.order, cfg.lam, host_only=True)
        t1 = time.perf_counter()
        geom = L.LSCGeometry(basis, cfg.l_in, basis.n_shells, np.deg2rad(cfg.radius_deg), cfg.rings, cfg.sectors,
                             cfg.window, host_only=True, neighbours=not cfg.resample)
        t2 = time.perf_counter()
        best_b, best_g = min(best_b, t1 - t0), min(best_g, t2 - t1)
        del geom, basis
    return {"sh_basis_ms": 1e3 * best_b, "lsc_geometry_ms": 1e3 * best_g, "precision": "f64",
            "where": "host, one thread, host-only handles", "repeats": repeats}


def run_fp32_leg(ch, cfg, dirs, bvals, idx, steps, tensor_cores):
    """The chain with FP32 activations on the inputs of the BF16 chain `ch`: voxels/s,
    per-call times and error on sampled voxels against the FP64 oracle.  tensor_cores:
    the LSC GEMMs as three-part BF16 splits on the tensor cores, else CUDA-core FP32."""
    import torch
    from paper_1808_01517_gb300 import _lib as L
    from paper_1808_01517_gb300.chain import Chain
    L.set_tensor_cores(L.TC_REQUIRE if tensor_cores else L.TC_OFF)
    try:
        ch32 = Chain(cfg, dirs, bvals, torch.float32)
        ch32.s_in.copy_(ch.s_in.float())
        ch32.ds_out.copy_(ch.ds_out.float())
        ch32.w.copy_(ch.w)
        ch32.b.copy_(ch.b)
        ch32.step()
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(ch32.calls) + 1)] for _ in range(steps)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(steps):
            ch32.step(events=ev[k])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        per_call = {name: float(np.mean([ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(steps)]))
                    for i, name in enumerate(ch32.calls)}
        out = {"value": cfg.n_vox / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
               "gemms": "tensor cores (required), three-part BF16 splits, six part products, FP32 accumulation"
               if tensor_cores else "CUDA cores, FP32 FMA", "per_call_ms": per_call,
               "err_vs_oracle": sampled_errors(ch32, cfg, dirs, bvals, idx)}
        del ch32
    finally:
        L.set_tensor_cores(True)
    torch.cuda.empty_cache()
    return out


def run_learned_leg(seconds=25.0, batch=8192, n_train=2_000_000, n_test=262_144, subjects=2, max_steps=20000):
    """The learned part, time-bounded: the 4-LSC network at its trained widths (64 channels,
    3 x 90 targets from 30 b=1000 inputs, 4 x 12 kernels, BF16) trained with the library's
    kernels at batch 8,192 for about `seconds` on seeded fibre-model voxels (a checkpoint
    written at the end); held-out voxels against the SH least-squares fallback; then
    whole-volume inference of `subjects` synthetic 145 x 174 x 145 subjects (about 900,000
    mask voxels each, per-subject perturbed tables, b0 division fused into the gathered
    Signal2SH) with the weights of that checkpoint, against the noise-free signal."""
    import tempfile
    import torch
    from paper_1808_01517_gb300 import net as N
    from paper_1808_01517_gb300 import volume as VOL
    cfg = N.NetConfig()
    dirs, bvals, sel = N.tables(cfg)
    tr = N.make_data(cfg, n_train, seed=cfg.seed)
    te = N.make_data(cfg, n_test, seed=cfg.seed + 1)
    # steps that fit the time budget, from a short run of a throwaway network
    probe = N.SphericalNet(cfg, dirs[sel], dirs, bvals).cuda()
    N.train(probe, tr, 10, batch, seed=2)
    t_probe = N.train(probe, tr, 30, batch, seed=3).seconds / 30
    del probe
    steps = int(max(100, min(max_steps, seconds / max(t_probe, 1e-6))))
    net = N.SphericalNet(cfg, dirs[sel], dirs, bvals).cuda()
    fb = N.Fallback(cfg, dirs[sel], dirs, bvals)
    with tempfile.TemporaryDirectory() as tmp:
        ck_path = os.path.join(tmp, "net.pt")
        log = N.train(net, tr, steps, batch, checkpoint=ck_path, checkpoint_every=steps)
        held = N.evaluate(net, fb, te)
        state = torch.load(ck_path, map_location="cuda", weights_only=True)["net"]
    del net, tr, te
    torch.cuda.empty_cache()
    subs = [VOL.Subject(i, cfg, state) for i in range(subjects)]
    outs, secs, vox = VOL.run(subs)
    acc = VOL.evaluate(subs, outs)
    del subs, outs
    torch.cuda.empty_cache()
    return {"train": {"steps": steps, "batch": batch, "seconds": log.seconds,
                      "train_voxels_per_s": log.steps * batch / max(log.seconds, 1e-9),
                      "loss_first_last": [log.losses[0], log.losses[-1]], "train_voxels": n_train,
                      "device_error_checks": log.device_error_checks},
            "heldout": held,
            "volume": {"subjects": subjects, "voxels": vox, "seconds": secs, "voxels_per_s": vox / secs,
                       "weights": "the checkpoint written by this leg's training", **acc}}


def run_chain_leg(cfg, dirs, bvals, steps=10, warm=3, fused=False):
    """Another chain configuration at full size (BF16): voxels/s, per-call times and
    error on sampled voxels against the FP64 oracle.  fused=True: the LSC forward and
    SH2Signal as one kernel (c_out never stored)."""
    import torch
    from paper_1808_01517_gb300 import synth
    from paper_1808_01517_gb300.chain import Chain
    ch = Chain(cfg, dirs, bvals, torch.bfloat16, fused=fused)
    ch.set_inputs(*chain_inputs(cfg, dirs, bvals, torch.bfloat16))
    for _ in range(warm):
        ch.step()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(ch.calls) + 1)] for _ in range(steps)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(steps):
        ch.step(events=ev[k])
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    per_call = {name: float(np.mean([ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(steps)]))
                for i, name in enumerate(ch.calls)}
    fl = ch.flops()
    idx = synth.voxel_subset(cfg.n_vox, 32, seed=cfg.seed + 97)
    out = {"workload": cfg.name(), "fused_lsc_sh2signal": ch.fused, "value": cfg.n_vox / (ms * 1e-3), "unit": UNIT,
           "ms_per_step": ms,
           "steps": steps, "step_tflops": sum(fl.values()) / (ms * 1e-3) / 1e12,
           "lsc_forward_tflops": (fl["lsc_forward_sh2signal"] / (per_call["lsc_forward_sh2signal"] * 1e-3) if ch.fused
                                  else fl["lsc_forward"] / (per_call["lsc_forward"] * 1e-3)) / 1e12,
           "per_call_ms": per_call, "err_vs_oracle": sampled_errors(ch, cfg, dirs, bvals, idx)}
    del ch
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def reduce_max_ms(ms: float, dist=None, device="cpu") -> float:
    """Max over ranks of the per-rank timed milliseconds (the slowest rank sets the step)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_vox_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job voxels/s: every rank processes its own batch (weak scaling)."""
    return world * n_vox_per_rank / (ms_max * 1e-3)


# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = workload_config(args.n_vox)
    dirs, bvals = table(cfg)

    if args.impl == "reference":
        if rank != 0:
            return
        steps, warm = args.steps, args.warmup
        oc = OracleChain(cfg, dirs, bvals)
        chunk = 64
        sig, w, b, ds = oracle_inputs(cfg, dirs, bvals, chunk, seed=cfg.seed)
        for _ in range(warm):
            oc.step(sig, w, b, ds)
        t0 = time.perf_counter()
        for _ in range(steps):
            oc.step(sig, w, b, ds)
        dt = time.perf_counter() - t0
        v = chunk * steps / dt
        cores = blas_threads()
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": steps,
                "warmup": warm, "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": cfg.name(), "sample_voxels_per_step": chunk},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"{chunk} voxels per step of the same workload, FP64 numpy oracle"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    from paper_1808_01517_gb300 import _lib as L
    from paper_1808_01517_gb300 import synth
    from paper_1808_01517_gb300.chain import Chain

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    V = cfg.n_vox
    act = torch.float32 if args.precision == "f32" else torch.bfloat16
    ch = Chain(cfg, dirs, bvals, act, fused=args.fused)
    s_in, ds_out, w, b = chain_inputs(cfg, dirs, bvals, act, rank)
    ch.set_inputs(s_in, ds_out, w, b)
    del s_in, ds_out
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # the timed chain must run on the tensor cores: under TC_REQUIRE a call that has no
    # tensor-core kernel for its shape is refused instead of running on the CUDA cores
    L.set_tensor_cores(L.TC_REQUIRE)
    fallbacks0 = L.cuda_core_fallbacks()
    for _ in range(max(3, args.warmup)):
        ch.step()
    barrier()

    # ---- timed region ----
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(ch.calls) + 1)] for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = L.get().delimit_kernel_launches()
    L.trace_enable(True)
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    t_start.record()
    for k in range(K):
        ch.step(events=ev[k])
    t_stop.record()
    barrier()
    launches = L.get().delimit_kernel_launches() - launches0
    trace = L.trace_summary()
    L.trace_enable(False)
    L.set_tensor_cores(L.TC_PREFER)
    clk = clocks.stop()
    cuda_core_kernels = sorted(n for n in trace if "simt" in n)
    if cuda_core_kernels or L.cuda_core_fallbacks() != fallbacks0:
        raise RuntimeError(f"timed chain ran CUDA-core GEMM kernels: {cuda_core_kernels}")
    ms = reduce_max_ms(t_start.elapsed_time(t_stop) / K, dist, "cuda")
    value = job_throughput(V, world, ms)
    per_call = {name: float(np.mean([ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(K)]))
                for i, name in enumerate(ch.calls)}
    # each step alone, from the event before its first call to the one after its last
    step_ms = [ev[k][0].elapsed_time(ev[k][len(ch.calls)]) for k in range(K)]
    st, code = L.device_error(torch.cuda.current_stream().cuda_stream)
    if st != L.OK:
        raise RuntimeError(f"device error word set: {code:#x}")

    import json as _json
    peaks = {}
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            peaks = _json.load(f)
        peak_src = "measured"
    except Exception:
        peak_src = "fallback"
    tf_burst = float(peaks.get("bf16_tflops", 1900.0))
    tf_sust = float(peaks.get("bf16_tflops_sustained", 1700.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # the peak for the clock the step ran at: the burst figure (a GEMM timed alone at the
    # maximum clock) when the SM clock sampled during the timed region stayed at its
    # maximum, else the sustained figure (a GEMM loop held to the power cap)
    at_max = bool(clk.get("sm_mhz") and clk.get("sm_max_mhz") and clk["sm_mhz"] >= 0.97 * clk["sm_max_mhz"])
    tf_peak = tf_burst if at_max else tf_sust
    tf_name = "bf16_tflops (burst: SM clock at its maximum)" if at_max else "bf16_tflops_sustained (SM clock below max)"
    fl, by = ch.flops(), ch.bytes()
    per_call_roof = {n: {"ms": per_call[n], "tflops": fl[n] / (per_call[n] * 1e-3) / 1e12,
                         "gbs": by[n] / (per_call[n] * 1e-3) / 1e9} for n in per_call}
    # per kernel group, timed live on the launch stream (library trace events)
    work = ch.kernel_work()
    kernels = {}
    for name, rec in trace.items():
        avg = rec["ms"] / max(1, rec["n"])
        f, bb = work.get(name, (0.0, 0.0))
        kernels[name] = {"launches": rec["n"], "avg_ms": avg, "share": 0.0, "tflops": f / (avg * 1e-3) / 1e12,
                         "gbs": bb / (avg * 1e-3) / 1e9, "traffic": ncu_traffic(name, V)}
    tot = sum(v["avg_ms"] * v["launches"] for v in kernels.values()) or 1.0
    for v in kernels.values():
        v["share"] = v["avg_ms"] * v["launches"] / tot
    dom = max(kernels, key=lambda k: kernels[k]["avg_ms"] * kernels[k]["launches"])
    tensor_bound = "_gemm" in dom
    if tensor_bound and dom.endswith("_f32"):
        # six BF16 part products per FP32 product: the split path's ceiling is a sixth of BF16's
        roofline = {"bound": "tensor", "achieved": kernels[dom]["tflops"], "peak": tf_peak / 6, "unit": "TFLOP/s",
                    "frac": kernels[dom]["tflops"] / (tf_peak / 6),
                    "frac_of_sustained": kernels[dom]["tflops"] / (tf_sust / 6),
                    "peak_source": f"{peak_src} {tf_name} / 6 (six BF16 products per FP32 product)"}
    elif tensor_bound:
        roofline = {"bound": "tensor", "achieved": kernels[dom]["tflops"], "peak": tf_peak, "unit": "TFLOP/s",
                    "frac": kernels[dom]["tflops"] / tf_peak, "frac_of_sustained": kernels[dom]["tflops"] / tf_sust,
                    "peak_source": f"{peak_src} {tf_name}"}
    else:
        roofline = {"bound": "hbm", "achieved": kernels[dom]["gbs"], "peak": hbm, "unit": "GB/s",
                    "frac": kernels[dom]["gbs"] / hbm, "peak_source": f"{peak_src} hbm_gbs"}
    roofline.update({"traffic": ncu_traffic(dom, V), "kernel": dom, "kernel_avg_ms": kernels[dom]["avg_ms"],
                     "step_tflops": sum(fl.values()) / (ms * 1e-3) / 1e12})
    roofline["step_frac_of_tensor_peak"] = roofline["step_tflops"] / tf_peak

    extras = {}
    if rank == 0 and not args.no_extras and args.precision == "bf16":
        # every leg below is optional: a failure is reported in its own entry, not fatal
        # ---- accuracy on sampled voxels vs the FP64 oracle ----
        idx = synth.voxel_subset(V, 32, seed=cfg.seed + 99)
        extras["err_vs_oracle_bf16"] = guarded("err_vs_oracle_bf16", sampled_errors, ch, cfg, dirs, bvals, idx)
        # ---- FP32 path: tensor cores through three-part BF16 splits (default), CUDA cores ----
        extras["fp32"] = guarded("fp32", run_fp32_leg, ch, cfg, dirs, bvals, idx, max(3, args.fp32_steps), True)
        extras["fp32_cuda_cores"] = guarded("fp32_cuda_cores", run_fp32_leg, ch, cfg, dirs, bvals, idx,
                                            args.fp32_steps, False)
        # ---- end to end through host buffers ----
        extras["e2e"] = guarded("e2e", run_e2e, ch, args.e2e_steps)
        # ---- the same step with the LSC forward and SH2Signal fused into one kernel ----
        extras["fused"] = guarded("fused", run_chain_leg, cfg, dirs, bvals, fused=True)
        # ---- mixed SH orders (4 -> 8) with every input shell mixed into every output shell ----
        from dataclasses import replace
        extras["mixed_orders_all_shells"] = guarded("mixed_orders_all_shells", run_chain_leg,
                                                    replace(cfg, order_in=4, window="all"), dirs, bvals)
        extras["resampling_free"] = guarded("resampling_free", run_chain_leg, replace(cfg, resample=False), dirs,
                                            bvals)
        # ---- stand-alone transforms at 1,048,576 voxels (FP32 and BF16-in / FP32-out) ----
        tr = guarded("transforms", run_transforms, cfg, dirs, bvals, args.transform_vox, hbm)
        if "unavailable" not in tr:
            tr["cpu_baseline"] = guarded("transforms cpu_baseline", time_oracle_transforms, cfg, dirs, bvals)
        extras["transforms"] = tr
        # ---- FP64 table build on the host (once per gradient table) ----
        extras["tables"] = guarded("tables", time_tables, cfg, dirs, bvals)
        # ---- the learned part: short training, held-out accuracy, volume inference ----
        if args.learned_seconds > 0:
            extras["learned"] = guarded("learned", run_learned_leg, args.learned_seconds)

        # ---- oracle on the host cores ----
        def cpu_leg():
            vps, nv, tw = time_oracle(cfg, dirs, bvals, args.cpu_seconds)
            return {"value": vps, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                    "sample": f"{nv} voxels of the same workload in 64-voxel chunks, "
                              f"{tw:.1f} s of FP64 numpy oracle work"}
        extras["cpu_baseline"] = guarded("cpu_baseline", cpu_leg)
        extras["cpu_baseline_single_thread"] = time_oracle_single_thread()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": max(3, args.warmup), "ms_per_step": ms,
                "ms_per_step_median": float(np.median(step_ms)), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": {"workload": cfg.name(), "fused_lsc_sh2signal": ch.fused, "n_vox": V,
                           "shells": list(cfg.dirs_per_shell),
                           "sh_order": cfg.order, "c_in": cfg.c_in, "c_out": cfg.c_out, "kernel_points": ch.geom.K,
                           "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"},
                "roofline": roofline, "kernels": kernels, "per_call": per_call_roof, "clocks": clk,
                "gpu_launches": int(launches),
                "device": {"gpu": torch.cuda.get_device_name(local),
                           "sms": torch.cuda.get_device_properties(local).multi_processor_count,
                           "host_cores": os.cpu_count()}}
        line.update({k: v for k, v in extras.items() if k in ("e2e", "cpu_baseline")})
        line["fp32"] = extras.get("fp32")
        line["fp32_cuda_cores"] = extras.get("fp32_cuda_cores")
        line["err_vs_oracle_bf16"] = extras.get("err_vs_oracle_bf16")
        line["transforms"] = extras.get("transforms")
        line["fused"] = extras.get("fused")
        line["mixed_orders_all_shells"] = extras.get("mixed_orders_all_shells")
        line["resampling_free"] = extras.get("resampling_free")
        line["tables"] = extras.get("tables")
        line["learned"] = extras.get("learned")
        line["cpu_baseline_single_thread"] = extras.get("cpu_baseline_single_thread")
        line["path"] = {"tensor_cores": "required in the timed region", "cuda_core_kernels": cuda_core_kernels}
        line["summary"] = tail_summary(line)  # last, so that a truncated tail of the line still shows it
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def tail_summary(line: dict) -> dict:
    """The headline figures of every leg in a few hundred characters: BF16 and FP32 chain
    voxels/s and errors, the roofline fractions, the stand-alone transforms' HBM fractions."""
    def g(d, *keys):
        for k in keys:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return float(f"{d:.4g}") if isinstance(d, float) else d
    out = {"bf16_vps": g(line, "value"), "fused_vps": g(line, "fused", "value"),
           "bf16_err": [g(line, "err_vs_oracle_bf16", "s_out"),
                                                      g(line, "err_vs_oracle_bf16", "ds_in")],
           "gemm_frac": g(line, "roofline", "frac"), "step_frac": g(line, "roofline", "step_frac_of_tensor_peak"),
           "fp32_vps": g(line, "fp32", "value"), "fp32_err": [g(line, "fp32", "err_vs_oracle", "s_out"),
                                                              g(line, "fp32", "err_vs_oracle", "ds_in")]}
    lr = line.get("learned") or {}
    if isinstance(lr.get("heldout"), dict):
        out["net_vs_fallback"] = [g(lr, "heldout", "rel_l2_net"), g(lr, "heldout", "rel_l2_fallback")]
    if isinstance(lr.get("volume"), dict):
        out["volume"] = [g(lr, "volume", "voxels_per_s"), g(lr, "volume", "rel_l2_net"),
                         g(lr, "volume", "rel_l2_fallback")]
    tr = line.get("transforms") or {}
    for k in ("signal2sh_f32", "sh2signal_f32", "signal2sh_bf16_in", "sh2signal_bf16_in"):
        if isinstance(tr.get(k), dict):
            out[k] = [g(tr, k, "frac_hbm"), g(tr, k, "err_vs_oracle")]
    return out


def sampled_errors(ch, cfg, dirs, bvals, idx):
    """Relative L2 of s_out, ds_in, db on sampled voxels against the FP64 oracle."""
    import torch
    ch.step()
    torch.cuda.synchronize()
    S, m = len(cfg.dirs_per_shell), cfg.dirs_per_shell[0]

    def rows_to_vcd(rows, C):  # library signal rows -> [V, C, dirs]
        x = rows.float().cpu().numpy().astype(np.float64)
        out = np.empty((x.shape[1], C, S * m))
        for s in range(S):
            out[:, :, s * m:(s + 1) * m] = x[s * C * m:(s + 1) * C * m].reshape(C, m, -1).transpose(2, 0, 1)
        return out

    sig = rows_to_vcd(ch.s_in[:, idx], cfg.c_in)
    dso = rows_to_vcd(ch.ds_out[:, idx], cfg.c_out)
    oc = OracleChain(cfg, dirs, bvals)
    s_out, ds_in, _, _ = oc.step(sig, ch.w.cpu().numpy().astype(np.float64), ch.b.cpu().numpy().astype(np.float64),
                                 dso)
    got_s = rows_to_vcd(ch.s_out[:, idx], cfg.c_out)
    got_d = rows_to_vcd(ch.ds_in[:, idx], cfg.c_in)
    rel = lambda a, r: float(np.linalg.norm(a - r) / np.linalg.norm(r))  # noqa: E731
    return {"s_out": rel(got_s, s_out), "ds_in": rel(got_d, ds_in), "voxels": int(len(idx))}


def run_transforms(cfg, dirs, bvals, V, hbm_gbs, steps=20, warm=3, n_check=4096):
    """Signal2SH and SH2Signal alone on V voxels of a one-channel 3 x 90-direction
    fibre signal, FP32 in / FP32 out and BF16 in / FP32 out.  Per variant: device
    time (CUDA events on the launch stream, inputs larger than L2), algorithmic
    bytes (input read once, output written once), fraction of the measured HBM
    copy bandwidth, and relative L2 error against the FP64 oracle on n_check
    sampled voxels."""
    import torch
    from oracle import sh as osh
    from paper_1808_01517_gb300 import _lib as L
    from paper_1808_01517_gb300 import layers, synth
    basis = L.SHBasis(dirs, bvals, cfg.order, cfg.lam)
    ob = osh.SHBasisOracle(dirs, bvals, cfg.order, cfg.lam)
    S, N, nd = basis.n_shells, basis.n_coef, basis.n_dirs
    sig32 = layers.empty_act(nd, V, torch.float32)
    sig32.copy_(synth.fibre_signal_torch(dirs, bvals, V, seed=cfg.seed + 5))
    sh32 = layers.transform("signal2sh", basis, sig32, 1)
    idx = synth.voxel_subset(V, n_check, seed=cfg.seed + 98)
    idx_t = torch.from_numpy(idx).cuda()
    out = {}
    for kind, src32 in (("signal2sh", sig32), ("sh2signal", sh32)):
        for tag, dt in (("f32", torch.float32), ("bf16_in", torch.bfloat16)):
            x = layers.empty_act(src32.shape[0], V, dt)
            x.copy_(src32)
            rows_out = S * N if kind == "signal2sh" else nd
            y = layers.empty_act(rows_out, V, torch.float32)
            for _ in range(warm):
                layers.transform(kind, basis, x, 1, torch.float32, out=y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(steps):
                layers.transform(kind, basis, x, 1, torch.float32, out=y)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            by = x.shape[0] * V * x.element_size() + rows_out * V * 4
            # FP64 oracle on the sampled voxels, from the same (rounded) input values
            xin = x[:, idx_t].double().cpu().numpy()
            if kind == "signal2sh":
                ref = ob.signal2sh(xin.T[:, None, :])[:, 0]  # [n, S, N]
                ref_rows = ref.transpose(1, 2, 0).reshape(S * N, -1)
            else:
                ref = ob.sh2signal(xin.T.reshape(-1, S, N)[:, None])  # [n, 1, dirs]
                ref_rows = ref[:, 0].T
            got = y[:, idx_t].double().cpu().numpy()
            err = float(np.linalg.norm(got - ref_rows) / np.linalg.norm(ref_rows))
            out[f"{kind}_{tag}"] = {"ms": ms, "voxels_per_s": V / (ms * 1e-3), "bytes": int(by),
                                    "gbs": by / (ms * 1e-3) / 1e9, "frac_hbm": by / (ms * 1e-3) / 1e9 / hbm_gbs,
                                    "err_vs_oracle": err}
            del x, y
    out["config"] = {"n_vox": V, "channels": 1, "shells": list(cfg.dirs_per_shell), "sh_order": cfg.order,
                     "check_voxels": n_check, "timed_steps": steps}
    return out


def time_oracle_transforms(cfg, dirs, bvals, n_vox=131072, reps=3):
    """The FP64 oracle's Signal2SH and SH2Signal (Sec. 2.2) on a bounded host sample of the
    stand-alone transform workload (one channel, the full direction table): voxels/s, best
    of ``reps``, on the host's BLAS threads."""
    from oracle import sh as osh
    from paper_1808_01517_gb300 import synth
    ob = osh.SHBasisOracle(dirs, bvals, cfg.order, cfg.lam)
    sig = synth.gaussian((n_vox, 1, dirs.shape[0]), 1.0, seed=cfg.seed, tag="grads", sub=11)
    sh = synth.gaussian((n_vox, 1, ob.n_shells, ob.n_coef), 1.0, seed=cfg.seed, tag="coeffs", sub=11)
    best = {}
    for name, fn, x in (("signal2sh", ob.signal2sh, sig), ("sh2signal", ob.sh2signal, sh)):
        dt = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            fn(x)
            dt = min(dt, time.perf_counter() - t0)
        best[f"{name}_voxels_per_s"] = n_vox / dt
    best.update({"kind": "oracle", "cores": blas_threads(),
                 "sample": f"{n_vox} voxels, one channel, FP64 numpy oracle, best of {reps}"})
    return best


def run_e2e(ch, steps):
    """The same step through the public API with host buffers: every step copies its
    inputs (s_in, ds_out) from pinned host memory and reads its result, the weight and
    bias gradients, back; the copies of neighbouring steps overlap the compute
    (HostPipeline).  The activation outputs stay on the device, as inside a network."""
    import torch
    from paper_1808_01517_gb300.chain import Chain, HostPipeline
    ch2 = Chain(ch.cfg, ch.basis._dirs, ch.basis._bvals, ch.dtype)
    ch2.w.copy_(ch.w)
    ch2.b.copy_(ch.b)
    pipe = HostPipeline([ch, ch2])
    host_in, host_out = HostPipeline.host_buffers(ch)
    host_in["s_in"].copy_(ch.s_in)
    host_in["ds_out"].copy_(ch.ds_out)
    h2d = sum(t.numel() * t.element_size() for t in host_in.values())
    d2h = sum(t.numel() * t.element_size() for t in host_out.values())
    for i in range(2):  # warm-up: both chains once
        pipe.step(i, host_in, host_out)
    pipe.synchronize()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        pipe.step(i, host_in, host_out)
    pipe.synchronize()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    del ch2
    return {"value": ch.cfg.n_vox / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": dt * 1e3, "steps": steps, "timing": "host wall clock around the pipelined steps"}


if __name__ == "__main__":
    main()
