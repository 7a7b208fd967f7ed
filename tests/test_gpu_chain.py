"""The metric chain (Signal2SH -> LSC -> SH2Signal, forward + backward): at the timed
workload against the FP64 oracle chain (sampled voxels, BF16 and FP32), and through
host buffers: HostPipeline's per-step results equal a direct device step on the same
inputs, bit for bit (same kernels, deterministic reductions), with two chains
alternating and copies overlapping compute on three streams."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1808_01517_gb300 import synth  # noqa: E402
from paper_1808_01517_gb300.chain import Chain, ChainConfig, HostPipeline  # noqa: E402

pytestmark = pytest.mark.gpu


def _inputs(cfg, dirs, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    s_in = torch.rand((cfg.c_in * dirs.shape[0], cfg.n_vox), generator=g, device="cuda").to(torch.bfloat16)
    ds_out = (0.1 * torch.randn((cfg.c_out * dirs.shape[0], cfg.n_vox), generator=g, device="cuda")).to(torch.bfloat16)
    return s_in, ds_out


@pytest.mark.parametrize("outputs", [("dw", "db"), ("dw", "db", "s_out", "ds_in")])
def test_host_pipeline_matches_direct_steps(outputs):
    cfg = ChainConfig(n_vox=4099, c_in=4, c_out=8)  # ragged voxel count
    dirs, bvals = synth.multishell_table(list(cfg.dirs_per_shell), list(cfg.bvals), seed=cfg.seed)
    S, K = 3, 1 + cfg.rings * cfg.sectors
    w = torch.from_numpy(synth.gaussian((cfg.c_out, S, cfg.c_in, S, K), 0.1, seed=3)).float().cuda()
    b = torch.from_numpy(synth.gaussian((cfg.c_out, S), 0.1, seed=4)).float().cuda()
    ch1, ch2, ref = (Chain(cfg, dirs, bvals) for _ in range(3))
    for c in (ch1, ch2, ref):
        c.w.copy_(w)
        c.b.copy_(b)
    pipe = HostPipeline([ch1, ch2])
    steps = 4
    inputs = [_inputs(cfg, dirs, 100 + i) for i in range(steps)]
    host_in = [HostPipeline.host_buffers(ch1, outputs)[0] for _ in range(steps)]
    host_out = [HostPipeline.host_buffers(ch1, outputs)[1] for _ in range(steps)]
    for i in range(steps):
        host_in[i]["s_in"].copy_(inputs[i][0])
        host_in[i]["ds_out"].copy_(inputs[i][1])
    torch.cuda.synchronize()
    for i in range(steps):
        pipe.step(i, host_in[i], host_out[i])
    pipe.synchronize()
    torch.cuda.synchronize()
    for i in range(steps):
        ref.set_inputs(inputs[i][0], inputs[i][1], w, b)
        ref.step()
        torch.cuda.synchronize()
        for k in outputs:
            assert torch.equal(host_out[i][k], getattr(ref, k).cpu()), (i, k)
    assert np.isfinite(host_out[-1]["dw"].numpy()).all()


@pytest.mark.parametrize("dtype,tol", [(torch.bfloat16, 1e-2), (torch.float32, 1e-5)])
def test_chain_full_size_sampled_vs_oracle(dtype, tol):
    """The timed workload (65,536 voxels, 3 x 90 directions, order 8, 16 -> 64 channels,
    adjacent shells, 4 x 12 kernel) in the launch configuration the benchmark times:
    s_out and ds_in on 24 sampled voxels, and the bias gradient (a plain reduction over
    all voxels of the upstream gradient), against the FP64 oracle chain."""
    from oracle import lsc as olsc
    from oracle import sh as osh
    cfg = ChainConfig(n_vox=65536)
    dirs, bvals = synth.multishell_table(list(cfg.dirs_per_shell), list(cfg.bvals), seed=cfg.seed)
    S, m, K = 3, 90, 1 + cfg.rings * cfg.sectors
    ch = Chain(cfg, dirs, bvals, dtype)
    w = synth.gaussian((cfg.c_out, S, cfg.c_in, S, K), 0.1, seed=5)
    b = synth.gaussian((cfg.c_out, S), 0.1, seed=6)
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    s_in = torch.rand((cfg.c_in * dirs.shape[0], cfg.n_vox), generator=g, device="cuda").to(dtype)
    ds_out = (0.1 * torch.randn((cfg.c_out * dirs.shape[0], cfg.n_vox), generator=g, device="cuda")).to(dtype)
    ch.set_inputs(s_in, ds_out, torch.from_numpy(w).float(), torch.from_numpy(b).float())
    ch.step()
    torch.cuda.synchronize()

    def rows_to_vcd(rows, C, idx):  # signal rows (s, c, i) -> [V, C, dirs]
        x = rows[:, idx].float().cpu().numpy().astype(np.float64)
        out = np.empty((x.shape[1], C, S * m))
        for s in range(S):
            out[:, :, s * m:(s + 1) * m] = x[s * C * m:(s + 1) * C * m].reshape(C, m, -1).transpose(2, 0, 1)
        return out

    idx = synth.voxel_subset(cfg.n_vox, 24, seed=11)
    ob = osh.SHBasisOracle(dirs, bvals, cfg.order, cfg.lam)
    og = olsc.LSCOracle(ob, cfg.order, S, np.deg2rad(cfg.radius_deg), cfg.rings, cfg.sectors, cfg.window)
    c_in = ob.signal2sh(rows_to_vcd(ch.s_in, cfg.c_in, idx))
    ref_s = ob.sh2signal(og.forward(c_in, w, b))
    dso = rows_to_vcd(ch.ds_out, cfg.c_out, idx)
    dc_in, _, _ = og.backward(c_in, w, ob.sh2signal_backward(dso))
    ref_ds = ob.signal2sh_backward(dc_in)
    rel = lambda a, r: float(np.linalg.norm(a - r) / np.linalg.norm(r))  # noqa: E731
    assert rel(rows_to_vcd(ch.s_out, cfg.c_out, idx), ref_s) <= tol
    assert rel(rows_to_vcd(ch.ds_in, cfg.c_in, idx), ref_ds) <= tol
    # db[co, s] = sum_v q_s . (B_s^T ds_out[v, co, s]) over all voxels, in FP64 from the inputs
    q = og.collapse_mats()[1]
    ds = ch.ds_out.double().cpu().numpy()
    ref_db = np.empty((cfg.c_out, S))
    for s in range(S):
        rows = ds[s * cfg.c_out * m:(s + 1) * cfg.c_out * m].reshape(cfg.c_out, m, -1).sum(axis=2)  # [co, i]
        ref_db[:, s] = rows @ (ob.B[s] @ q[s])
    assert rel(ch.db.cpu().numpy(), ref_db) <= tol
