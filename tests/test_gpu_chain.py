"""The metric chain (Signal2SH -> LSC -> SH2Signal, forward + backward) through host
buffers: HostPipeline's per-step results equal a direct device step on the same
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
