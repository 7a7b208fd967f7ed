"""Whole-volume helpers on the GPU: mask compaction (table T5, bit-exact against the
oracle), voxel gather/scatter, and the leaky ReLU pair."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lsc as olsc  # noqa: E402
from paper_1808_01517_gb300 import _lib as L  # noqa: E402
from paper_1808_01517_gb300 import layers, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,target", [((145, 174, 145), 900_000), ((7, 9, 11), 300), ((1, 1, 5), 3)])
def test_mask_compaction_bit_exact(shape, target):
    m = synth.ellipsoid_mask(shape, target, seed=5)
    ref = olsc.mask_to_index(m)
    n = m.size
    md = torch.from_numpy(m.reshape(-1).astype(np.uint8)).cuda()
    idx = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws_n = L.get().delimit_mask_compact_workspace_size(n)
    ws = torch.empty(ws_n, dtype=torch.uint8, device="cuda")
    L.check(L.get().delimit_mask_compact(md.data_ptr(), n, idx.data_ptr(), cnt.data_ptr(), ws.data_ptr(), ws_n, None),
            "delimit_mask_compact")
    torch.cuda.synchronize()
    k = int(cnt.item())
    assert k == len(ref)
    np.testing.assert_array_equal(idx[:k].cpu().numpy(), ref)
    # empty and full masks
    for val in (0, 1):
        md.fill_(val)
        L.check(L.get().delimit_mask_compact(md.data_ptr(), n, idx.data_ptr(), cnt.data_ptr(), ws.data_ptr(), ws_n,
                                             None), "delimit_mask_compact")
        torch.cuda.synchronize()
        assert int(cnt.item()) == (n if val else 0)
        if val:
            np.testing.assert_array_equal(idx.cpu().numpy(), np.arange(n))


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_gather_scatter_round_trip(dtype):
    rows, n_src = 30, 5000
    src = layers.empty_act(rows, n_src, dtype)
    src.copy_(torch.randn(rows, n_src))
    idx_np = np.sort(synth.rng(3, "subset").choice(n_src, 1234, replace=False)).astype(np.int64)
    idx = torch.from_numpy(idx_np).cuda()
    dst = layers.empty_act(rows, len(idx_np), dtype)
    code = layers._code(src)
    L.check(L.get().delimit_gather_voxels(src.data_ptr(), src.stride(0), n_src, rows, idx.data_ptr(), len(idx_np),
                                          dst.data_ptr(), dst.stride(0), code, None), "gather")
    back = layers.empty_act(rows, n_src, dtype)
    back.zero_()
    L.check(L.get().delimit_scatter_voxels(dst.data_ptr(), dst.stride(0), rows, idx.data_ptr(), len(idx_np),
                                           back.data_ptr(), back.stride(0), n_src, code, None), "scatter")
    torch.cuda.synchronize()
    assert torch.equal(dst.cpu(), src[:, idx_np].cpu())
    assert torch.equal(back[:, idx_np].cpu(), src[:, idx_np].cpu())
    mask = np.ones(n_src, bool)
    mask[idx_np] = False
    assert float(back[:, torch.from_numpy(mask).cuda()].abs().sum()) == 0.0


def test_leaky_relu_pair():
    x = layers.empty_act(45, 1001, torch.float32)
    x.copy_(torch.randn(45, 1001))
    y = layers.leaky_relu(x, 0.1)
    g = torch.randn(45, 1001, device="cuda")
    xa = x.detach().clone().requires_grad_(True)
    ya = layers.LeakyReLU(0.1)(xa)
    ya.backward(g)
    torch.cuda.synchronize()
    xn, gn = x.cpu().numpy(), g.cpu().numpy()
    np.testing.assert_array_equal(y.cpu().numpy(), np.where(xn > 0, xn, np.float32(0.1) * xn))
    np.testing.assert_allclose(xa.grad.cpu().numpy(), np.where(xn > 0, gn, 0.1 * gn), rtol=1e-7)


def test_volume_run_fused_normalisation_matches_unfused_network():
    """volume.run (mask compaction -> Signal2SH with the b0 division fused into its
    gathered load -> network -> scatter) against the plain network on the same
    voxels normalised outside the library."""
    from paper_1808_01517_gb300 import volume
    from paper_1808_01517_gb300.net import NetConfig, SphericalNet, tables
    cfg = NetConfig(hidden=8)
    dirs, bvals, sel = tables(cfg)
    net = SphericalNet(cfg, dirs[sel], dirs, bvals).cuda()
    state = net.state_dict()
    shape = (18, 21, 17)
    subs = [volume.Subject(i, cfg, state, shape=shape, mask_voxels=2500) for i in range(2)]
    outs, secs, vox = volume.run(subs, chunk=1000)
    assert vox == sum(int(s.mask.sum()) for s in subs)
    for sb, out in zip(subs, outs):
        m = torch.from_numpy(sb.mask.reshape(-1)).cuda()
        midx = torch.nonzero(m).flatten()
        x = (sb.volume[:, midx].float() / sb.b0[midx]).to(torch.bfloat16)  # normalised outside the library
        with torch.no_grad():
            ref = sb.net(x).float()
        got = out[:, midx].float()
        assert torch.isfinite(got).all()
        assert float((got - ref).norm() / ref.norm()) < 2e-2
        assert bool((out[:, ~m] == 0).all())
