"""The algorithmic work behind every roofline figure (Chain.flops, bytes, kernel_work),
against per-voxel figures derived independently from the layer definitions of Sec. 2.2
and 2.3 at the benchmark workload: 65,536 voxels, 3 shells x 90 directions, order 8
(45 coefficients), 16 -> 64 channels, adjacent-shell mixing (7 shell pairs), 4 x 12
kernel (K = 49), BF16 activations.

  one LSC GEMM (collapsed, Sec. 2.3):  2 * 7 * (64 * 45) * (16 * 45) = 29,030,400 FLOP/voxel
  Signal2SH on 16 channels:            2 * 16 * 270 * 45           =    388,800 FLOP/voxel
  SH2Signal on 64 channels:            2 * 64 * 270 * 45           =  1,555,200 FLOP/voxel
  Signal2SH bytes (BF16 read + write): 2 * (16 * 270 + 16 * 135)   =     12,960 B/voxel
  SH2Signal bytes:                     2 * (64 * 135 + 64 * 270)   =     51,840 B/voxel
  forward + backward of the chain:     2 * 388,800 + 2 * 1,555,200 + 3 * 29,030,400 = 90,979,200 FLOP/voxel

The chain is built on the CPU (host-only handles, host buffers); nothing runs on a GPU.
"""
import functools

import pytest
import torch

from paper_1808_01517_gb300 import _lib as L
from paper_1808_01517_gb300 import chain as chain_mod
from paper_1808_01517_gb300 import synth
from paper_1808_01517_gb300.chain import Chain, ChainConfig


@pytest.fixture
def host_chain(monkeypatch):
    monkeypatch.setattr(chain_mod.L, "SHBasis", functools.partial(L.SHBasis, host_only=True), raising=True)
    monkeypatch.setattr(chain_mod.L, "LSCGeometry", functools.partial(L.LSCGeometry, host_only=True), raising=True)

    def make(**kw):
        cfg = ChainConfig(**kw)
        dirs, bvals = synth.multishell_table(list(cfg.dirs_per_shell), list(cfg.bvals), seed=cfg.seed)
        return Chain(cfg, dirs, bvals, torch.bfloat16, device="cpu")
    return make


def test_rows_of_the_benchmark_workload(host_chain):
    ch = host_chain(n_vox=1024)
    assert ch.rows == dict(s_in=16 * 270, c_in=3 * 16 * 45, c_out=3 * 64 * 45, s_out=64 * 270)
    assert ch.geom.K == 49 and ch._pairs() == 7
    assert tuple(ch.w.shape) == (64, 3, 16, 3, 49) and tuple(ch.b.shape) == (64, 3)


def test_flops_and_bytes_per_voxel(host_chain):
    V = 65536
    ch = host_chain(n_vox=V)
    fl, by, kw = ch.flops(), ch.bytes(), ch.kernel_work()
    gemm, s2sh, sh2s = 29_030_400, 388_800, 1_555_200
    assert kw["lsc_fwd_gemm"][0] == kw["lsc_dgrad_gemm"][0] == kw["lsc_wgrad_gemm"][0] == gemm * V
    assert fl["signal2sh"] == fl["signal2sh_backward"] == s2sh * V
    assert fl["sh2signal"] == fl["sh2signal_backward"] == sh2s * V
    assert by["signal2sh"] == by["signal2sh_backward"] == 12_960 * V
    assert by["sh2signal"] == by["sh2signal_backward"] == 51_840 * V
    # the operator build (once per step, not per voxel): 2 * 7 * 64 * 16 * 45 * 45 * 49 FLOP
    build = 2 * 7 * 64 * 16 * 45 * 45 * 49
    assert kw["lsc_build_w"][0] == build and kw["lsc_build_w_tc"] == kw["lsc_build_w"]
    # per call: the forward is one GEMM plus the build, the backward two GEMMs, the build
    # and the reduction of dW to the kernel points (the same size as the build)
    assert fl["lsc_forward"] == gemm * V + build
    assert fl["lsc_backward"] == 2 * gemm * V + 2 * build
    transforms = fl["signal2sh"] + fl["signal2sh_backward"] + fl["sh2signal"] + fl["sh2signal_backward"]
    assert transforms / V + 3 * gemm == 90_979_200
    # the GEMMs' compulsory bytes: the voxel-streamed operands read and the output written once
    assert kw["lsc_fwd_gemm"][1] == 2 * V * (3 * 16 * 45 + 3 * 64 * 45)


def test_mixed_orders_and_all_shells(host_chain):
    """Order 4 -> 8 with every input shell feeding every output shell: 9 shell pairs,
    2 * 9 * (64 * 45) * (16 * 15) FLOP per GEMM per voxel."""
    ch = host_chain(n_vox=1024, order_in=4, window="all")
    assert ch._pairs() == 9 and ch.rows["c_in"] == 3 * 16 * 15
    assert ch.kernel_work()["lsc_fwd_gemm"][0] == 2 * 9 * (64 * 45) * (16 * 15) * 1024 == 12_441_600 * 1024
