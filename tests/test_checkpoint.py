"""Checkpoint / resume of the network's training (net.save_checkpoint, net.load_checkpoint).

The training loop's state is the weights, the Adam moments, the cosine schedule and the
batch sampler's generator.  A run interrupted at a checkpoint and resumed into freshly
built (differently initialised) objects must end bit for bit where the uninterrupted run
ends.  Checked on the CPU with a small torch model driven by the same loop structure as
net.train (the network itself runs only on the GPU kernels).
"""
import os

import torch

from paper_1808_01517_gb300 import net


def _fresh(init_seed: int):
    torch.manual_seed(init_seed)
    model = torch.nn.Sequential(torch.nn.Linear(8, 16), torch.nn.Tanh(), torch.nn.Linear(16, 4)).double()
    opt = torch.optim.Adam(model.parameters(), lr=1e-2)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=6)
    gen = torch.Generator()
    gen.manual_seed(3)
    return model, opt, sched, gen


def _data():
    g = torch.Generator()
    g.manual_seed(1)
    return torch.randn(64, 8, generator=g, dtype=torch.float64), torch.randn(64, 4, generator=g, dtype=torch.float64)


def _loop(model, opt, sched, gen, X, Y, start, stop):
    for _ in range(start, stop):
        idx = torch.randint(0, X.shape[0], (16,), generator=gen)
        loss = torch.mean((model(X[idx]) - Y[idx]) ** 2)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        sched.step()


def _params(model):
    return [p.detach().clone() for p in model.parameters()]


def test_resumed_run_matches_the_uninterrupted_run(tmp_path):
    X, Y = _data()
    a = _fresh(0)
    _loop(*a, X, Y, 0, 6)

    b = _fresh(0)
    _loop(*b, X, Y, 0, 3)
    path = str(tmp_path / "ckpt.pt")
    net.save_checkpoint(path, *b, next_step=3)
    assert os.path.exists(path) and not os.path.exists(path + ".tmp")

    c = _fresh(1)  # other initial weights: everything must come from the checkpoint
    start = net.load_checkpoint(path, *c)
    assert start == 3
    _loop(*c, X, Y, start, 6)
    for p, q in zip(_params(a[0]), _params(c[0])):
        assert torch.equal(p, q)
    assert c[2].get_last_lr() == a[2].get_last_lr()


def test_resume_depends_on_the_sampler_state(tmp_path):
    """Re-seeding the batch sampler after loading (dropping its saved state) changes the
    result: the generator state is part of what must be restored."""
    X, Y = _data()
    a = _fresh(0)
    _loop(*a, X, Y, 0, 6)
    b = _fresh(0)
    _loop(*b, X, Y, 0, 3)
    path = str(tmp_path / "ckpt.pt")
    net.save_checkpoint(path, *b, next_step=3)
    c = _fresh(0)
    start = net.load_checkpoint(path, *c)
    c[3].manual_seed(3)
    _loop(*c, X, Y, start, 6)
    assert any(not torch.equal(p, q) for p, q in zip(_params(a[0]), _params(c[0])))
