"""Seeded synthetic inputs for the spherical layers (shared by tests, bench and oracle checks).

This module only *draws inputs*: gradient tables, multi-compartment fibre-model
diffusion signals, LSC weights and upstream gradients.  It contains none of the
method's arithmetic (no spherical-harmonic basis, no pseudo-inverse, no LSC), so
both the FP64 oracle and the CUDA path can be fed from it without sharing any
computation.

Every generator takes an explicit integer seed and a purpose tag; draws for
different purposes come from independent numpy PCG64 streams keyed by
``(seed, tag)``.  The fibre model is the stick + zeppelin mixture used to stand
in for the paper's brain scans (Sec. 2.2, "Efficiency of Signal2SH and
SH2Signal": a full scan of about 450,000 voxels; Sec. 3: HCP data with 3 shells
of 90 directions); the paper's datasets are not available here.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1808

# purpose tags -> independent streams
_TAGS = {
    "dirs": 1,
    "fibres": 2,
    "noise": 3,
    "weights": 4,
    "grads": 5,
    "rotation": 6,
    "jitter": 7,
    "coeffs": 8,
    "subset": 9,
    "snr": 10,
}

D_PAR = 1.7e-3  # mm^2/s, stick / zeppelin axial diffusivity
D_PERP = 0.3e-3  # mm^2/s, zeppelin radial diffusivity


def rng(seed: int, tag: str, sub: int = 0) -> np.random.Generator:
    """An independent PCG64 stream for (seed, purpose, sub-index)."""
    return np.random.default_rng([int(seed), _TAGS[tag], int(sub)])


def hemisphere_directions(n: int, seed: int = BASE_SEED, sub: int = 0) -> np.ndarray:
    """n unit vectors, uniform on the sphere, each flipped into z >= 0.

    "Antipodally symmetrised" is read as folding every direction onto the upper
    hemisphere (a gradient g and -g measure the same signal), not as doubling
    the set.  Returns float64 [n, 3].
    """
    g = rng(seed, "dirs", sub).standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    flip = g[:, 2] < 0
    g[flip] *= -1.0
    return g


def multishell_table(dirs_per_shell, bvals, seed: int = BASE_SEED):
    """Concatenated per-shell direction sets, grouped by shell in the given order.

    Each shell gets its own independently drawn hemisphere set.  Returns
    (dirs float64 [sum m_s, 3], bvals float64 [sum m_s]).
    """
    ds, bs = [], []
    for s, (m, b) in enumerate(zip(dirs_per_shell, bvals)):
        ds.append(hemisphere_directions(m, seed, sub=s))
        bs.append(np.full(m, float(b)))
    return np.concatenate(ds, 0), np.concatenate(bs, 0)


def random_rotation(max_angle_rad: float, seed: int, sub: int = 0) -> np.ndarray:
    """A rotation about a uniform random axis by an angle uniform in [0, max]."""
    r = rng(seed, "rotation", sub)
    axis = r.standard_normal(3)
    axis /= np.linalg.norm(axis)
    ang = r.uniform(0.0, max_angle_rad)
    kx = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(ang) * kx + (1 - np.cos(ang)) * (kx @ kx)


def perturbed_table(dirs: np.ndarray, max_rot_rad: float, max_jitter_rad: float, seed: int, sub: int):
    """A subject's gradient table: a seeded global rotation plus per-direction jitter."""
    R = random_rotation(max_rot_rad, seed, sub)
    g = dirs @ R.T
    r = rng(seed, "jitter", sub)
    # jitter: tilt each direction by an angle <= max_jitter about a random tangent axis
    t = r.standard_normal(g.shape)
    t -= np.sum(t * g, axis=1, keepdims=True) * g
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    ang = r.uniform(0.0, max_jitter_rad, size=(g.shape[0], 1))
    g = np.cos(ang) * g + np.sin(ang) * t
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g


def _fibre_params(n_vox: int, max_fibres: int, min_fibres: int, seed: int, sub: int):
    r = rng(seed, "fibres", sub)
    nf = r.integers(min_fibres, max_fibres + 1, size=n_vox)
    u = r.standard_normal((n_vox, max_fibres, 3))
    u /= np.linalg.norm(u, axis=2, keepdims=True)
    # fractions uniform on the simplex of the active fibres
    e = r.exponential(1.0, size=(n_vox, max_fibres))
    active = np.arange(max_fibres)[None, :] < nf[:, None]
    e = np.where(active, e, 0.0)
    w = e / e.sum(axis=1, keepdims=True)
    nu = r.uniform(0.5, 0.8, size=(n_vox, max_fibres))
    return u, w, nu


def fibre_signal(dirs: np.ndarray, bvals: np.ndarray, n_vox: int, *, seed: int = BASE_SEED,
                 sub: int = 0, min_fibres: int = 1, max_fibres: int = 2, snr=20.0,
                 chunk: int = 65536, dtype=np.float32) -> np.ndarray:
    """b0-normalised stick + zeppelin signals with Rician noise, [n_vox, n_dirs].

    S(g,b) = sum_f w_f [ nu e^{-b d_par (g.u_f)^2} + (1-nu) e^{-b (d_perp + (d_par-d_perp)(g.u_f)^2)} ]
    with S0 = 1, then |S + sigma n1 + i sigma n2| with sigma = 1/SNR.  ``snr`` is a
    number or a (lo, hi) range drawn uniformly per voxel.
    """
    dirs = np.asarray(dirs, np.float64)
    bvals = np.asarray(bvals, np.float64)
    out = np.empty((n_vox, dirs.shape[0]), dtype=dtype)
    u, w, nu = _fibre_params(n_vox, max_fibres, min_fibres, seed, sub)
    rn = rng(seed, "noise", sub)
    if isinstance(snr, (tuple, list)):
        sig_all = 1.0 / rng(seed, "snr", sub).uniform(snr[0], snr[1], size=n_vox)
    else:
        sig_all = np.full(n_vox, 1.0 / float(snr))
    for v0 in range(0, n_vox, chunk):
        v1 = min(n_vox, v0 + chunk)
        cos2 = np.einsum("gk,vfk->vfg", dirs, u[v0:v1]) ** 2  # [v, f, g]
        b = bvals[None, None, :]
        stick = np.exp(-b * D_PAR * cos2)
        zep = np.exp(-b * (D_PERP + (D_PAR - D_PERP) * cos2))
        s = np.einsum("vf,vfg->vg", w[v0:v1], nu[v0:v1, :, None] * stick + (1 - nu[v0:v1, :, None]) * zep)
        sig = sig_all[v0:v1, None]
        n1 = rn.standard_normal(s.shape)
        n2 = rn.standard_normal(s.shape)
        out[v0:v1] = np.sqrt((s + sig * n1) ** 2 + (sig * n2) ** 2)
    return out


def gaussian(shape, std: float, seed: int = BASE_SEED, tag: str = "weights", sub: int = 0,
             dtype=np.float64) -> np.ndarray:
    """Seeded N(0, std^2) array (LSC weights, upstream gradients, test coefficients)."""
    return (rng(seed, tag, sub).standard_normal(shape) * std).astype(dtype)


def voxel_subset(n_vox: int, k: int, seed: int = BASE_SEED) -> np.ndarray:
    """k distinct voxel indices in ascending order (sampled parity checks at full size)."""
    return np.sort(rng(seed, "subset").choice(n_vox, size=min(k, n_vox), replace=False))


def ellipsoid_mask(shape=(145, 174, 145), target_voxels: int = 900_000, seed: int = BASE_SEED,
                   sub: int = 0) -> np.ndarray:
    """A brain-like boolean mask: an ellipsoid with a seeded, slightly perturbed radius,
    scaled so that about ``target_voxels`` voxels are inside."""
    r = rng(seed, "subset", 100 + sub)
    X, Y, Z = np.meshgrid(*(np.arange(n) - (n - 1) / 2 for n in shape), indexing="ij")
    axes = np.array(shape, np.float64) / 2 * r.uniform(0.92, 1.0, size=3)
    q = (X / axes[0]) ** 2 + (Y / axes[1]) ** 2 + (Z / axes[2]) ** 2
    # choose the level set that holds target_voxels voxels
    thr = np.partition(q.ravel(), target_voxels - 1)[target_voxels - 1]
    return q <= thr


def fibre_signal_torch(dirs, bvals, n_vox: int, *, seed: int = BASE_SEED, sub: int = 0, max_fibres: int = 2,
                       min_fibres: int = 1, snr=20.0, device="cuda", dtype=None, return_clean: bool = False):
    """The same stick + zeppelin + Rician model as :func:`fibre_signal`, drawn on the
    device with a seeded torch generator (for workloads too large to draw on the host).
    ``snr`` is a number or a (lo, hi) range drawn uniformly per voxel.  Returns
    [n_dirs, n_vox] (feature rows x voxel columns), float32 unless ``dtype``; with
    ``return_clean`` also the noise-free signal."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + int(sub) * 7919 + _TAGS["fibres"])
    g = torch.as_tensor(np.asarray(dirs, np.float64), dtype=torch.float32, device=device)
    b = torch.as_tensor(np.asarray(bvals, np.float64), dtype=torch.float32, device=device)
    nf = torch.randint(min_fibres, max_fibres + 1, (n_vox,), generator=gen, device=device)
    u = torch.randn((max_fibres, n_vox, 3), generator=gen, device=device)
    u = u / u.norm(dim=2, keepdim=True)
    e = -torch.log(torch.rand((max_fibres, n_vox), generator=gen, device=device).clamp_min(1e-12))
    e = torch.where(torch.arange(max_fibres, device=device)[:, None] < nf[None, :], e, torch.zeros_like(e))
    w = e / e.sum(0, keepdim=True)
    nu = 0.5 + 0.3 * torch.rand((max_fibres, n_vox), generator=gen, device=device)
    s = torch.zeros((g.shape[0], n_vox), device=device)
    for f in range(max_fibres):
        cos2 = (g @ u[f].T) ** 2  # [dirs, vox]
        stick = torch.exp(-b[:, None] * D_PAR * cos2)
        zep = torch.exp(-b[:, None] * (D_PERP + (D_PAR - D_PERP) * cos2))
        s += w[f][None, :] * (nu[f][None, :] * stick + (1 - nu[f][None, :]) * zep)
    if isinstance(snr, (tuple, list)):
        sigma = 1.0 / (snr[0] + (snr[1] - snr[0]) * torch.rand((1, n_vox), generator=gen, device=device))
    else:
        sigma = 1.0 / float(snr)
    n1 = torch.randn(s.shape, generator=gen, device=device)
    n2 = torch.randn(s.shape, generator=gen, device=device)
    out = torch.sqrt((s + sigma * n1) ** 2 + (sigma * n2) ** 2)
    if dtype is not None:
        out = out.to(dtype)
    if return_clean:
        return out, (s if dtype is None else s.to(dtype))
    return out
