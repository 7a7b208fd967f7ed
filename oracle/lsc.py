"""Oracle: local spherical convolution (Sec. 2.3 and "Extension to multiple b-values").

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What the paper fixes (Sec. 2.3): a circular kernel made of an origin plus
points on a circle at angular distance alpha, stored as a vector of n+1
weights; every acquired direction's neighbourhood is *resampled* at the kernel
points through the SH interpolant, giving an m x (n+1) matrix; the layer
multiplies every row point-wise with the kernel vector and sums (a cross
correlation), giving m values.  The LSC's own parameters include the output SH
order and a Laplace-Beltrami lambda, and its example maps SH -> LSC -> SH, so
the m values are projected back onto SH.  With several b-values, shells act as
channels with a weight per input shell, and each output shell has its own
kernels.

Readings where the paper is silent or garbled (all also used by the library):

* Kernel geometry: ``kernel_sizes`` is read as R rings of ``sectors`` points
  each, ring r (1..R) at polar angle theta_r = r * alpha / R; point q of a
  ring at azimuth 2 pi q / sectors; vector order [origin, ring 1 (q = 0..),
  ring 2, ...]; K = 1 + R * sectors.  The paper's case ``[5]``, pi/5 is one
  ring of 5.
* Tangent frame at g: a = the coordinate axis with the smallest |g_k| (ties to
  the lowest k), e1 = normalise(a - (a.g) g), e2 = g x e1,
  p = cos(theta) g + sin(theta) (cos(phi) e1 + sin(phi) e2).
* The two parameter descriptions that both read "number of output shells" are
  taken as: ``lb_lambda`` = lambda of the LSC's output projection,
  ``angular_distance`` = the kernel's outer radius alpha.
* Sampled directions: output shell s is sampled on that shell's own directions
  of the output gradient table.
* Weights are independent per kernel point (no tying across sectors); layout
  [C_out, S_out, C_in, S_in, K]; entries outside the shell window are unused.
  The ring-tied variant (``ring_expand``) shares one weight per ring; with more
  sectors than the input order it acts per SH band (``ring_band_multipliers``).
* Shell windows: 'same' (s' = s), 'adjacent' (|s - s'| <= 1), 'all'.
* Neighbour table T3 of direction i: {j : |g_i . g_j| >= cos(alpha)} (antipodal
  aware, i itself included, ascending j, FP64 comparison, equality inside).
"""
from __future__ import annotations

import numpy as np

from .sh import SHBasisOracle, n_coef, real_sh

WINDOWS = {"same": 0, "adjacent": 1, "all": -1}


def tangent_frame(g: np.ndarray):
    """(e1, e2) of the reading above for one unit vector g."""
    g = np.asarray(g, np.float64)
    k = int(np.argmin(np.abs(g)))  # argmin returns the first (lowest) index on ties
    a = np.zeros(3)
    a[k] = 1.0
    e1 = a - np.dot(a, g) * g
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(g, e1)
    return e1, e2


def kernel_points(dirs: np.ndarray, radius: float, rings: int, sectors: int) -> np.ndarray:
    """Kernel points p[i, k] around every direction g_i, float64 [m, 1 + rings*sectors, 3]."""
    dirs = np.asarray(dirs, np.float64)
    K = 1 + rings * sectors
    out = np.empty((dirs.shape[0], K, 3))
    for i, g in enumerate(dirs):
        e1, e2 = tangent_frame(g)
        out[i, 0] = g
        for r in range(1, rings + 1):
            th = r * radius / rings
            for q in range(sectors):
                ph = 2.0 * np.pi * q / sectors
                out[i, 1 + (r - 1) * sectors + q] = (np.cos(th) * g
                                                     + np.sin(th) * (np.cos(ph) * e1 + np.sin(ph) * e2))
    return out


def ring_expand(w_ring: np.ndarray, rings: int, sectors: int) -> np.ndarray:
    """Ring-tied kernel weights [.., rings + 1] (origin, then one weight per ring,
    shared by the ring's points) as the per-point vector [.., 1 + rings * sectors]
    in the kernel order [origin, ring 1, ring 2, ...]."""
    w_ring = np.asarray(w_ring, np.float64)
    assert w_ring.shape[-1] == rings + 1
    return np.concatenate([w_ring[..., :1]] + [np.repeat(w_ring[..., r:r + 1], sectors, axis=-1)
                                               for r in range(1, rings + 1)], axis=-1)


def ring_reduce(dw: np.ndarray, rings: int, sectors: int) -> np.ndarray:
    """Adjoint of ring_expand: the gradient of the ring weights (sum over each ring's points)."""
    dw = np.asarray(dw, np.float64)
    return np.concatenate([dw[..., :1]] + [dw[..., 1 + r * sectors:1 + (r + 1) * sectors].sum(-1, keepdims=True)
                                           for r in range(rings)], axis=-1)


def ring_band_multipliers(w_ring: np.ndarray, order: int, radius: float, rings: int, sectors: int) -> np.ndarray:
    """mu[.., j] = w_0 + sectors * sum_r w_r P_l(j)(cos(r radius / rings)): by the
    Funk-Hecke theorem, each ring's sum of the interpolant of band l around g
    equals sectors * P_l(cos theta_r) times its value at g when sectors > l."""
    from scipy.special import eval_legendre  # a library routine for P_l
    w_ring = np.asarray(w_ring, np.float64)
    lvals = np.array([l for l in range(0, order + 1, 2) for _ in range(2 * l + 1)])
    mu = np.repeat(w_ring[..., :1], len(lvals), axis=-1).copy()
    for r in range(1, rings + 1):
        mu += sectors * w_ring[..., r:r + 1] * eval_legendre(lvals, np.cos(r * radius / rings))
    return mu


def kernel_row_index(m_per_shell, K: int):
    """Table T4: row of kernel point (s, i, k) in the stacked kernel-point list,
    row = (dir_off[s] + i) * K + k.  Returned as an int64 array [sum m_s, K]."""
    total = int(np.sum(m_per_shell))
    return np.arange(total * K, dtype=np.int64).reshape(total, K)


def shell_window(s_out: int, s_in: int, mode: str) -> np.ndarray:
    """Table T2: boolean [S_out, S_in], True where input shell s' feeds output shell s."""
    if mode == "all":
        return np.ones((s_out, s_in), bool)
    if s_out != s_in:
        raise ValueError("'same' and 'adjacent' windows need as many input as output shells")
    s = np.arange(s_out)
    d = np.abs(s[:, None] - s[None, :])
    return d == 0 if mode == "same" else d <= 1


def neighbour_csr(dirs: np.ndarray, radius: float):
    """Table T3: antipodal-aware neighbours within ``radius``: (indptr, indices) int64."""
    g = np.asarray(dirs, np.float64)
    c = np.cos(radius)
    indptr = [0]
    idx = []
    for i in range(g.shape[0]):
        for j in range(g.shape[0]):
            if abs(float(np.dot(g[i], g[j]))) >= c:
                idx.append(j)
        indptr.append(len(idx))
    return np.array(indptr, np.int64), np.array(idx, np.int64)


def mask_to_index(mask: np.ndarray) -> np.ndarray:
    """Table T5: ascending C-order linear indices of the True voxels of a volume whose
    last axis is fastest (the paper's subjects x dirs x H x W x D tensor, Sec. 2.1)."""
    return np.flatnonzero(np.asarray(mask, bool).reshape(-1)).astype(np.int64)


class LSCOracle:
    """One LSC layer: input SH of order ``order_in`` on ``shells_in`` shells, output SH on
    the shells of ``out_basis`` (its directions are the sampled directions, its order and
    lambda those of the output projection)."""

    def __init__(self, out_basis: SHBasisOracle, order_in: int, shells_in: int, radius: float,
                 rings: int, sectors: int, window: str = "same"):
        self.ob = out_basis
        self.order_in = order_in
        self.n_in = n_coef(order_in)
        self.n_out = out_basis.n_coef
        self.s_in = shells_in
        self.s_out = out_basis.n_shells
        self.radius = float(radius)
        self.rings, self.sectors = rings, sectors
        self.K = 1 + rings * sectors
        self.win = shell_window(self.s_out, self.s_in, window)
        self.dirs = [out_basis.dirs[r] for r in out_basis.rows]
        self.kpts = [kernel_points(d, radius, rings, sectors) for d in self.dirs]
        # basis of the input order at every kernel point: BK[s][i, k, j]
        self.BK = [real_sh(order_in, p.reshape(-1, 3)).reshape(p.shape[0], self.K, self.n_in)
                   for p in self.kpts]
        self.Pout = out_basis.P

    # ---- literal form: resample -> point-wise product -> projection (Sec. 2.3) ----
    def resample(self, c_in: np.ndarray, s: int) -> np.ndarray:
        """U[v, ci, s', i, k]: input shell s' interpolant at output-shell-s kernel points."""
        return np.einsum("ikj,vcpj->vcpik", self.BK[s], c_in, optimize=True)

    def direction_space(self, c_in, w, b) -> list:
        """y[s][v, co, i] = sum_{ci, s' in win(s), k} w[co,s,ci,s',k] U[v,ci,s',i,k] + b[co,s]."""
        ys = []
        for s in range(self.s_out):
            U = self.resample(c_in, s)
            mask = self.win[s].astype(np.float64)
            ws = w[:, s] * mask[None, None, :, None]  # [co, ci, s', k]
            ys.append(np.einsum("acpk,vcpik->vai", ws, U, optimize=True) + b[None, :, s, None])
        return ys

    def forward(self, c_in, w, b) -> np.ndarray:
        """c_out[v, co, s, :] = P_out,s y[s][v, co, :]."""
        ys = self.direction_space(c_in, w, b)
        return np.stack([y @ P.T for y, P in zip(ys, self.Pout)], axis=2)

    # ---- algebraic collapse (linearity), an independent second route ----
    def collapse_mats(self):
        """M[s][k] = P_out,s B^K_{s,k} ([N_out, N_in]) and q[s] = P_out,s 1."""
        M = [np.einsum("ai,ikj->kaj", P, BK) for P, BK in zip(self.Pout, self.BK)]
        q = [P.sum(axis=1) for P in self.Pout]
        return M, q

    def pair_mats(self, s: int, p: int) -> np.ndarray:
        """The collapse matrices [K, N_out, N_in] acting on input shell p for output shell s
        (in the resampled form they do not depend on p)."""
        return self.collapse_mats()[0][s]

    def forward_collapsed(self, c_in, w, b) -> np.ndarray:
        _, q = self.collapse_mats()
        V, Co = c_in.shape[0], w.shape[0]
        out = np.zeros((V, Co, self.s_out, self.n_out))
        for s in range(self.s_out):
            for p in range(self.s_in):
                if not self.win[s, p]:
                    continue
                Weff = np.einsum("ack,kxy->axcy", w[:, s, :, p, :], self.pair_mats(s, p))  # [co, a, ci, b]
                out[:, :, s, :] += np.einsum("axcy,vcy->vax", Weff, c_in[:, :, p, :])
            out[:, :, s, :] += b[None, :, s, None] * q[s][None, None, :]
        return out

    # ---- analytic gradients of the literal form ----
    def backward(self, c_in, w, d_out):
        """(dc_in, dw, db) for upstream gradient d_out [V, Co, S_out, N_out]."""
        dc_in = np.zeros_like(c_in)
        dw = np.zeros_like(w)
        db = np.zeros((w.shape[0], self.s_out))
        for s in range(self.s_out):
            dy = d_out[:, :, s, :] @ self.Pout[s]  # [v, co, i]
            db[:, s] = dy.sum(axis=(0, 2))
            U = self.resample(c_in, s)  # [v, ci, s', i, k]
            mask = self.win[s].astype(np.float64)
            dw[:, s] = np.einsum("vai,vcpik->acpk", dy, U, optimize=True) * mask[None, None, :, None]
            dU = np.einsum("acpk,vai->vcpik", w[:, s] * mask[None, None, :, None], dy, optimize=True)
            dc_in += self.resample_adjoint(dU, s)
        return dc_in, dw, db

    def resample_adjoint(self, dU: np.ndarray, s: int) -> np.ndarray:
        """Adjoint of ``resample``: dc[v, ci, s', j] = sum_{i,k} B^K_s[i,k,j] dU[v,ci,s',i,k]."""
        return np.einsum("ikj,vcpik->vcpj", self.BK[s], dU, optimize=True)


def neighbour_bins(g_i: np.ndarray, kpts_i: np.ndarray, dirs_in: np.ndarray, radius: float):
    """Acquired neighbours of one output direction g_i among the directions ``dirs_in`` of
    an input shell, and the kernel point each one is binned to (resampling-free form).

    Neighbour: |g_i . g_j| >= cos(radius) (antipodal aware, equality inside, ascending j).
    The neighbour's oriented direction u = g_j, or -g_j when g_i . g_j < 0 (the signal is
    antipodally symmetric), goes to the kernel point of g_i nearest to it on the sphere:
    the largest p_{i,k} . u, the lowest k on ties.  Returns (indices, bins), int64."""
    c = np.cos(radius)
    idx, bins = [], []
    for j in range(dirs_in.shape[0]):
        d = float(np.dot(g_i, dirs_in[j]))
        if abs(d) >= c:
            u = dirs_in[j] if d >= 0.0 else -dirs_in[j]
            idx.append(j)
            bins.append(int(np.argmax(kpts_i @ u)))  # argmax returns the first maximum
    return np.array(idx, np.int64), np.array(bins, np.int64)


class LSCNeighbourOracle(LSCOracle):
    """The LSC without resampling (the alternative Sec. 2.3 argues against): the kernel
    acts on the *acquired* neighbours of every direction instead of on interpolated
    kernel points.

    Readings (the paper describes this alternative only by what it lacks):

    * Input shell s' is sampled on the gradient table's shell-s' directions (the
      output basis' table), so it needs as many input as output shells; its values
      there are the input SH of order ``order_in`` evaluated at those directions.
    * Each acquired neighbour j of output direction i (shell s) in input shell s'
      (``neighbour_bins``) is assigned to the nearest kernel point of i; a kernel
      point takes the mean of the values assigned to it, 0 when none is.  The
      resulting m x (n + 1) neighbourhood matrix then meets the kernel exactly as in
      the resampled form (point-wise product, sum, bias, projection onto SH).

    Linearity again collapses the layer: M_{s,s',k} = P_out,s A^{s,s'}_k B_in,s', with
    A^{s,s'}_k[i, j] = 1 / (number of neighbours in bin (i, k)) for j in that bin."""

    def __init__(self, out_basis: SHBasisOracle, order_in: int, shells_in: int, radius: float,
                 rings: int, sectors: int, window: str = "same"):
        super().__init__(out_basis, order_in, shells_in, radius, rings, sectors, window)
        if shells_in != self.s_out:
            raise ValueError("the resampling-free LSC samples input shell s' on the table's shell s'")
        # input basis of order_in at every acquired direction of every shell
        self.B_in = [real_sh(order_in, d) for d in self.dirs]
        # neighbour tables per (output shell s, input shell s'): CSR + bin of each entry
        self.nb = {}
        self.A = {}
        for s in range(self.s_out):
            for p in range(self.s_in):
                m_o, m_i = self.dirs[s].shape[0], self.dirs[p].shape[0]
                indptr, indices, bins = [0], [], []
                A = np.zeros((m_o, self.K, m_i))
                for i in range(m_o):
                    ix, bx = neighbour_bins(self.dirs[s][i], self.kpts[s][i], self.dirs[p], self.radius)
                    indices.extend(ix.tolist())
                    bins.extend(bx.tolist())
                    indptr.append(len(indices))
                    for k in range(self.K):
                        sel = ix[bx == k]
                        if sel.size:
                            A[i, k, sel] = 1.0 / sel.size
                self.nb[s, p] = (np.array(indptr, np.int64), np.array(indices, np.int64),
                                 np.array(bins, np.int64))
                self.A[s, p] = A

    def acquired(self, c_in: np.ndarray, p: int) -> np.ndarray:
        """x[v, ci, j]: input shell p's SH evaluated at that shell's acquired directions."""
        return c_in[:, :, p, :] @ self.B_in[p].T

    def resample(self, c_in: np.ndarray, s: int) -> np.ndarray:
        """U[v, ci, s', i, k]: mean of input shell s' over the neighbours of output
        direction i binned to kernel point k (0 for an empty bin)."""
        V, Ci = c_in.shape[0], c_in.shape[1]
        m = self.dirs[s].shape[0]
        U = np.zeros((V, Ci, self.s_in, m, self.K))
        for p in range(self.s_in):
            U[:, :, p] = np.einsum("ikj,vcj->vcik", self.A[s, p], self.acquired(c_in, p), optimize=True)
        return U

    def resample_adjoint(self, dU: np.ndarray, s: int) -> np.ndarray:
        out = np.zeros(dU.shape[:3] + (self.n_in,))
        for p in range(self.s_in):
            dx = np.einsum("ikj,vcik->vcj", self.A[s, p], dU[:, :, p], optimize=True)  # [v, ci, j]
            out[:, :, p, :] = dx @ self.B_in[p]
        return out

    def collapse_mats(self):
        """M[s][s'] = P_out,s A^{s,s'}_k B_in,s' ([K, N_out, N_in]) and q[s] = P_out,s 1."""
        M = [[np.einsum("ai,ikj,jb->kab", self.Pout[s], self.A[s, p], self.B_in[p], optimize=True)
              for p in range(self.s_in)] for s in range(self.s_out)]
        q = [P.sum(axis=1) for P in self.Pout]
        return M, q

    def pair_mats(self, s: int, p: int) -> np.ndarray:
        return np.einsum("ai,ikj,jb->kab", self.Pout[s], self.A[s, p], self.B_in[p], optimize=True)
