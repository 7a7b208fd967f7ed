"""Oracle: spherical-harmonic transforms (Sec. 2.2, Signal2SH and SH2Signal).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper names the basis only through its citation of Descoteaux et al. 2007
(Sec. 1) and says the GPU transforms are mathematically identical to the
dipy ``sf_to_sh`` / ``sh_to_sf`` pair (Sec. 2.2, efficiency paragraph).
Readings taken here:

* basis: real, symmetric (even l only), index j = l(l+1)/2 + m, m = -l..l,
  Y_j = sqrt(2) Re(Y_l^|m|) for m < 0, Y_l^0 for m = 0, sqrt(2) Im(Y_l^m) for
  m > 0, with the complex Y_l^m orthonormal and carrying the Condon-Shortley
  phase; theta = polar angle from +z, phi = atan2(y, x).
* Signal2SH: c = P s with P = (B^T B + lambda L)^-1 B^T, L = diag(l_j^2 (l_j+1)^2)
  (the Laplace-Beltrami penalty of the cited method; lambda is the paper's
  ``lb_lambda``, not normalised by the number of directions).
* SH2Signal: s = B(targets) c, no regularisation.
* Shells: rows are grouped by b-value rounded to an integer, shells in order of
  ascending b, rows within a shell in input order.
"""
from __future__ import annotations

from math import factorial, pi, sqrt

import numpy as np


def n_coef(order: int) -> int:
    """Number of real even-order coefficients up to ``order``: (L+1)(L+2)/2."""
    if order < 0 or order % 2:
        raise ValueError("SH order must be even and >= 0")
    return (order + 1) * (order + 2) // 2


def sh_lm(order: int):
    """Table T1: (l, m) of every coefficient index j = l(l+1)/2 + m."""
    ls, ms = [], []
    for l in range(0, order + 1, 2):
        for m in range(-l, l + 1):
            ls.append(l)
            ms.append(m)
    return np.array(ls, np.int64), np.array(ms, np.int64)


def sh_index(l: int, m: int) -> int:
    """Inverse of T1."""
    return l * (l + 1) // 2 + m


def assoc_legendre(l: int, m: int, x: np.ndarray) -> np.ndarray:
    """P_l^m(x) for 0 <= m <= l with the Condon-Shortley phase (-1)^m.

    Standard three-term recurrence in l, started from
    P_m^m = (-1)^m (2m-1)!! (1-x^2)^(m/2) and P_{m+1}^m = x (2m+1) P_m^m.
    """
    x = np.asarray(x, np.float64)
    pmm = np.ones_like(x)
    if m > 0:
        somx2 = np.sqrt(np.clip((1.0 - x) * (1.0 + x), 0.0, None))
        dfact = 1.0
        for _ in range(m):
            pmm = -pmm * dfact * somx2
            dfact += 2.0
    if l == m:
        return pmm
    pmmp1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pmmp1
    p_lm2, p_lm1 = pmm, pmmp1
    for ll in range(m + 2, l + 1):
        p_l = ((2 * ll - 1) * x * p_lm1 - (ll + m - 1) * p_lm2) / (ll - m)
        p_lm2, p_lm1 = p_lm1, p_l
    return p_lm1


def _norm(l: int, m: int) -> float:
    return sqrt((2 * l + 1) / (4 * pi) * factorial(l - m) / factorial(l + m))


def real_sh(order: int, dirs: np.ndarray) -> np.ndarray:
    """Basis matrix B[i, j] = Y_j(g_i) of the real symmetric basis, float64 [n, N]."""
    g = np.asarray(dirs, np.float64)
    r = np.linalg.norm(g, axis=1)
    ct = np.clip(g[:, 2] / r, -1.0, 1.0)
    phi = np.arctan2(g[:, 1], g[:, 0])
    out = np.empty((g.shape[0], n_coef(order)))
    for l in range(0, order + 1, 2):
        for m in range(-l, l + 1):
            am = abs(m)
            base = _norm(l, am) * assoc_legendre(l, am, ct)
            if m < 0:
                val = sqrt(2.0) * base * np.cos(am * phi)
            elif m == 0:
                val = base
            else:
                val = sqrt(2.0) * base * np.sin(am * phi)
            out[:, sh_index(l, m)] = val
    return out


def lb_penalty(order: int) -> np.ndarray:
    """Diagonal of the Laplace-Beltrami penalty: l_j^2 (l_j + 1)^2."""
    l, _ = sh_lm(order)
    return (l * (l + 1)).astype(np.float64) ** 2


def pinv_normal(B: np.ndarray, order: int, lam: float) -> np.ndarray:
    """Route 1: P = (B^T B + lambda L)^-1 B^T by a Cholesky solve of the normal equations."""
    A = B.T @ B + lam * np.diag(lb_penalty(order))
    Lc = np.linalg.cholesky(A)
    Y = np.linalg.solve(Lc, B.T)
    return np.linalg.solve(Lc.T, Y)


def pinv_qr(B: np.ndarray, order: int, lam: float) -> np.ndarray:
    """Route 2: the same operator as the least-squares solution of the augmented
    system [B; sqrt(lambda) diag(l(l+1))] c ~= [s; 0], by Householder QR."""
    l, _ = sh_lm(order)
    aug = np.vstack([B, sqrt(lam) * np.diag((l * (l + 1)).astype(np.float64))])
    Q, R = np.linalg.qr(aug)
    n = B.shape[0]
    return np.linalg.solve(R, Q[:n].T)


def group_shells(bvals: np.ndarray):
    """Shell grouping: integer-rounded b-values, ascending; returns (shell_b, rows per shell)."""
    b = np.rint(np.asarray(bvals, np.float64)).astype(np.int64)
    if np.any(b <= 0):
        raise ValueError("b = 0 rows must be removed (the paper normalises by b0 first)")
    shells = np.unique(b)
    return shells, [np.nonzero(b == sb)[0] for sb in shells]


class SHBasisOracle:
    """Per-shell B_s and P_s of one gradient table (the Signal2SH constructor, Sec. 2.2)."""

    def __init__(self, dirs, bvals, order: int, lam: float):
        self.dirs = np.asarray(dirs, np.float64)
        self.order = order
        self.lam = float(lam)
        self.shell_b, self.rows = group_shells(bvals)
        self.B = [real_sh(order, self.dirs[r]) for r in self.rows]
        self.P = [pinv_normal(Bs, order, lam) for Bs in self.B]
        self.n_coef = n_coef(order)
        self.m = [len(r) for r in self.rows]

    @property
    def n_shells(self):
        return len(self.rows)

    def signal2sh(self, sig: np.ndarray) -> np.ndarray:
        """sig [..., n_dirs] (input row order) -> sh [..., S, N]."""
        return np.stack([sig[..., r] @ P.T for r, P in zip(self.rows, self.P)], axis=-2)

    def sh2signal(self, sh: np.ndarray) -> np.ndarray:
        """sh [..., S, N] -> sig [..., n_dirs] on this table's own directions."""
        out = np.empty(sh.shape[:-2] + (self.dirs.shape[0],))
        for s, (r, B) in enumerate(zip(self.rows, self.B)):
            out[..., r] = sh[..., s, :] @ B.T
        return out

    def signal2sh_backward(self, d_sh: np.ndarray) -> np.ndarray:
        """Adjoint of signal2sh: d_sig = P_s^T d_c per shell."""
        out = np.empty(d_sh.shape[:-2] + (self.dirs.shape[0],))
        for s, (r, P) in enumerate(zip(self.rows, self.P)):
            out[..., r] = d_sh[..., s, :] @ P
        return out

    def sh2signal_backward(self, d_sig: np.ndarray) -> np.ndarray:
        """Adjoint of sh2signal: d_c = B_s^T d_s per shell."""
        return np.stack([d_sig[..., r] @ B for r, B in zip(self.rows, self.B)], axis=-2)
