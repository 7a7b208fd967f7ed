"""Test helpers: convert between the oracle's voxel-major arrays and the library's
feature-row x voxel-column layout, and measure relative L2 errors.  No arithmetic
of the method lives here."""
import numpy as np


def sig_to_rows(sig, m_list):
    """oracle signal [V, C, sum m] (shell-grouped directions) -> library rows [C*sum m, V]."""
    V, Cc, _ = sig.shape
    parts, off = [], 0
    for m in m_list:
        parts.append(np.transpose(sig[:, :, off:off + m], (1, 2, 0)).reshape(Cc * m, V))
        off += m
    return np.concatenate(parts, 0)


def rows_to_sig(rows, m_list, Cc):
    V = rows.shape[1]
    out = np.empty((V, Cc, int(sum(m_list))), dtype=np.float64)
    r0 = off = 0
    for m in m_list:
        out[:, :, off:off + m] = np.transpose(rows[r0:r0 + Cc * m].reshape(Cc, m, V), (2, 0, 1))
        r0 += Cc * m
        off += m
    return out


def sh_to_rows(sh):
    """oracle SH [V, C, S, N] -> library rows [S*C*N, V]."""
    V, Cc, S, N = sh.shape
    return np.transpose(sh, (2, 1, 3, 0)).reshape(S * Cc * N, V)


def rows_to_sh(rows, S, Cc, N):
    return np.transpose(rows.reshape(S, Cc, N, -1), (3, 1, 0, 2)).astype(np.float64)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


# tolerances stated by the method's accuracy targets
TOL_F32 = 1e-5
TOL_BF16 = 1e-2
