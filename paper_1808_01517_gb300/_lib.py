"""ctypes binding of ``libdelimit.so`` (the C ABI in ``include/delimit.h``).

Argument marshalling only: every function of the C ABI is exposed under its
own name on :data:`lib` with full argtypes, plus small wrappers that take torch
tensors (device pointers, sizes and strides are read off the tensors).  There
is no fallback: if the library cannot be built or loaded, importing the layers
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

OK = 0
ERR_INVALID_ARG = 1
ERR_RANK_DEFICIENT = 2
ERR_UNSUPPORTED = 3
ERR_ALIGNMENT = 4
ERR_CUDA = 5
ERR_DEVICE_TIMEOUT = 6
ERR_OOM = 7
ERR_WORKSPACE = 8

F32 = 0
BF16 = 1
OPERATOR_READY = 1
HOST_ONLY = 1
LSC_NEIGHBOURS = 4
EVAL_ONLY = 2
WINDOW_SAME, WINDOW_ADJACENT, WINDOW_ALL = 0, 1, -1
WINDOWS = {"same": WINDOW_SAME, "adjacent": WINDOW_ADJACENT, "all": WINDOW_ALL}

_vp = C.c_void_p
_i64 = C.c_int64
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_i64p = C.POINTER(C.c_int64)

# name -> (restype, argtypes)
SIGNATURES = {
    "delimit_sh_basis_create": (C.c_int, [_dp, _dp, C.c_int, C.c_int, C.c_double, C.c_uint, C.POINTER(_vp)]),
    "delimit_sh_basis_destroy": (C.c_int, [_vp]),
    "delimit_sh_basis_info": (C.c_int, [_vp, _ip, _ip, _ip]),
    "delimit_sh_basis_shell": (C.c_int, [_vp, C.c_int, _ip, _ip, _dp]),
    "delimit_sh_basis_tables": (C.c_int, [_vp, C.c_int, _dp, _dp, _ip]),
    "delimit_signal2sh": (C.c_int, [_vp, _vp, _vp, _i64, C.c_int, _i64, _i64, C.c_int, C.c_int, _vp]),
    "delimit_lsc_ring_expand": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _vp]),
    "delimit_lsc_ring_reduce": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _vp]),
    "delimit_signal2sh_gather": (C.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _i64, _vp, _i64, C.c_int, C.c_int, C.c_int,
                                           _vp]),
    "delimit_sh2signal": (C.c_int, [_vp, _vp, _vp, _i64, C.c_int, _i64, _i64, C.c_int, C.c_int, _vp]),
    "delimit_signal2sh_backward": (C.c_int, [_vp, _vp, _vp, _i64, C.c_int, _i64, _i64, C.c_int, C.c_int, _vp]),
    "delimit_sh2signal_backward": (C.c_int, [_vp, _vp, _vp, _i64, C.c_int, _i64, _i64, C.c_int, C.c_int, _vp]),
    "delimit_lsc_geometry_create": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int,
                                              C.c_uint, C.POINTER(_vp)]),
    "delimit_lsc_geometry_destroy": (C.c_int, [_vp]),
    "delimit_lsc_geometry_info": (C.c_int, [_vp, _ip, _ip, _ip, _ip, _ip, _i64p]),
    "delimit_lsc_geometry_tables": (C.c_int, [_vp, C.c_int, _dp, _dp, _dp, _i64p, _i64p, _i64p, C.POINTER(C.c_ubyte)]),
    "delimit_lsc_neighbour_table": (C.c_int, [_vp, C.c_int, C.c_int, _i64p, _i64p, C.POINTER(C.c_int32)]),
    "delimit_selftest_wait_timeout": (C.c_int, [_vp]),
    "delimit_lsc_workspace_size": (C.c_size_t, [_vp, _i64, C.c_int, C.c_int, C.c_int, C.c_int]),
    "delimit_lsc_forward": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _i64, C.c_int, C.c_int, _i64, _i64, C.c_int, C.c_uint,
                                      _vp, C.c_size_t, _vp]),
    "delimit_lsc_backward": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i64, C.c_int, C.c_int, _i64, _i64,
                                       C.c_int, C.c_uint, _vp, C.c_size_t, _vp]),
    "delimit_lsc_forward_sh2signal": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _i64, C.c_int, C.c_int, _i64, _i64,
                                                C.c_int, C.c_uint, _vp, C.c_size_t, _vp]),
    "delimit_lsc_forward_sh2signal_supported": (C.c_int, [_vp, _i64, C.c_int, C.c_int, C.c_int]),
    "delimit_leaky_relu": (C.c_int, [_vp, _vp, _i64, _i64, _i64, _i64, C.c_float, C.c_int, _vp]),
    "delimit_leaky_relu_backward": (C.c_int, [_vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, C.c_float, C.c_int, _vp]),
    "delimit_mask_compact_workspace_size": (C.c_size_t, [_i64]),
    "delimit_mask_compact": (C.c_int, [_vp, _i64, _vp, _vp, _vp, C.c_size_t, _vp]),
    "delimit_gather_voxels": (C.c_int, [_vp, _i64, _i64, _i64, _vp, _i64, _vp, _i64, C.c_int, _vp]),
    "delimit_scatter_voxels": (C.c_int, [_vp, _i64, _i64, _vp, _i64, _vp, _i64, _i64, C.c_int, _vp]),
    "delimit_lsc_forward_noalloc": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _i64, C.c_int, C.c_int, _i64, _i64, C.c_int,
                                              _vp]),
    "delimit_device_error": (C.c_int, [_vp, _ip]),
    "delimit_set_tensor_cores": (C.c_int, [C.c_int]),
    "delimit_kernel_launches": (C.c_uint64, []),
    "delimit_cuda_core_fallbacks": (C.c_uint64, []),
    "delimit_set_gemm_cluster": (C.c_int, [C.c_int]),
    "delimit_trace_enable": (C.c_int, [C.c_int]),
    "delimit_trace_summary": (C.c_int64, [C.c_char_p, C.c_size_t]),
    "delimit_status_string": (C.c_char_p, [C.c_int]),
    "delimit_last_error": (C.c_char_p, []),
    "delimit_version": (C.c_int, []),
}


class DelimitError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = get().delimit_last_error().decode(errors="replace")
        name = get().delimit_status_string(status).decode()
        super().__init__(f"{where}: {name} ({status}): {msg}")


def get():
    """The loaded library (built in-tree on first use if needed).  DELIMIT_LIB names
    another build of it to load instead (e.g. the sanitized host build); it must exist."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("DELIMIT_LIB") or _build.LIB
            if os.environ.get("DELIMIT_LIB"):
                if not os.path.exists(path):
                    raise RuntimeError(f"DELIMIT_LIB={path} does not exist")
            elif not os.path.exists(path) or os.environ.get("DELIMIT_REBUILD"):
                path = _build.build()
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status: int, where: str):
    if status != OK:
        raise DelimitError(status, where)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


class SHBasis:
    """Handle of ``delimit_sh_basis`` (per-shell B_s and P_s of one gradient table)."""

    def __init__(self, dirs, bvals, order: int, lam: float = 0.0, host_only: bool = False, eval_only: bool = False):
        lib = get()
        self._dirs = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 3))
        self._bvals = np.ascontiguousarray(np.asarray(bvals, np.float64).reshape(-1))
        h = _vp()
        check(lib.delimit_sh_basis_create(_dptr(self._dirs), _dptr(self._bvals), self._dirs.shape[0], int(order),
                                          float(lam), (HOST_ONLY if host_only else 0) | (EVAL_ONLY if eval_only else 0),
                                          C.byref(h)),
              "delimit_sh_basis_create")
        self.handle = h
        self.order = int(order)
        self.lam = float(lam)
        ns, nc, nd = C.c_int(), C.c_int(), C.c_int()
        check(lib.delimit_sh_basis_info(h, C.byref(ns), C.byref(nc), C.byref(nd)), "delimit_sh_basis_info")
        self.n_shells, self.n_coef, self.n_dirs = ns.value, nc.value, nd.value
        self.m, self.dir_off, self.bval = [], [], []
        for s in range(self.n_shells):
            m, off, b = C.c_int(), C.c_int(), C.c_double()
            check(lib.delimit_sh_basis_shell(h, s, C.byref(m), C.byref(off), C.byref(b)), "delimit_sh_basis_shell")
            self.m.append(m.value)
            self.dir_off.append(off.value)
            self.bval.append(b.value)

    def tables(self, s: int):
        B = np.empty((self.m[s], self.n_coef))
        P = np.empty((self.n_coef, self.m[s]))
        idx = np.empty(self.m[s], np.int32)
        check(get().delimit_sh_basis_tables(self.handle, s, _dptr(B), _dptr(P), idx.ctypes.data_as(_ip)),
              "delimit_sh_basis_tables")
        return B, P, idx

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.delimit_sh_basis_destroy(h)
            self.handle = None


class LSCGeometry:
    """Handle of ``delimit_lsc_geometry`` (kernel points, collapse matrices, tables)."""

    def __init__(self, out_basis: SHBasis, order_in: int, shells_in: int, radius: float, rings: int, sectors: int,
                 window="same", host_only: bool = False, neighbours: bool = False):
        lib = get()
        self.out_basis = out_basis  # keep alive
        win = WINDOWS[window] if isinstance(window, str) else int(window)
        h = _vp()
        flags = (HOST_ONLY if host_only else 0) | (LSC_NEIGHBOURS if neighbours else 0)
        check(lib.delimit_lsc_geometry_create(out_basis.handle, int(order_in), int(shells_in), float(radius),
                                              int(rings), int(sectors), win, flags, C.byref(h)),
              "delimit_lsc_geometry_create")
        self.neighbours = bool(neighbours)
        self.handle = h
        K, ni, no, si, so, nn = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int64()
        check(lib.delimit_lsc_geometry_info(h, C.byref(K), C.byref(ni), C.byref(no), C.byref(si), C.byref(so),
                                            C.byref(nn)), "delimit_lsc_geometry_info")
        self.K, self.n_in, self.n_out = K.value, ni.value, no.value
        self.s_in, self.s_out, self.n_neighbours = si.value, so.value, nn.value
        self.rings, self.sectors, self.radius = int(rings), int(sectors), float(radius)

    def tables(self, s: int):
        ob = self.out_basis
        m = ob.m[s]
        kp = np.empty((m, self.K, 3))
        M = np.empty(((self.s_in,) if self.neighbours else ()) + (self.K, self.n_out, self.n_in))
        q = np.empty(self.n_out)
        ip = np.empty(m + 1, np.int64)
        lib = get()
        check(lib.delimit_lsc_geometry_tables(self.handle, s, None, None, None, ip.ctypes.data_as(_i64p), None, None,
                                              None), "delimit_lsc_geometry_tables")
        ix = np.empty(max(1, ip[-1]), np.int64)
        ri = np.empty((m, self.K), np.int64)
        win = np.empty(self.s_in, np.uint8)
        check(lib.delimit_lsc_geometry_tables(self.handle, s, _dptr(kp), _dptr(M), _dptr(q), ip.ctypes.data_as(_i64p),
                                              ix.ctypes.data_as(_i64p), ri.ctypes.data_as(_i64p),
                                              win.ctypes.data_as(C.POINTER(C.c_ubyte))),
              "delimit_lsc_geometry_tables")
        return {"kpts": kp, "M": M, "q": q, "nb_indptr": ip, "nb_indices": ix[:ip[-1]], "row_index": ri,
                "window": win.astype(bool)}

    def neighbour_table(self, s: int, s_in: int):
        """(indptr, indices, bins) of the resampling-free form for shell pair (s, s_in)."""
        lib = get()
        ip = np.empty(self.out_basis.m[s] + 1, np.int64)
        check(lib.delimit_lsc_neighbour_table(self.handle, s, s_in, ip.ctypes.data_as(_i64p), None, None),
              "delimit_lsc_neighbour_table")
        ix = np.empty(max(1, ip[-1]), np.int64)
        bx = np.empty(max(1, ip[-1]), np.int32)
        check(lib.delimit_lsc_neighbour_table(self.handle, s, s_in, ip.ctypes.data_as(_i64p), ix.ctypes.data_as(_i64p),
                                              bx.ctypes.data_as(C.POINTER(C.c_int32))), "delimit_lsc_neighbour_table")
        return ip, ix[:ip[-1]], bx[:ip[-1]]

    def workspace_size(self, n_vox: int, c_in: int, c_out: int, dtype: int, backward: bool) -> int:
        return int(get().delimit_lsc_workspace_size(self.handle, int(n_vox), int(c_in), int(c_out), int(dtype),
                                                    1 if backward else 0))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.delimit_lsc_geometry_destroy(h)
            self.handle = None


TC_OFF, TC_PREFER, TC_REQUIRE = 0, 1, 2


def set_tensor_cores(mode):
    """False / TC_OFF: CUDA cores only; True / TC_PREFER: tensor cores where a kernel takes
    the call (else CUDA cores, counted); TC_REQUIRE: a call without a tensor-core kernel
    is refused with ERR_UNSUPPORTED."""
    m = int(mode) if not isinstance(mode, bool) else (TC_PREFER if mode else TC_OFF)
    check(get().delimit_set_tensor_cores(m), "delimit_set_tensor_cores")


def cuda_core_fallbacks() -> int:
    return int(get().delimit_cuda_core_fallbacks())


def set_gemm_cluster(ctas: int):
    """CTAs per cluster of the LSC tensor-core GEMMs: 0 = each GEMM's default, 1 = single
    CTAs, 2 = CTA pairs with 2-SM MMAs where the tiles allow."""
    check(get().delimit_set_gemm_cluster(int(ctas)), "delimit_set_gemm_cluster")


def device_error(stream_ptr: int = 0):
    code = C.c_int()
    st = get().delimit_device_error(_vp(stream_ptr), C.byref(code))
    return st, code.value


def check_device_error(where: str, stream_ptr: int | None = None):
    """Synchronises the stream and raises DelimitError if a kernel recorded an error in the
    device error word (a bounded wait that ran out, a gather index out of range): such a
    kernel returns with its output partly written, so results computed after it are not
    trusted.  Default stream: torch's current one."""
    if stream_ptr is None:
        import torch
        stream_ptr = torch.cuda.current_stream().cuda_stream
    st, _ = device_error(stream_ptr)
    check(st, where)


def trace_enable(on: bool):
    check(get().delimit_trace_enable(1 if on else 0), "delimit_trace_enable")


def trace_summary() -> dict:
    """Per-name launch counts and total device milliseconds since tracing was enabled."""
    import json
    n = get().delimit_trace_summary(None, 0)
    buf = C.create_string_buffer(int(n) + 1)
    get().delimit_trace_summary(buf, len(buf))
    return json.loads(buf.value.decode())


def exported_names():
    return list(SIGNATURES)
