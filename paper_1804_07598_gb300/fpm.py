"""Thin ctypes binding of libfpm (include/fpm.h): same names, argument
marshalling only.  Every step of the hot path runs in the library's CUDA
kernels; there is no Python or CPU fallback.  Tensors are torch CUDA tensors
(device memory and streams are PyTorch's); ``None`` passes NULL.

A call that returns a status other than FPM_OK raises ``FpmError`` carrying
the library's last-error text.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(HERE, "libfpm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "fpm.h")

FPM_OK, FPM_ERR_INVALID, FPM_ERR_CAPACITY, FPM_ERR_DOMAIN, FPM_ERR_CUDA, FPM_ERR_TIMEOUT, FPM_ERR_WORKSPACE = range(7)
FPM_F32, FPM_F64 = 0, 1
FPM_FLAG_CAPACITY, FPM_FLAG_DOMAIN, FPM_FLAG_TIMEOUT = 1, 2, 4
STATUS_BYTES = 64
# int32 word of fpm_dev_status.max_staged in a status tensor
STATUS_MAX_STAGED = 6

_c = ctypes
_VP = _c.c_void_p


class FpmError(RuntimeError):
    def __init__(self, status: int, text: str):
        super().__init__(f"fpm status {status}: {text}")
        self.status = status


class fpm_box(_c.Structure):
    _fields_ = [("L", _c.c_double * 3), ("periodic", _c.c_int32 * 3)]


class fpm_grid(_c.Structure):
    _fields_ = [("nc", _c.c_int32 * 3), ("ncell", _c.c_int32), ("inv", _c.c_float * 3), ("tiles_x", _c.c_int32),
                ("stage_cap", _c.c_int32), ("sweep_blocks", _c.c_int32)]

    @property
    def shape(self):
        return tuple(self.nc)


class fpm_replica(_c.Structure):
    _fields_ = [("box", fpm_box), ("grid", fpm_grid), ("p0", _c.c_int32), ("n", _c.c_int32), ("c0", _c.c_int32),
                ("t0", _c.c_int32)]


class fpm_batch(_c.Structure):
    _fields_ = [("R", _c.c_int32), ("n_total", _c.c_int32), ("ncell_total", _c.c_int32),
                ("ntiles_total", _c.c_int32), ("max_n", _c.c_int32), ("max_ncell", _c.c_int32),
                ("stage_cap", _c.c_int32), ("sweep_blocks", _c.c_int32), ("sweep_threads", _c.c_int32),
                ("step_blocks_per_sm", _c.c_int32)]


class fpm_dev_status(_c.Structure):
    _fields_ = [("flags", _c.c_uint32), ("max_nn", _c.c_uint32), ("rebuild", _c.c_uint32),
                ("nrebuild", _c.c_uint32), ("max_disp2", _c.c_uint32), ("bad_index", _c.c_uint32),
                ("max_staged", _c.c_uint32), ("spilled", _c.c_uint32), ("reserved", _c.c_uint32 * 8)]


class fpm_sph_params(_c.Structure):
    _fields_ = [("h", _c.c_double), ("mass", _c.c_double), ("rho0", _c.c_double), ("c0", _c.c_double),
                ("gamma", _c.c_double), ("alpha", _c.c_double), ("eta2", _c.c_double), ("g", _c.c_double * 3),
                ("kernel", _c.c_int32)]


class fpm_dem_params(_c.Structure):
    _fields_ = [("R", _c.c_double), ("m", _c.c_double), ("I", _c.c_double), ("kn", _c.c_double),
                ("kt", _c.c_double), ("gn", _c.c_double), ("gt", _c.c_double), ("mu", _c.c_double),
                ("dt", _c.c_double), ("g", _c.c_double * 3)]


_lock = threading.Lock()
_lib = None

# Number of kernels the wrappers below have enqueued (each wrapper knows how
# many kernels its C call launches); benchmarks read it to report launches.
launches = 0


def _count(k: int):
    global launches
    launches += int(k)

# name -> (restype, argtypes); mirrors include/fpm.h
_SIG = {
    "fpm_status_string": (_c.c_char_p, [_c.c_int]),
    "fpm_last_error": (_c.c_char_p, []),
    "fpm_status_from_device": (_c.c_int, [_c.POINTER(fpm_dev_status)]),
    "fpm_nbr_ld": (_c.c_int64, [_c.c_int32]),
    "fpm_graph_if_begin": (_c.c_int, [_VP, _VP, _VP, _c.POINTER(_c.c_int32)]),
    "fpm_graph_if_end": (_c.c_int, [_VP]),
    "fpm_grid_make": (_c.c_int, [_c.POINTER(fpm_box), _c.c_double, _c.c_int32, _c.POINTER(fpm_grid)]),
    "fpm_celllist_workspace": (_c.c_int, [_c.c_int32, _c.POINTER(fpm_grid), _c.c_int, _c.POINTER(_c.c_size_t)]),
    "fpm_celllist_build": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _c.c_int,
                                      _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _c.c_size_t, _VP, _VP, _VP]),
    "fpm_reorder": (_c.c_int, [_c.c_int32, _c.c_int32, _VP, _VP, _VP, _VP, _VP]),
    "fpm_verlet_list_bytes": (_c.c_int, [_c.c_int32, _c.POINTER(fpm_grid), _c.c_int32, _c.POINTER(_c.c_size_t)]),
    "fpm_verlet_build": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _c.c_int, _VP, _VP,
                                    _c.c_double, _c.c_int32, _VP, _c.c_size_t, _VP, _VP, _VP, _VP, _VP]),
    "fpm_verlet_build_half": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _c.c_int, _VP, _VP,
                                         _c.c_double, _c.c_int32, _VP, _c.c_size_t, _VP, _VP, _VP, _VP, _VP]),
    "fpm_lj_forces_half": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _VP, _VP, _VP,
                                      _c.c_int32, _c.c_double, _c.c_double, _c.c_double, _VP, _VP, _VP, _c.c_size_t,
                                      _VP, _c.c_size_t, _VP, _VP, _c.c_double, _VP]),
    "fpm_lj_half_acc_bytes": (_c.c_int, [_c.c_int32, _c.POINTER(_c.c_size_t)]),
    "fpm_verlet_decode": (_c.c_int, [_c.POINTER(fpm_grid), _c.c_int32, _c.c_int32, _VP, _VP, _VP, _VP]),
    "fpm_verlet_check": (_c.c_int, [_c.POINTER(fpm_box), _c.c_int32, _c.c_int, _VP, _VP, _c.c_double, _VP, _VP]),
    "fpm_reduce_workspace": (_c.c_int, [_c.c_int32, _c.POINTER(fpm_grid), _c.POINTER(_c.c_size_t)]),
    "fpm_lj_forces": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _c.c_int, _VP, _VP, _VP,
                                 _c.c_int32, _c.c_double, _c.c_double, _c.c_double, _VP, _VP, _VP, _c.c_size_t, _VP,
                                 _VP]),
    "fpm_lj_forces_kick": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _c.c_int, _VP, _VP,
                                      _VP, _c.c_int32, _c.c_double, _c.c_double, _c.c_double, _VP, _VP, _VP,
                                      _c.c_size_t, _VP, _VP, _c.c_double, _VP]),
    "fpm_lj_forces_noalloc": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _c.c_int, _VP, _VP,
                                         _VP, _c.c_int32, _c.c_double, _c.c_double, _c.c_double, _VP, _VP, _VP, _VP]),
    "fpm_vv_step": (_c.c_int, [_c.POINTER(fpm_box), _c.c_int32, _c.c_int, _c.c_int32, _c.c_double, _VP, _VP, _VP,
                               _VP]),
    "fpm_vv_drift_check": (_c.c_int, [_c.POINTER(fpm_box), _c.c_int32, _c.c_int, _c.c_double, _VP, _VP, _VP, _VP,
                                      _c.c_double, _VP, _VP]),
    "fpm_sph_forces": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _VP, _VP, _VP, _VP,
                                  _c.c_int32, _c.POINTER(fpm_sph_params), _VP, _VP, _VP, _c.c_size_t, _VP, _VP]),
    "fpm_sph_density": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _VP, _VP, _VP,
                                   _c.c_int32, _c.POINTER(fpm_sph_params), _VP, _VP, _c.c_size_t, _VP, _VP]),
    "fpm_sph_predict": (_c.c_int, [_c.POINTER(fpm_box), _c.c_int32, _c.POINTER(fpm_sph_params), _c.c_double, _VP,
                                   _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _c.c_double, _VP, _VP]),
    "fpm_sph_correct": (_c.c_int, [_c.POINTER(fpm_box), _c.c_int32, _c.POINTER(fpm_sph_params), _VP, _VP, _VP, _VP,
                                   _VP, _VP, _VP, _c.c_double, _VP, _VP, _VP]),
    "fpm_dem_forces": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _VP, _VP, _VP, _VP, _VP,
                                  _c.c_int32, _c.POINTER(fpm_dem_params), _VP, _VP, _VP, _VP, _VP, _c.c_size_t, _VP,
                                  _VP]),
    "fpm_dem_leapfrog": (_c.c_int, [_c.POINTER(fpm_box), _c.c_int32, _c.POINTER(fpm_dem_params), _VP, _VP, _VP, _VP,
                                    _VP, _VP, _c.c_double, _VP, _VP]),
    "fpm_dem_packed_bytes": (_c.c_size_t, [_c.c_int32]),
    "fpm_dem_rebuild_begin": (_c.c_int, [_c.POINTER(fpm_grid), _c.c_int32, _c.c_int32, _VP, _VP, _VP, _VP, _VP, _VP,
                                         _VP, _VP, _VP]),
    "fpm_dem_rebuild_end": (_c.c_int, [_c.POINTER(fpm_grid), _c.c_int32, _c.c_int32, _VP, _VP, _VP, _VP, _VP, _VP,
                                       _VP, _VP]),
    "fpm_mesh_grid": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(_c.c_int32), _c.POINTER(fpm_grid)]),
    "fpm_p2m": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _VP, _VP, _VP, _VP, _VP, _VP]),
    "fpm_m2p": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _VP, _VP, _VP, _VP, _VP]),
    "fpm_lj_backward": (_c.c_int, [_c.POINTER(fpm_box), _c.POINTER(fpm_grid), _c.c_int32, _c.c_int, _VP, _VP, _VP,
                                   _c.c_int32, _c.c_double, _c.c_double, _c.c_double, _VP, _c.c_double, _VP, _VP,
                                   _VP, _c.c_size_t, _VP, _VP]),
    "fpm_vv_adjoint": (_c.c_int, [_c.c_int32, _c.c_int, _VP, _VP, _c.c_double, _c.c_double, _VP, _VP, _VP, _VP,
                                  _VP, _VP]),
    "fpm_adjoint_seed": (_c.c_int, [_c.c_int32, _c.c_int, _VP, _VP, _VP, _VP, _VP]),
    "fpm_adjoint_loss": (_c.c_int, [_VP, _VP, _VP, _VP]),
    "fpm_test_wait_budget": (_c.c_int, [_c.c_int64]),
    "fpm_adjoint_finish": (_c.c_int, [_c.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "fpm_kinetic": (_c.c_int, [_c.c_int32, _c.c_int, _VP, _VP, _VP, _c.c_size_t, _VP]),
    "fpm_unpack_xyz": (_c.c_int, [_c.c_int32, _c.c_int, _VP, _VP, _VP]),
    "fpm_pack_xyz": (_c.c_int, [_c.c_int32, _c.c_int, _VP, _VP, _VP]),
    "fpm_batch_plan": (_c.c_int, [_c.c_int32, _c.POINTER(fpm_box), _c.POINTER(_c.c_int32), _c.c_double, _c.c_int32,
                                  _c.POINTER(fpm_replica), _c.POINTER(fpm_batch)]),
    "fpm_batch_drift_check": (_c.c_int, [_c.POINTER(fpm_batch), _VP, _c.c_double, _VP, _VP, _VP, _VP, _c.c_double,
                                         _VP, _VP]),
    "fpm_batch_celllist_workspace": (_c.c_int, [_c.POINTER(fpm_batch), _c.POINTER(_c.c_size_t)]),
    "fpm_batch_celllist_build": (_c.c_int, [_c.POINTER(fpm_batch), _VP, _VP, _VP, _VP, _VP, _VP, _VP, _c.c_size_t,
                                            _VP, _VP, _VP]),
    "fpm_batch_list_bytes": (_c.c_int, [_c.POINTER(fpm_batch), _c.c_int32, _c.POINTER(_c.c_size_t)]),
    "fpm_batch_verlet_build": (_c.c_int, [_c.POINTER(fpm_batch), _VP, _VP, _VP, _c.c_double, _c.c_int32, _VP,
                                          _c.c_size_t, _VP, _VP, _VP, _VP, _VP]),
    "fpm_batch_verlet_decode": (_c.c_int, [_c.POINTER(fpm_batch), _c.c_int32, _VP, _VP, _VP, _VP]),
    "fpm_batch_workspace": (_c.c_int, [_c.POINTER(fpm_batch), _c.POINTER(_c.c_size_t)]),
    "fpm_batch_lj_forces": (_c.c_int, [_c.POINTER(fpm_batch), _VP, _VP, _VP, _VP, _c.c_int32, _c.c_double,
                                       _c.c_double, _c.c_double, _VP, _VP, _VP, _c.c_size_t, _VP, _VP]),
    "fpm_batch_lj_forces_kick": (_c.c_int, [_c.POINTER(fpm_batch), _VP, _VP, _VP, _VP, _c.c_int32, _c.c_double,
                                            _c.c_double, _c.c_double, _VP, _VP, _VP, _c.c_size_t, _VP, _VP,
                                            _c.c_double, _VP]),
    "fpm_batch_step": (_c.c_int, [_c.POINTER(fpm_batch), _VP, _c.c_double, _c.c_double, _c.c_double, _c.c_int32,
                                  _c.c_double, _c.c_double, _c.c_double, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                  _c.c_size_t, _VP, _VP, _VP, _c.c_size_t, _VP, _c.c_size_t, _VP, _VP, _VP]),
}


def header_functions() -> list:
    """Names of every function declared in include/fpm.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fpm_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Load libfpm.so (built in-tree by paper_1804_07598_gb300.build).  Fails
    loudly when the library is missing: there is no fallback path."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO_PATH):
                raise RuntimeError(f"libfpm.so not built ({SO_PATH}); run paper_1804_07598_gb300.build.build()")
            L = _c.CDLL(SO_PATH)
            for name, (res, args) in _SIG.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("libfpm takes device tensors only")
    if not t.is_contiguous():
        raise ValueError("libfpm takes contiguous tensors only")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int):
    if status != FPM_OK:
        raise FpmError(status, lib().fpm_last_error().decode())


def _nbytes(t):
    return 0 if t is None else t.numel() * t.element_size()


def make_box(L, periodic=(1, 1, 1)) -> fpm_box:
    b = fpm_box()
    for d in range(3):
        b.L[d] = float(L[d] if hasattr(L, "__len__") else L)
        b.periodic[d] = int(periodic[d] if hasattr(periodic, "__len__") else periodic)
    return b


def prec_of(t) -> int:
    import torch
    return FPM_F64 if t.dtype == torch.float64 else FPM_F32


# ------------------------------------------------------------------ helpers

def fpm_status_string(s: int) -> str:
    return lib().fpm_status_string(int(s)).decode()


def fpm_last_error() -> str:
    return lib().fpm_last_error().decode()


def fpm_status_from_device(host_status: fpm_dev_status) -> int:
    return lib().fpm_status_from_device(_c.byref(host_status))


def fpm_graph_if_begin(d_flag, body_stream, stream=None) -> bool:
    """Opens a device-decided branch in the graph being captured on `stream`
    (see include/fpm.h); returns False (nothing added) when not capturing."""
    cap = _c.c_int32(0)
    _check(lib().fpm_graph_if_begin(_ptr(d_flag), _stream(stream), _stream(body_stream), _c.byref(cap)))
    if cap.value:
        _count(1)
    return bool(cap.value)


def fpm_graph_if_end(body_stream):
    _check(lib().fpm_graph_if_end(_stream(body_stream)))


def fpm_nbr_ld(n: int) -> int:
    return int(lib().fpm_nbr_ld(int(n)))


def fpm_grid_make(box: fpm_box, r_cell: float, n_hint: int = 0) -> fpm_grid:
    g = fpm_grid()
    _check(lib().fpm_grid_make(_c.byref(box), float(r_cell), int(n_hint), _c.byref(g)))
    return g


def fpm_verlet_list_bytes(n: int, grid: fpm_grid, cap: int) -> int:
    b = _c.c_size_t(0)
    _check(lib().fpm_verlet_list_bytes(int(n), _c.byref(grid), int(cap), _c.byref(b)))
    return b.value


def fpm_celllist_workspace(n: int, grid: fpm_grid, prec: int) -> int:
    b = _c.c_size_t(0)
    _check(lib().fpm_celllist_workspace(int(n), _c.byref(grid), int(prec), _c.byref(b)))
    return b.value


def fpm_reduce_workspace(n: int, grid: fpm_grid = None) -> int:
    b = _c.c_size_t(0)
    _check(lib().fpm_reduce_workspace(int(n), _c.byref(grid) if grid is not None else None, _c.byref(b)))
    return b.value


def read_status(d_status) -> fpm_dev_status:
    """Copy a device status block (a 64-byte tensor) to the host."""
    h = d_status.detach().cpu().contiguous()
    s = fpm_dev_status()
    _c.memmove(_c.addressof(s), h.data_ptr(), STATUS_BYTES)
    return s


# ------------------------------------------------------------------ kernels

def fpm_celllist_build(box, grid, n, prec, pos_in, vel_in, id_in, pos_out, vel_out, id_out, cell_start, perm,
                       workspace, d_status=None, d_gate=None, stream=None):
    _check(lib().fpm_celllist_build(_c.byref(box), _c.byref(grid), int(n), int(prec), _ptr(pos_in), _ptr(vel_in),
                                    _ptr(id_in), _ptr(pos_out), _ptr(vel_out), _ptr(id_out), _ptr(cell_start),
                                    _ptr(perm), _ptr(workspace), _nbytes(workspace), _ptr(d_status), _ptr(d_gate),
                                    _stream(stream)))
    _count(6 if n > 0 else 3)


def fpm_reorder(n, elem_bytes, perm, src, dst, d_gate=None, stream=None):
    _check(lib().fpm_reorder(int(n), int(elem_bytes), _ptr(perm), _ptr(src), _ptr(dst), _ptr(d_gate),
                             _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_verlet_build(box, grid, n, prec, pos, cell_start, r_list, cap, list_obj, nn, pos_ref=None, d_status=None,
                     d_gate=None, stream=None):
    _check(lib().fpm_verlet_build(_c.byref(box), _c.byref(grid), int(n), int(prec), _ptr(pos), _ptr(cell_start),
                                  float(r_list), int(cap), _ptr(list_obj), _nbytes(list_obj), _ptr(nn),
                                  _ptr(pos_ref), _ptr(d_status), _ptr(d_gate), _stream(stream)))
    _count((3 if n > 0 else 0) + (1 if d_gate is not None else 0))


def fpm_verlet_build_half(box, grid, n, prec, pos, cell_start, r_list, cap, list_obj, nn, pos_ref=None,
                          d_status=None, d_gate=None, stream=None):
    _check(lib().fpm_verlet_build_half(_c.byref(box), _c.byref(grid), int(n), int(prec), _ptr(pos),
                                       _ptr(cell_start), float(r_list), int(cap), _ptr(list_obj), _nbytes(list_obj),
                                       _ptr(nn), _ptr(pos_ref), _ptr(d_status), _ptr(d_gate), _stream(stream)))
    _count((3 if n > 0 else 0) + (1 if d_gate is not None else 0))


def fpm_lj_half_acc_bytes(n: int) -> int:
    b = _c.c_size_t(0)
    _check(lib().fpm_lj_half_acc_bytes(int(n), _c.byref(b)))
    return b.value


def fpm_lj_forces_half(box, grid, n, pos, list_obj, nn, cap, eps, sigma, rc, force, d_energy, acc, workspace,
                       d_status=None, vel=None, dt=0.0, stream=None):
    _check(lib().fpm_lj_forces_half(_c.byref(box), _c.byref(grid), int(n), _ptr(pos), _ptr(list_obj), _ptr(nn),
                                    int(cap), float(eps), float(sigma), float(rc), _ptr(force), _ptr(d_energy),
                                    _ptr(acc), _nbytes(acc), _ptr(workspace), _nbytes(workspace), _ptr(d_status),
                                    _ptr(vel), float(dt), _stream(stream)))
    _count(2 if n > 0 else 0)


def fpm_verlet_decode(grid, n, cap, list_obj, nn, out, stream=None):
    _check(lib().fpm_verlet_decode(_c.byref(grid), int(n), int(cap), _ptr(list_obj), _ptr(nn), _ptr(out),
                                   _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_verlet_check(box, n, prec, pos, pos_ref, skin, d_status, stream=None):
    _check(lib().fpm_verlet_check(_c.byref(box), int(n), int(prec), _ptr(pos), _ptr(pos_ref), float(skin),
                                  _ptr(d_status), _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_lj_forces(box, grid, n, prec, pos, list_obj, nn, cap, eps, sigma, rc, force, d_energy=None,
                  workspace=None, d_status=None, stream=None):
    _check(lib().fpm_lj_forces(_c.byref(box), _c.byref(grid), int(n), int(prec), _ptr(pos), _ptr(list_obj), _ptr(nn),
                               int(cap), float(eps), float(sigma), float(rc), _ptr(force), _ptr(d_energy),
                               _ptr(workspace), _nbytes(workspace), _ptr(d_status), _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_lj_forces_kick(box, grid, n, prec, pos, list_obj, nn, cap, eps, sigma, rc, force, d_energy, workspace,
                       d_status, vel, dt, stream=None):
    """fpm_lj_forces, then vel += dt/2 F in the same launch."""
    _check(lib().fpm_lj_forces_kick(_c.byref(box), _c.byref(grid), int(n), int(prec), _ptr(pos), _ptr(list_obj),
                                    _ptr(nn), int(cap), float(eps), float(sigma), float(rc), _ptr(force),
                                    _ptr(d_energy), _ptr(workspace), _nbytes(workspace), _ptr(d_status), _ptr(vel),
                                    float(dt), _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_lj_forces_noalloc(box, grid, n, prec, pos, list_obj, nn, cap, eps, sigma, rc, force, d_energy=None,
                          d_status=None, stream=None):
    """fpm_lj_forces for callers that cannot allocate device memory: the
    reduction scratch is built into the library (n <= 2^24); concurrent calls
    on one device must be serialised by the caller."""
    _check(lib().fpm_lj_forces_noalloc(_c.byref(box), _c.byref(grid), int(n), int(prec), _ptr(pos), _ptr(list_obj),
                                       _ptr(nn), int(cap), float(eps), float(sigma), float(rc), _ptr(force),
                                       _ptr(d_energy), _ptr(d_status), _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_test_wait_budget(cycles):
    """Test hook: budget (SM cycles) of the LJ sweeps' first wait per work
    item; 0 restores the default."""
    _check(lib().fpm_test_wait_budget(int(cycles)))


def fpm_vv_step(box, n, prec, half, dt, pos, vel, force, stream=None):
    _check(lib().fpm_vv_step(_c.byref(box), int(n), int(prec), int(half), float(dt), _ptr(pos), _ptr(vel),
                             _ptr(force), _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_vv_drift_check(box, n, prec, dt, pos, vel, force, pos_ref, skin, d_status, stream=None):
    _check(lib().fpm_vv_drift_check(_c.byref(box), int(n), int(prec), float(dt), _ptr(pos), _ptr(vel), _ptr(force),
                                    _ptr(pos_ref), float(skin), _ptr(d_status), _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_kinetic(n, prec, vel, d_out, workspace, stream=None):
    _check(lib().fpm_kinetic(int(n), int(prec), _ptr(vel), _ptr(d_out), _ptr(workspace), _nbytes(workspace),
                             _stream(stream)))
    _count(1)


def fpm_lj_backward(box, grid, n, prec, pos, list_obj, nn, cap, eps, sigma, rc, a, scale, adj_pos, d_params=None,
                    workspace=None, d_status=None, stream=None):
    _check(lib().fpm_lj_backward(_c.byref(box), _c.byref(grid), int(n), int(prec), _ptr(pos), _ptr(list_obj),
                                 _ptr(nn), int(cap), float(eps), float(sigma), float(rc), _ptr(a), float(scale),
                                 _ptr(adj_pos), _ptr(d_params), _ptr(workspace), _nbytes(workspace), _ptr(d_status),
                                 _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_vv_adjoint(n, prec, perm, dt, c, xbar_in, vbar_in, xbar_out, vbar_out, a_out, d_gate=None, stream=None):
    _check(lib().fpm_vv_adjoint(int(n), int(prec), _ptr(perm), _ptr(d_gate), float(dt), float(c), _ptr(xbar_in),
                                _ptr(vbar_in), _ptr(xbar_out), _ptr(vbar_out), _ptr(a_out), _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_adjoint_seed(n, prec, force, xbar, vbar, a_out, stream=None):
    _check(lib().fpm_adjoint_seed(int(n), int(prec), _ptr(force), _ptr(xbar), _ptr(vbar), _ptr(a_out),
                                  _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_adjoint_loss(d_energy, d_half_sumf2, d_loss, stream=None):
    _check(lib().fpm_adjoint_loss(_ptr(d_energy), _ptr(d_half_sumf2), _ptr(d_loss), _stream(stream)))
    _count(1)


def fpm_adjoint_finish(n, ids, xbar, vbar, theta_seed, theta_steps, grad_x, grad_v, grad_theta, stream=None):
    _check(lib().fpm_adjoint_finish(int(n), _ptr(ids), _ptr(xbar), _ptr(vbar), _ptr(theta_seed), _ptr(theta_steps),
                                    _ptr(grad_x), _ptr(grad_v), _ptr(grad_theta), _stream(stream)))
    _count(1)


def fpm_sph_forces(box, grid, n, pos, vr, list_obj, nn, cap, params, acc, d_dtcons=None, workspace=None,
                   d_status=None, stream=None):
    _check(lib().fpm_sph_forces(_c.byref(box), _c.byref(grid), int(n), _ptr(pos), _ptr(vr), _ptr(list_obj),
                                _ptr(nn), int(cap), _c.byref(params), _ptr(acc), _ptr(d_dtcons), _ptr(workspace),
                                _nbytes(workspace), _ptr(d_status), _stream(stream)))
    _count(1 if n > 0 else 0)


def dem_params(R=0.06, m=1.0, I=1.44e-3, kn=7.849, kt=2.243, gn=3.401, gt=0.0, mu=0.5, dt=0.01,
               g=(0.0, 0.0, 0.0)) -> fpm_dem_params:
    p = fpm_dem_params()
    p.R, p.m, p.I, p.kn, p.kt, p.gn, p.gt, p.mu, p.dt = R, m, I, kn, kt, gn, gt, mu, dt
    for d in range(3):
        p.g[d] = g[d]
    return p


def fpm_dem_forces(box, grid, n, pos, vel, omega, list_obj, nn, cap, params, hist, force, torque, d_ncontact=None,
                   workspace=None, d_status=None, stream=None):
    _check(lib().fpm_dem_forces(_c.byref(box), _c.byref(grid), int(n), _ptr(pos), _ptr(vel), _ptr(omega),
                                _ptr(list_obj), _ptr(nn), int(cap), _c.byref(params), _ptr(hist), _ptr(force),
                                _ptr(torque), _ptr(d_ncontact), _ptr(workspace), _nbytes(workspace), _ptr(d_status),
                                _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_dem_leapfrog(box, n, params, pos, vel, omega, force, torque, pos_ref=None, skin=0.0, d_status=None,
                     stream=None):
    _check(lib().fpm_dem_leapfrog(_c.byref(box), int(n), _c.byref(params), _ptr(pos), _ptr(vel), _ptr(omega),
                                  _ptr(force), _ptr(torque), _ptr(pos_ref), float(skin), _ptr(d_status),
                                  _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_dem_packed_bytes(n) -> int:
    return int(lib().fpm_dem_packed_bytes(int(n)))


def fpm_dem_rebuild_begin(grid, n, cap, list_obj, nn, hist, omega, packed, d_gate, d_pending, d_status=None,
                          stream=None):
    _check(lib().fpm_dem_rebuild_begin(_c.byref(grid), int(n), int(cap), _ptr(list_obj), _ptr(nn), _ptr(hist),
                                       _ptr(omega), _ptr(packed), _ptr(d_gate), _ptr(d_pending), _ptr(d_status),
                                       _stream(stream)))
    _count(2 if n > 0 else 0)


def fpm_dem_rebuild_end(grid, n, cap, list_obj, nn, perm, packed, hist, omega, d_pending, stream=None):
    _check(lib().fpm_dem_rebuild_end(_c.byref(grid), int(n), int(cap), _ptr(list_obj), _ptr(nn), _ptr(perm),
                                     _ptr(packed), _ptr(hist), _ptr(omega), _ptr(d_pending), _stream(stream)))
    _count(2 if n > 0 else 0)


def fpm_mesh_grid(box, N) -> fpm_grid:
    g = fpm_grid()
    arr = (_c.c_int32 * 3)(*[int(v) for v in N])
    _check(lib().fpm_mesh_grid(_c.byref(box), arr, _c.byref(g)))
    return g


def fpm_p2m(box, mesh_grid, n, pos, val, cell_start, mesh, d_status=None, stream=None):
    _check(lib().fpm_p2m(_c.byref(box), _c.byref(mesh_grid), int(n), _ptr(pos), _ptr(val), _ptr(cell_start),
                         _ptr(mesh), _ptr(d_status), _stream(stream)))
    _count(1)


def fpm_m2p(box, mesh_grid, n, pos, mesh, val, order=None, stream=None):
    _check(lib().fpm_m2p(_c.byref(box), _c.byref(mesh_grid), int(n), _ptr(pos), _ptr(mesh), _ptr(order), _ptr(val),
                         _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_sph_density(box, grid, n, pos, list_obj, nn, cap, params, rho, workspace, d_status=None, stream=None):
    _check(lib().fpm_sph_density(_c.byref(box), _c.byref(grid), int(n), _ptr(pos), _ptr(list_obj), _ptr(nn),
                                 int(cap), _c.byref(params), _ptr(rho), _ptr(workspace), _nbytes(workspace),
                                 _ptr(d_status), _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_sph_predict(box, n, params, cfl, pos, vr, acc, d_dtcons, pos_h, vr_h, d_dt, d_dtcons_h, pos_ref=None,
                    skin=0.0, d_status=None, stream=None):
    _check(lib().fpm_sph_predict(_c.byref(box), int(n), _c.byref(params), float(cfl), _ptr(pos), _ptr(vr), _ptr(acc),
                                 _ptr(d_dtcons), _ptr(pos_h), _ptr(vr_h), _ptr(d_dt), _ptr(d_dtcons_h),
                                 _ptr(pos_ref), float(skin), _ptr(d_status), _stream(stream)))
    _count(1)


def fpm_sph_correct(box, n, params, pos, vr, vr_h, acc_h, d_dt, d_dtcons, pos_ref=None, skin=0.0, d_status=None,
                    d_time=None, stream=None):
    _check(lib().fpm_sph_correct(_c.byref(box), int(n), _c.byref(params), _ptr(pos), _ptr(vr), _ptr(vr_h),
                                 _ptr(acc_h), _ptr(d_dt), _ptr(d_dtcons), _ptr(pos_ref), float(skin), _ptr(d_status),
                                 _ptr(d_time), _stream(stream)))
    _count(1)


# ------------------------------------------------------------------ batched replicas

def fpm_batch_plan(boxes, counts, r_cell: float, tile_target: int = 0):
    """(reps: ctypes array of fpm_replica [R], batch: fpm_batch) for replicas
    with the given fpm_box list and particle counts."""
    R = len(boxes)
    barr = (fpm_box * R)(*boxes)
    carr = (_c.c_int32 * R)(*[int(c) for c in counts])
    reps = (fpm_replica * R)()
    b = fpm_batch()
    _check(lib().fpm_batch_plan(int(R), barr, carr, float(r_cell), int(tile_target), reps, _c.byref(b)))
    return reps, b


def fpm_batch_drift_check(batch, d_reps, dt, pos, vel, force, pos_ref, skin, d_rep_flag, stream=None):
    _check(lib().fpm_batch_drift_check(_c.byref(batch), _ptr(d_reps), float(dt), _ptr(pos), _ptr(vel), _ptr(force),
                                       _ptr(pos_ref), float(skin), _ptr(d_rep_flag), _stream(stream)))
    _count(1 if batch.n_total > 0 else 0)


def fpm_batch_celllist_workspace(batch) -> int:
    n = _c.c_size_t()
    _check(lib().fpm_batch_celllist_workspace(_c.byref(batch), _c.byref(n)))
    return n.value


def fpm_batch_celllist_build(batch, d_reps, pos, vel, ids, cell_start, perm, workspace, d_rep_flag=None,
                             d_status=None, stream=None):
    _check(lib().fpm_batch_celllist_build(_c.byref(batch), _ptr(d_reps), _ptr(pos), _ptr(vel), _ptr(ids),
                                          _ptr(cell_start), _ptr(perm), _ptr(workspace), _nbytes(workspace),
                                          _ptr(d_rep_flag), _ptr(d_status), _stream(stream)))
    _count(1)


def fpm_batch_list_bytes(batch, cap: int) -> int:
    n = _c.c_size_t()
    _check(lib().fpm_batch_list_bytes(_c.byref(batch), int(cap), _c.byref(n)))
    return n.value


def fpm_batch_verlet_build(batch, d_reps, pos, cell_start, r_list, cap, list_obj, nn, pos_ref=None,
                           d_rep_flag=None, d_status=None, stream=None):
    _check(lib().fpm_batch_verlet_build(_c.byref(batch), _ptr(d_reps), _ptr(pos), _ptr(cell_start), float(r_list),
                                        int(cap), _ptr(list_obj), _nbytes(list_obj), _ptr(nn), _ptr(pos_ref),
                                        _ptr(d_rep_flag), _ptr(d_status), _stream(stream)))
    _count(2)  # the work list, the scan (which also writes the tile descriptors)


def fpm_batch_verlet_decode(batch, cap, list_obj, nn, out, stream=None):
    _check(lib().fpm_batch_verlet_decode(_c.byref(batch), int(cap), _ptr(list_obj), _ptr(nn), _ptr(out),
                                         _stream(stream)))
    _count(1)


def fpm_batch_workspace(batch) -> int:
    n = _c.c_size_t()
    _check(lib().fpm_batch_workspace(_c.byref(batch), _c.byref(n)))
    return n.value


def fpm_batch_lj_forces_kick(batch, d_reps, pos, list_obj, nn, cap, eps, sigma, rc, force, d_energy, workspace,
                             d_status, vel, dt, stream=None):
    _check(lib().fpm_batch_lj_forces_kick(_c.byref(batch), _ptr(d_reps), _ptr(pos), _ptr(list_obj), _ptr(nn),
                                          int(cap), float(eps), float(sigma), float(rc), _ptr(force),
                                          _ptr(d_energy), _ptr(workspace), _nbytes(workspace), _ptr(d_status),
                                          _ptr(vel), float(dt), _stream(stream)))
    _count(1)


def fpm_batch_step(batch, d_reps, dt, skin, r_list, cap, eps, sigma, rc, pos, vel, force, pos_ref, ids, cell_start,
                   perm, list_obj, nn, d_rep_flag, cell_ws, workspace, d_energy=None, d_status=None, stream=None):
    _check(lib().fpm_batch_step(_c.byref(batch), _ptr(d_reps), float(dt), float(skin), float(r_list), int(cap),
                                float(eps), float(sigma), float(rc), _ptr(pos), _ptr(vel), _ptr(force),
                                _ptr(pos_ref), _ptr(ids), _ptr(cell_start), _ptr(perm), _ptr(list_obj),
                                _nbytes(list_obj), _ptr(nn), _ptr(d_rep_flag), _ptr(cell_ws), _nbytes(cell_ws),
                                _ptr(workspace), _nbytes(workspace), _ptr(d_energy), _ptr(d_status),
                                _stream(stream)))
    _count(1)


def fpm_batch_lj_forces(batch, d_reps, pos, list_obj, nn, cap, eps, sigma, rc, force, d_energy=None,
                        workspace=None, d_status=None, stream=None):
    _check(lib().fpm_batch_lj_forces(_c.byref(batch), _ptr(d_reps), _ptr(pos), _ptr(list_obj), _ptr(nn), int(cap),
                                     float(eps), float(sigma), float(rc), _ptr(force), _ptr(d_energy),
                                     _ptr(workspace), _nbytes(workspace), _ptr(d_status), _stream(stream)))
    _count(1)


# ------------------------------------------------------------------ host-layout transfers

def _host_or_device_ptr(t):
    """A device tensor, or a pinned host tensor (mapped into the device's
    address space): the packed side of fpm_pack_xyz / fpm_unpack_xyz."""
    if t is not None and not isinstance(t, int) and not t.is_cuda:
        if not t.is_pinned():
            raise ValueError("libfpm takes device tensors or pinned host tensors here")
        if not t.is_contiguous():
            raise ValueError("libfpm takes contiguous tensors only")
        return t.data_ptr()
    return _ptr(t)


def fpm_unpack_xyz(n, prec, src_xyz, dst4, stream=None):
    _check(lib().fpm_unpack_xyz(int(n), int(prec), _host_or_device_ptr(src_xyz), _ptr(dst4), _stream(stream)))
    _count(1 if n > 0 else 0)


def fpm_pack_xyz(n, prec, src4, dst_xyz, stream=None):
    _check(lib().fpm_pack_xyz(int(n), int(prec), _ptr(src4), _host_or_device_ptr(dst_xyz), _stream(stream)))
    _count(1 if n > 0 else 0)
