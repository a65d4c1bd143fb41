"""Oracle: a plain FP64 CPU reference of the particle hot path (arXiv 1804.07598).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_1804_07598_gb300``) never imports it and
shares no code with it: the arithmetic lives in ``fpm_oracle.c`` (plain C,
compiled by gcc with ``-ffp-contract=off``); this module marshals numpy
arrays and, for the adjoint, applies the reverse of velocity Verlet step by
step in plain numpy on top of the C force and Hessian-vector routines.

Every function cites the passage of the paper it follows; the conventions the
paper leaves open are listed at the top of ``fpm_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fpm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C part with gcc (no GPU, no nvcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        # OpenMP only spreads the multi-core timing loop (orc_lj_nve_omp);
        # without it that loop runs on one thread
        if subprocess.call(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _P(dtype):
    return np.ctypeslib.ndpointer(dtype=dtype, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i32, f64, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
            sig = {
                "orc_cell_grid": (i32, [_P(np.float64), _P(np.int32), f64, _P(np.int32), _P(np.float32)]),
                "orc_wrap_f32": (None, [i32, _P(np.float32), _P(np.float64), _P(np.int32)]),
                "orc_wrap_f64": (None, [i32, _P(np.float64), _P(np.float64), _P(np.int32)]),
                "orc_cell_index_f32": (i32, [i32, _P(np.float32), _P(np.int32), _P(np.float32),
                                             _P(np.float64), _P(np.uint32)]),
                "orc_cell_index_f64": (i32, [i32, _P(np.float64), _P(np.int32), _P(np.float32),
                                             _P(np.float64), _P(np.uint32)]),
                "orc_counting_sort": (None, [i32, i32, _P(np.uint32), _P(np.uint32), _P(np.uint32)]),
                "orc_neighbors_f32": (i64, [i32, _P(np.float32), _P(np.float64), _P(np.int32), f64, i64,
                                            _P(np.int64), _P(np.uint32)]),
                "orc_neighbors_f64": (i64, [i32, _P(np.float64), _P(np.float64), _P(np.int32), f64, i64,
                                            _P(np.int64), _P(np.uint32)]),
                "orc_neighbors_one_f32": (i32, [i32, _P(np.float32), _P(np.float64), _P(np.int32), f64, i32,
                                                i32, _P(np.uint32)]),
                "orc_neighbors_one_f64": (i32, [i32, _P(np.float64), _P(np.float64), _P(np.int32), f64, i32,
                                                i32, _P(np.uint32)]),
                "orc_max_disp_f32": (i32, [i32, _P(np.float32), _P(np.float32), _P(np.float64), _P(np.int32),
                                           f64, ctypes.POINTER(f64)]),
                "orc_max_disp_f64": (i32, [i32, _P(np.float64), _P(np.float64), _P(np.float64), _P(np.int32),
                                           f64, ctypes.POINTER(f64)]),
                "orc_lj_forces": (i32, [i32, _P(np.float64), _P(np.float64), _P(np.int32), f64, f64, f64, i32,
                                        _P(np.float64), _P(np.float64)]),
                "orc_lj_force_one": (None, [i32, _P(np.float64), _P(np.float64), _P(np.int32), f64, f64, f64,
                                            i32, i32, _P(np.float64)]),
                "orc_vv_kick_drift": (None, [i32, f64, _P(np.float64), _P(np.float64), _P(np.float64),
                                             _P(np.float64), _P(np.int32)]),
                "orc_vv_kick": (None, [i32, f64, _P(np.float64), _P(np.float64)]),
                "orc_lj_nve": (i32, [i32, _P(np.float64), _P(np.float64), _P(np.float64), _P(np.int32), f64, f64,
                                     f64, f64, i32, ctypes.c_void_p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _box(L, periodic):
    L = np.ascontiguousarray(np.broadcast_to(np.asarray(L, np.float64), (3,)))
    p = np.ascontiguousarray(np.broadcast_to(np.asarray(periodic, np.int32), (3,)))
    return L, p


def _pos4(x, dtype):
    x = np.asarray(x)
    if x.ndim != 2 or x.shape[1] not in (3, 4):
        raise ValueError("positions must be [n,3] or [n,4]")
    out = np.zeros((x.shape[0], 4), dtype)
    out[:, :3] = x[:, :3]
    if x.shape[1] == 4:
        out[:, 3] = x[:, 3]
    return out


# --------------------------------------------------------------------------
# Cell lists (Sec. 2; getCellListSym / updateCellListSym in Listing 4.1)
# --------------------------------------------------------------------------

def cell_grid(L, periodic, r_cell):
    """Cells per dimension and the single-precision inverse cell width."""
    Lb, pb = _box(L, periodic)
    nc = np.zeros(3, np.int32)
    inv = np.zeros(3, np.float32)
    if lib().orc_cell_grid(Lb, pb, float(r_cell), nc, inv):
        raise ValueError("box too small for the cutoff (periodic L must exceed 2*r_cell)")
    return nc, inv


def wrap(pos, L, periodic):
    """One-step periodic wrap into [0, L) in the positions' own precision."""
    dtype = np.float32 if np.asarray(pos).dtype == np.float32 else np.float64
    p = _pos4(pos, dtype)
    Lb, pb = _box(L, periodic)
    (lib().orc_wrap_f32 if dtype == np.float32 else lib().orc_wrap_f64)(p.shape[0], p, Lb, pb)
    return p


def cell_index(pos, L, periodic, r_cell):
    """Cell id of every (already wrapped) particle; returns (cell, nbad, nc)."""
    nc, inv = cell_grid(L, periodic, r_cell)
    dtype = np.float32 if np.asarray(pos).dtype == np.float32 else np.float64
    p = _pos4(pos, dtype)
    Lb, _ = _box(L, periodic)
    cell = np.zeros(p.shape[0], np.uint32)
    fn = lib().orc_cell_index_f32 if dtype == np.float32 else lib().orc_cell_index_f64
    nbad = fn(p.shape[0], p, nc, inv, Lb, cell)
    return cell, nbad, nc


def counting_sort(cell, ncell):
    """Stable counting sort (Sec. 3.6 re-sorting): (cell_start[ncell+1], perm)."""
    cell = np.ascontiguousarray(cell, np.uint32)
    cs = np.zeros(int(ncell) + 1, np.uint32)
    perm = np.zeros(cell.shape[0], np.uint32)
    lib().orc_counting_sort(cell.shape[0], int(ncell), cell, cs, perm)
    return cs, perm


def celllist_build(pos, L, periodic, r_cell, vel=None, ids=None):
    """The whole cell-list build: wrap -> cell index -> counting sort -> reorder.

    Returns dict(pos, vel, ids, cell_start, perm, nc, nbad) with every
    per-particle array in sorted order (pos wrapped)."""
    pw = wrap(pos, L, periodic)
    cell, nbad, nc = cell_index(pw, L, periodic, r_cell)
    cs, perm = counting_sort(cell, int(np.prod(nc)))
    out = dict(pos=pw[perm], cell_start=cs, perm=perm, nc=nc, nbad=nbad, cell=cell[perm])
    if vel is not None:
        out["vel"] = np.asarray(vel)[perm]
    if ids is not None:
        out["ids"] = np.asarray(ids)[perm]
    return out


# --------------------------------------------------------------------------
# Verlet lists (Sec. 2, Sec. 4.1)
# --------------------------------------------------------------------------

def neighbors(pos, L, periodic, r_list):
    """Full neighbour lists (CSR) of every particle within r_list, decided in the
    positions' precision. Returns (offsets[n+1] int64, nbr uint32)."""
    dtype = np.float32 if np.asarray(pos).dtype == np.float32 else np.float64
    p = _pos4(pos, dtype)
    Lb, pb = _box(L, periodic)
    n = p.shape[0]
    fn = lib().orc_neighbors_f32 if dtype == np.float32 else lib().orc_neighbors_f64
    offs = np.zeros(n + 1, np.int64)
    cap = max(1, 96 * n)
    while True:
        nbr = np.zeros(cap, np.uint32)
        tot = fn(n, p, Lb, pb, float(r_list), cap, offs, nbr)
        if tot == -2:
            raise ValueError("box too small for the cutoff")
        if tot >= 0:
            return offs, nbr[:tot]
        cap = int(offs[n]) + 1


def neighbors_one(pos, L, periodic, r_list, i):
    """Neighbour set of one particle by an O(n) scan (sampled checks)."""
    dtype = np.float32 if np.asarray(pos).dtype == np.float32 else np.float64
    p = _pos4(pos, dtype)
    Lb, pb = _box(L, periodic)
    fn = lib().orc_neighbors_one_f32 if dtype == np.float32 else lib().orc_neighbors_one_f64
    out = np.zeros(4096, np.uint32)
    k = fn(p.shape[0], p, Lb, pb, float(r_list), int(i), out.shape[0], out)
    if k > out.shape[0]:
        out = np.zeros(k, np.uint32)
        k = fn(p.shape[0], p, Lb, pb, float(r_list), int(i), out.shape[0], out)
    return out[:k]


def max_disp(pos, ref, L, periodic, skin):
    """Rebuild test: (flag, max squared minimum-image displacement)."""
    dtype = np.float32 if np.asarray(pos).dtype == np.float32 else np.float64
    p, r = _pos4(pos, dtype), _pos4(ref, dtype)
    Lb, pb = _box(L, periodic)
    m = ctypes.c_double(0.0)
    fn = lib().orc_max_disp_f32 if dtype == np.float32 else lib().orc_max_disp_f64
    flag = fn(p.shape[0], p, r, Lb, pb, float(skin), ctypes.byref(m))
    return int(flag), float(m.value)


# --------------------------------------------------------------------------
# Lennard-Jones (Sec. 4.1, its potential and Listing 4.1's pair force)
# --------------------------------------------------------------------------

def lj_forces(pos, L, periodic, eps, sigma, rc, mask_f32=False):
    """FP64 forces [n,4] (w = per-particle half pair energy), U, W, pairs.

    mask_f32: decide r < rc in single precision on the (single-precision)
    positions, as a single-precision path does."""
    p = _pos4(pos, np.float64)
    Lb, pb = _box(L, periodic)
    f = np.zeros_like(p)
    out = np.zeros(3, np.float64)
    if lib().orc_lj_forces(p.shape[0], p, Lb, pb, float(eps), float(sigma), float(rc), int(bool(mask_f32)),
                           f, out):
        raise ValueError("box too small for the cutoff")
    return f, float(out[0]), float(out[1]), int(out[2])


def lj_force_one(pos, L, periodic, eps, sigma, rc, i, mask_f32=False):
    p = _pos4(pos, np.float64)
    Lb, pb = _box(L, periodic)
    out = np.zeros(4, np.float64)
    lib().orc_lj_force_one(p.shape[0], p, Lb, pb, float(eps), float(sigma), float(rc), int(bool(mask_f32)),
                           int(i), out)
    return out


# --------------------------------------------------------------------------
# Velocity Verlet (Listing 4.1 time loop, unit mass)
# --------------------------------------------------------------------------

def vv_kick_drift(pos, vel, force, dt, L, periodic):
    """v += dt/2 F; x += dt v; wrap. Returns new (pos, vel) as FP64 [n,4]."""
    p, v, f = _pos4(pos, np.float64), _pos4(vel, np.float64), _pos4(force, np.float64)
    Lb, pb = _box(L, periodic)
    lib().orc_vv_kick_drift(p.shape[0], float(dt), p, v, f, Lb, pb)
    return p, v


def vv_kick(vel, force, dt):
    v, f = _pos4(vel, np.float64), _pos4(force, np.float64)
    lib().orc_vv_kick(v.shape[0], float(dt), v, f)
    return v


def lj_nve(pos, vel, L, periodic, eps, sigma, rc, dt, nsteps, record=True):
    """nsteps of NVE velocity Verlet in FP64. Returns (pos, vel, energies) with
    energies[s] = (KE, U, W, pairs) after step s (s=0: initial state)."""
    p, v = _pos4(pos, np.float64), _pos4(vel, np.float64)
    Lb, pb = _box(L, periodic)
    e = np.zeros((nsteps + 1, 4), np.float64) if record else None
    ptr = e.ctypes.data_as(ctypes.c_void_p) if record else None
    if lib().orc_lj_nve(p.shape[0], p, v, Lb, pb, float(eps), float(sigma), float(rc), float(dt), int(nsteps),
                        ptr):
        raise ValueError("box too small for the cutoff")
    return p, v, e


def threads() -> int:
    """Threads the oracle's OpenMP loops use (1 if built without OpenMP)."""
    L_ = lib()
    L_.orc_threads.restype = ctypes.c_int
    return int(L_.orc_threads())


def lj_forces_omp(pos, L, periodic, eps, sigma, rc):
    """orc_lj_forces on all host cores (each particle's sum from its own
    side).  Returns (force [n,4], (U, W, pairs))."""
    L_ = lib()
    L_.orc_lj_forces_omp.restype = ctypes.c_int
    L_.orc_lj_forces_omp.argtypes = [ctypes.c_int, _P(np.float64), _P(np.float64), _P(np.int32), ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, _P(np.float64), _P(np.float64)]
    p = _pos4(pos, np.float64)
    Lb, pb = _box(L, periodic)
    f = np.zeros_like(p)
    out = np.zeros(3)
    if L_.orc_lj_forces_omp(p.shape[0], p, Lb, pb, float(eps), float(sigma), float(rc), f, out):
        raise ValueError("box too small for the cutoff")
    return f, out


def lj_nve_omp(pos, vel, L, periodic, eps, sigma, rc, dt, nsteps):
    """lj_nve on all host cores (for timing the oracle as a multi-core CPU
    baseline).  Returns (pos, vel)."""
    L_ = lib()
    L_.orc_lj_nve_omp.restype = ctypes.c_int
    L_.orc_lj_nve_omp.argtypes = [ctypes.c_int, _P(np.float64), _P(np.float64), _P(np.float64), _P(np.int32),
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    p, v = _pos4(pos, np.float64), _pos4(vel, np.float64)
    Lb, pb = _box(L, periodic)
    if L_.orc_lj_nve_omp(p.shape[0], p, v, Lb, pb, float(eps), float(sigma), float(rc), float(dt), int(nsteps)):
        raise ValueError("box too small for the cutoff")
    return p, v


# --------------------------------------------------------------------------
# Adjoint of the LJ force and of velocity Verlet (the differentiable workload;
# the paper has no adjoint: these are the chain rule applied to Sec. 4.1's
# force and Listing 4.1's integrator)
# --------------------------------------------------------------------------

def lj_hvp(pos, a, L, periodic, eps, sigma, rc, mask_f32=False):
    """(J a) with J = dF/dx (symmetric), a.dF/d(eps, sigma) and dU/d(eps, sigma).
    Returns (Ja [n,4], dtheta[2], dU[2])."""
    lib_ = lib()
    if not hasattr(lib_.orc_lj_hvp, "_set"):
        lib_.orc_lj_hvp.restype = ctypes.c_int
        lib_.orc_lj_hvp.argtypes = [ctypes.c_int, _P(np.float64), _P(np.float64), _P(np.int32), ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int, _P(np.float64), _P(np.float64),
                                    _P(np.float64), _P(np.float64)]
        lib_.orc_lj_hvp._set = True
    p, av = _pos4(pos, np.float64), _pos4(a, np.float64)
    Lb, pb = _box(L, periodic)
    out = np.zeros_like(p)
    dth = np.zeros(2)
    dU = np.zeros(2)
    if lib_.orc_lj_hvp(p.shape[0], p, Lb, pb, float(eps), float(sigma), float(rc), int(bool(mask_f32)), av, out,
                       dth, dU):
        raise ValueError("box too small for the cutoff")
    return out, dth, dU


def lj_rollout_loss(pos, vel, L, periodic, eps, sigma, rc, dt, nsteps):
    """Loss of the differentiable workload: run nsteps of NVE velocity Verlet
    from (pos, vel) in FP64, then L = U(x_T) + sum_i |F_i(x_T)|^2."""
    p, v, _ = lj_nve(pos, vel, L, periodic, eps, sigma, rc, dt, nsteps, record=False)
    f, U, _, _ = lj_forces(p, L, periodic, eps, sigma, rc)
    return U + float(np.sum(f[:, :3] ** 2))


def lj_rollout_grad(pos, vel, L, periodic, eps, sigma, rc, dt, nsteps):
    """Gradient of lj_rollout_loss w.r.t. the initial positions, the initial
    velocities, eps and sigma, by the reverse of velocity Verlet:
      seed   xbar = -F_T + 2 J(x_T) F_T, vbar = 0,
             thbar = dU/dth + 2 F_T . dF/dth;
      step n+1 -> n:
             xbar += J(x_{n+1}) (dt/2 vbar); thbar += (dt/2 vbar) . dF/dth(x_{n+1})
             vbar += dt xbar
             xbar += J(x_n) (dt/2 vbar);     thbar += (dt/2 vbar) . dF/dth(x_n)
    Returns (loss, xbar0 [n,3], vbar0 [n,3], thbar [2])."""
    p = _pos4(pos, np.float64)
    v = _pos4(vel, np.float64)
    xs = [p.copy()]
    for _ in range(nsteps):
        p, v, _ = lj_nve(p, v, L, periodic, eps, sigma, rc, dt, 1, record=False)
        xs.append(p.copy())
    fT, U, _, _ = lj_forces(xs[-1], L, periodic, eps, sigma, rc)
    loss = U + float(np.sum(fT[:, :3] ** 2))
    fT[:, 3] = 0.0
    JF, dth, dU = lj_hvp(xs[-1], fT, L, periodic, eps, sigma, rc)
    xbar = -fT[:, :3] + 2.0 * JF[:, :3]
    vbar = np.zeros_like(xbar)
    thbar = dU + 2.0 * dth
    h = 0.5 * dt
    for n in range(nsteps - 1, -1, -1):
        a = np.zeros((xbar.shape[0], 4))
        a[:, :3] = h * vbar
        Ja, dth, _ = lj_hvp(xs[n + 1], a, L, periodic, eps, sigma, rc)
        xbar = xbar + Ja[:, :3]
        thbar = thbar + dth
        vbar = vbar + dt * xbar
        a[:, :3] = h * vbar
        Ja, dth, _ = lj_hvp(xs[n], a, L, periodic, eps, sigma, rc)
        xbar = xbar + Ja[:, :3]
        thbar = thbar + dth
    return loss, xbar, vbar, thbar


# --------------------------------------------------------------------------
# Weakly compressible SPH (Sec. 4.2, Eqs. 1-5)
# --------------------------------------------------------------------------

class _SphParams(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("m", ctypes.c_double), ("rho0", ctypes.c_double), ("c0", ctypes.c_double),
                ("gamma", ctypes.c_double), ("alpha", ctypes.c_double), ("eta2", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("kernel", ctypes.c_int)]


def sph_params(h, m, rho0=1000.0, c0=None, gamma=7.0, alpha=0.1, g=(0.0, 0.0, -9.81), kernel="wendland",
               h_swl=0.3):
    """SPH parameter block.  c0 defaults to 20 sqrt(|g| h_swl) (the reading of
    Eq. 4's c_sound = 20); eta^2 = 0.01 h^2."""
    if c0 is None:
        c0 = 20.0 * float(np.sqrt(np.linalg.norm(g) * h_swl))
    p = _SphParams()
    p.h, p.m, p.rho0, p.c0, p.gamma, p.alpha, p.eta2 = h, m, rho0, c0, gamma, alpha, 0.01 * h * h
    for d in range(3):
        p.g[d] = g[d]
    p.kernel = 0 if kernel == "wendland" else 1
    return p


def _sph_sig():
    L_ = lib()
    if getattr(L_, "_sph_set", False):
        return L_
    PP = ctypes.POINTER(_SphParams)
    f64 = ctypes.c_double
    for name, res, args in [
        ("orc_sph_kernel", None, [ctypes.c_int, f64, f64, ctypes.POINTER(f64), ctypes.POINTER(f64)]),
        ("orc_sph_eos", f64, [PP, f64]),
        ("orc_sph_density_sum", ctypes.c_int, [ctypes.c_int, _P(np.float64), _P(np.float64), _P(np.int32), PP,
                                               _P(np.float64)]),
        ("orc_sph_rates", ctypes.c_int, [ctypes.c_int, _P(np.float64), _P(np.float64), _P(np.float64),
                                         _P(np.float64), _P(np.int32), PP, ctypes.c_int, _P(np.float64),
                                         _P(np.float64), _P(np.float64)]),
        ("orc_sph_dt", f64, [PP, _P(np.float64), f64]),
        ("orc_sph_step", f64, [ctypes.c_int, _P(np.float64), _P(np.float64), _P(np.float64), _P(np.float64),
                               _P(np.int32), PP, f64]),
    ]:
        fn = getattr(L_, name)
        fn.restype = res
        fn.argtypes = args
    L_._sph_set = True
    return L_


def sph_kernel(p, r):
    """(W(r), dW/dr(r)) for an array of distances."""
    L_ = _sph_sig()
    r = np.atleast_1d(np.asarray(r, np.float64))
    W, D = np.zeros_like(r), np.zeros_like(r)
    w, d = ctypes.c_double(), ctypes.c_double()
    for k, x in enumerate(r):
        L_.orc_sph_kernel(p.kernel, p.h, float(x), ctypes.byref(w), ctypes.byref(d))
        W[k], D[k] = w.value, d.value
    return W, D


def sph_eos(p, rho):
    L_ = _sph_sig()
    return np.array([L_.orc_sph_eos(ctypes.byref(p), float(x)) for x in np.atleast_1d(rho)])


def sph_density_sum(pos, L, periodic, p):
    L_ = _sph_sig()
    x = _pos4(pos, np.float64)
    Lb, pb = _box(L, periodic)
    rho = np.zeros(x.shape[0])
    if L_.orc_sph_density_sum(x.shape[0], x, Lb, pb, ctypes.byref(p), rho):
        raise ValueError("box too small for the support")
    return rho


def sph_rates(pos, vel, rho, L, periodic, p, mask_f32=False):
    """Eqs. 1-2 rates: (acc [n,4], drho [n], (max|a| fluid, max|mu|)).
    pos[:,3] is the particle type (0 fluid, 1 fixed boundary)."""
    L_ = _sph_sig()
    x, v = _pos4(pos, np.float64), _pos4(vel, np.float64)
    r = np.ascontiguousarray(rho, np.float64)
    Lb, pb = _box(L, periodic)
    acc = np.zeros_like(x)
    dr = np.zeros(x.shape[0])
    dtc = np.zeros(2)
    if L_.orc_sph_rates(x.shape[0], x, v, r, Lb, pb, ctypes.byref(p), int(bool(mask_f32)), acc, dr, dtc):
        raise ValueError("box too small for the support")
    return acc, dr, dtc


def sph_dt(p, dtc, cfl=0.2):
    return float(_sph_sig().orc_sph_dt(ctypes.byref(p), np.ascontiguousarray(dtc, np.float64), float(cfl)))


def sph_step(pos, vel, rho, L, periodic, p, cfl=0.2):
    """One symplectic step; returns (pos, vel, rho, dt)."""
    L_ = _sph_sig()
    x, v = _pos4(pos, np.float64), _pos4(vel, np.float64)
    r = np.array(rho, np.float64)
    Lb, pb = _box(L, periodic)
    dt = L_.orc_sph_step(x.shape[0], x, v, r, Lb, pb, ctypes.byref(p), float(cfl))
    if dt < 0:
        raise ValueError("box too small for the support")
    return x, v, r, dt


# ---------------------------------------------------------------------------
# DEM (Sec. 4.5, Eqs. 9-13): the Silbert grain model with Hertzian contacts.
# The readings the paper leaves open are listed with the C functions.

DEM_MAXC = 32  # contacts per particle the history holds (ORC_DEM_MAXC)


class _DemParams(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("m", ctypes.c_double), ("I", ctypes.c_double), ("kn", ctypes.c_double),
                ("kt", ctypes.c_double), ("gn", ctypes.c_double), ("gt", ctypes.c_double), ("mu", ctypes.c_double),
                ("dt", ctypes.c_double), ("g", ctypes.c_double * 3)]


def dem_params(R=0.06, m=1.0, I=1.44e-3, kn=7.849, kt=2.243, gn=3.401, gt=0.0, mu=0.5, dt=0.01,
               g=(0.0, 0.0, 0.0)):
    """DEM parameter block; defaults are the constants printed in Sec. 4.5
    (gamma_t and mu are not printed: 0 and 0.5, the grain model's usual
    values)."""
    p = _DemParams()
    p.R, p.m, p.I, p.kn, p.kt, p.gn, p.gt, p.mu, p.dt = R, m, I, kn, kt, gn, gt, mu, dt
    for d in range(3):
        p.g[d] = g[d]
    return p


def _dem_sig():
    L_ = lib()
    if getattr(L_, "_dem_set", False):
        return L_
    PP = ctypes.POINTER(_DemParams)
    i64 = ctypes.c_int64
    for name, res, args in [
        ("orc_dem_forces", i64, [ctypes.c_int, _P(np.float64), _P(np.float64), _P(np.float64), _P(np.float64),
                                 _P(np.int32), PP, _P(np.int32), _P(np.uint32), _P(np.float64), _P(np.float64),
                                 _P(np.float64), _P(np.int32), _P(np.uint32), _P(np.float64)]),
        ("orc_dem_leapfrog", None, [ctypes.c_int, _P(np.float64), _P(np.float64), _P(np.float64), _P(np.float64),
                                    _P(np.float64), PP]),
        ("orc_dem_run", i64, [ctypes.c_int, ctypes.c_int, _P(np.float64), _P(np.float64), _P(np.float64),
                              _P(np.float64), _P(np.int32), PP, _P(np.int32), _P(np.uint32), _P(np.float64),
                              _P(np.float64), _P(np.float64)]),
    ]:
        fn = getattr(L_, name)
        fn.restype = res
        fn.argtypes = args
    L_._dem_set = True
    return L_


def dem_empty_history(n):
    """No contacts: (cnt [n], partner [n, MAXC], u [n, MAXC, 3])."""
    return (np.zeros(n, np.int32), np.zeros((n, DEM_MAXC), np.uint32), np.zeros((n, DEM_MAXC, 3)))


def dem_forces(pos, vel, om, L, periodic, p, hist=None):
    """Contact forces and torques at one state (Eqs. 9-12).  `hist` is the
    contact history of the previous step (dem_empty_history for none);
    returns (force [n,4], torque [n,4], new history, ordered contacts).
    pos[:,3] != 0 marks a fixed particle."""
    L_ = _dem_sig()
    x, v, w = _pos4(pos, np.float64), _pos4(vel, np.float64), _pos4(om, np.float64)
    n = x.shape[0]
    Lb, pb = _box(L, periodic)
    h_in = hist if hist is not None else dem_empty_history(n)
    h_out = dem_empty_history(n)
    F, T = np.zeros_like(x), np.zeros_like(x)
    r = L_.orc_dem_forces(n, x, v, w, Lb, pb, ctypes.byref(p), h_in[0], h_in[1], h_in[2], F, T, h_out[0],
                          h_out[1], h_out[2])
    if r == -1:
        raise ValueError("more than %d contacts on a particle" % DEM_MAXC)
    if r < 0:
        raise ValueError("box too small for the contact cell list")
    return F, T, h_out, int(r)


def dem_leapfrog(pos, vel, om, force, torque, p):
    """Eq. 13 (fixed particles, pos[:,3] != 0, stay put); returns new arrays."""
    L_ = _dem_sig()
    x, v, w = _pos4(pos, np.float64), _pos4(vel, np.float64), _pos4(om, np.float64)
    L_.orc_dem_leapfrog(x.shape[0], x, v, w, _pos4(force, np.float64), _pos4(torque, np.float64), ctypes.byref(p))
    return x, v, w


def dem_run(pos, vel, om, L, periodic, p, nsteps, hist=None):
    """nsteps DEM steps; returns (pos, vel, om, force, torque of the last
    step, history, contacts of the last step)."""
    L_ = _dem_sig()
    x, v, w = _pos4(pos, np.float64), _pos4(vel, np.float64), _pos4(om, np.float64)
    n = x.shape[0]
    Lb, pb = _box(L, periodic)
    h = tuple(a.copy() for a in hist) if hist is not None else dem_empty_history(n)
    F, T = np.zeros_like(x), np.zeros_like(x)
    r = L_.orc_dem_run(n, int(nsteps), x, v, w, Lb, pb, ctypes.byref(p), h[0], h[1], h[2], F, T)
    if r == -1:
        raise ValueError("more than %d contacts on a particle" % DEM_MAXC)
    if r < 0:
        raise ValueError("box too small for the contact cell list")
    return x, v, w, F, T, h, int(r)


def dem_history_dict(hist):
    """{(p, q): u_t} of a history triple (test helper)."""
    cnt, ids, u = hist
    return {(int(i), int(ids[i, k])): u[i, k].copy() for i in range(len(cnt)) for k in range(int(cnt[i]))}


# ---------------------------------------------------------------------------
# Particle-mesh interpolation with the M'4 kernel (Sec. 4.4: the vortex
# method's particle-to-mesh and mesh-to-particle interpolations).
# Reading: a periodic mesh of N[d] nodes per dimension at x = i h_d,
# h_d = L_d / N_d; a particle at x (wrapped into [0, L)) touches the nodes
# i0 - 1 .. i0 + 2 (mod N), i0 = floor(x / h), with weight
# prod_d M'4((x_d - i_d h_d) / h_d).  Plain numpy, FP64.

def m4p(x):
    """The M'4 kernel (Monaghan's third-order B-spline correction):
    1 - 5/2 x^2 + 3/2 |x|^3 for |x| < 1, (2 - |x|)^2 (1 - |x|) / 2 for
    1 <= |x| < 2, 0 beyond."""
    a = np.abs(np.asarray(x, np.float64))
    return np.where(a < 1.0, 1.0 - 2.5 * a ** 2 + 1.5 * a ** 3,
                    np.where(a < 2.0, 0.5 * (2.0 - a) ** 2 * (1.0 - a), 0.0))


def _m4_stencil(pos, L, N):
    """Per particle and dimension: the 4 node indices and weights."""
    x = np.asarray(pos, np.float64)[:, :3] % np.asarray(L, np.float64)
    h = np.asarray(L, np.float64) / np.asarray(N)
    s = x / h
    i0 = np.floor(s).astype(np.int64)
    idx, w = [], []
    for d in range(3):
        nodes = i0[:, d:d + 1] + np.arange(-1, 3)[None, :]
        idx.append(np.mod(nodes, N[d]))
        w.append(m4p(s[:, d:d + 1] - nodes))
    return idx, w


def p2m(pos, val, L, N):
    """Particle-to-mesh: mesh[k, j, i] = sum_p val_p W(x_node - x_p); val
    [n, c], mesh [Nz, Ny, Nx, c] (FP64)."""
    N = tuple(int(v) for v in N)
    val = np.asarray(val, np.float64)
    c = val.shape[1]
    mesh = np.zeros((N[2], N[1], N[0], c))
    (ix, iy, iz), (wx, wy, wz) = _m4_stencil(pos, L, N)
    for a in range(4):
        for b in range(4):
            for e in range(4):
                wgt = wx[:, a] * wy[:, b] * wz[:, e]
                np.add.at(mesh, (iz[:, e], iy[:, b], ix[:, a]), wgt[:, None] * val)
    return mesh


def m2p(pos, mesh, L):
    """Mesh-to-particle: val_p = sum_nodes mesh[node] W(x_node - x_p)."""
    mesh = np.asarray(mesh, np.float64)
    N = (mesh.shape[2], mesh.shape[1], mesh.shape[0])
    (ix, iy, iz), (wx, wy, wz) = _m4_stencil(pos, L, N)
    out = np.zeros((np.asarray(pos).shape[0], mesh.shape[3]))
    for a in range(4):
        for b in range(4):
            for e in range(4):
                wgt = wx[:, a] * wy[:, b] * wz[:, e]
                out += wgt[:, None] * mesh[iz[:, e], iy[:, b], ix[:, a]]
    return out
