"""Helpers for the GPU parity tests: run libfpm calls on torch device tensors
and bring the results back as numpy."""
import numpy as np
import torch

from paper_1804_07598_gb300 import fpm


def dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def tdtype(prec):
    return torch.float32 if prec == "f32" else torch.float64


def npdtype(prec):
    return np.float32 if prec == "f32" else np.float64


def fprec(prec):
    return fpm.FPM_F32 if prec == "f32" else fpm.FPM_F64


def status_tensor():
    return torch.zeros(fpm.STATUS_BYTES // 4, dtype=torch.int32, device="cuda")


def gpu_celllist(pos4, L, periodic, r_cell, prec, vel4=None, ids=None, inplace=False):
    """Run fpm_celllist_build; returns dict of numpy results."""
    n = pos4.shape[0]
    td = tdtype(prec)
    box = fpm.make_box(L, periodic)
    grid = fpm.fpm_grid_make(box, r_cell, n)
    p_in = dev(pos4, td)
    v_in = dev(vel4, td) if vel4 is not None else None
    i_in = dev(np.asarray(ids, np.uint32).view(np.int32), torch.int32) if ids is not None else None
    if inplace:
        p_out, v_out, i_out = p_in, v_in, (i_in if i_in is not None else torch.zeros(max(n, 1), dtype=torch.int32,
                                                                                       device="cuda"))
    else:
        p_out = torch.full_like(p_in, -7.0)
        v_out = torch.full_like(v_in, -7.0) if v_in is not None else None
        i_out = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    cs = torch.full((grid.ncell + 1,), -1, dtype=torch.int32, device="cuda")
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    ws = torch.full((fpm.fpm_celllist_workspace(n, grid, fprec(prec)),), 0x5A, dtype=torch.uint8, device="cuda")
    st = status_tensor()
    fpm.fpm_celllist_build(box, grid, n, fprec(prec), p_in, v_in, i_in, p_out, v_out, i_out, cs, perm, ws, st)
    torch.cuda.synchronize()
    out = dict(pos=p_out.cpu().numpy()[:n], cell_start=u32(cs), perm=u32(perm)[:n], ids=u32(i_out)[:n],
               status=fpm.read_status(st), grid=grid, box=box,
               dev=dict(pos=p_out, cs=cs, perm=perm, ids=i_out, vel=v_out))
    if v_out is not None:
        out["vel"] = v_out.cpu().numpy()[:n]
    return out


def gpu_verlet(res, r_list, prec, cap=None, gate=None):
    """Run fpm_verlet_build on the sorted output of gpu_celllist and decode the
    list into particle indices."""
    n = res["pos"].shape[0]
    cap = cap or 160
    ld = fpm.fpm_nbr_ld(n)
    lst = torch.full((fpm.fpm_verlet_list_bytes(n, res["grid"], cap),), 0xA5, dtype=torch.uint8, device="cuda")
    nn = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    ref = torch.zeros_like(res["dev"]["pos"])
    st = status_tensor()
    fpm.fpm_verlet_build(res["box"], res["grid"], n, fprec(prec), res["dev"]["pos"], res["dev"]["cs"], r_list, cap,
                         lst, nn, ref, st, gate)
    nbr = torch.full((max(1, cap * ld),), -1, dtype=torch.int32, device="cuda")
    fpm.fpm_verlet_decode(res["grid"], n, cap, lst, nn, nbr)
    torch.cuda.synchronize()
    return dict(nbr=u32(nbr)[:cap * ld].reshape(cap, ld) if n else np.zeros((cap, 0), np.uint32),
                nn=u32(nn)[:n], ref=ref, status=fpm.read_status(st), cap=cap, ld=ld,
                dev=dict(list=lst, nn=nn))


def ell_sets(v, n):
    nn = v["nn"]
    return [set(v["nbr"][:nn[i], i].tolist()) for i in range(n)]


def csr_sets(offs, nbr):
    return [set(nbr[offs[i]:offs[i + 1]].tolist()) for i in range(len(offs) - 1)]


def ell_equal_csr(v, offs, onbr, n):
    """Exact equality of the GPU ELL list and the oracle CSR lists as sets
    (vectorised: sort each row)."""
    nn = v["nn"].astype(np.int64)
    if not np.array_equal(nn, np.diff(offs)):
        bad = np.nonzero(nn != np.diff(offs))[0]
        return False, f"counts differ at {bad[:10]} (gpu {nn[bad[:10]]} oracle {np.diff(offs)[bad[:10]]})"
    cap = v["nbr"].shape[0]
    m = int(nn.max()) if n else 0
    g = v["nbr"][:m, :n].T.astype(np.int64).copy()
    mask = np.arange(m)[None, :] >= nn[:, None]
    g[mask] = np.iinfo(np.int64).max
    g.sort(axis=1)
    o = np.full((n, m), np.iinfo(np.int64).max, np.int64)
    rows = np.repeat(np.arange(n), nn)
    cols = np.arange(len(onbr)) - np.repeat(offs[:-1], nn)
    o[rows, cols] = onbr
    o.sort(axis=1)
    if not np.array_equal(g, o):
        bad = np.nonzero(np.any(g != o, axis=1))[0]
        return False, f"sets differ at {bad[:10]}"
    return True, ""
