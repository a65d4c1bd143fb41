"""GPU parity of the batched replicas (R periodic LJ systems of uneven size
advanced together) against the oracle run replica by replica, on identical
positions.

Bit-exact: each replica's cell_start segment, sort permutation, sorted
positions and neighbour sets.  Forces: max_i |F_i - F_i^ref| / RMS(F^ref)
<= 1e-5; U relative <= 1e-6; pair counts exact (FP32 path, the oracle
taking the FP32 box).  The virial W of a small replica is a strongly
cancelling sum (|W| can be a few hundredths of sum |r_ij . F_ij|), and the
rounding of a sum of FP32 pair terms scales with the sum of their magnitudes
(the classical bound for recursive summation), so W is held to
|dW| <= 1e-6 * sum_{i<j} |r_ij . F_ij|."""
import numpy as np
import pytest
import torch

import oracle
from paper_1804_07598_gb300 import autotune, fpm, inputs
from paper_1804_07598_gb300.batch import LJBatch

pytestmark = pytest.mark.gpu

TOL_F, TOL_E = 1e-5, 1e-6
PER = (1, 1, 1)


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def small_ensemble(seed=5, extra=5):
    """Replicas covering one cell per dimension (all-pairs: N=256 at 0.95, N=300
    at 0.70), 3, 3 and 4 cells per dimension, plus log-uniform draws."""
    specs = [(256, 0.95, 0.8), (300, 0.70, 1.2), (700, 0.80, 0.9), (1000, 0.85, 1.4), (1500, 0.75, 0.6)]
    N, rho, T = inputs.batched_replicas(extra, seed, 256, 4000)
    specs += [(int(N[k]), float(rho[k]), float(T[k])) for k in range(extra)]
    return [inputs.replica_state(n, r, t, seed * 100 + k) for k, (n, r, t) in enumerate(specs)]


def fbox(L):
    return np.asarray(L, np.float64).astype(np.float32).astype(np.float64)


def force_error(f, fref):
    rms = np.sqrt(np.mean(np.sum(fref[:, :3] ** 2, axis=1)))
    return np.max(np.linalg.norm(f[:, :3] - fref[:, :3], axis=1)) / rms


def replica_sets(nbr, nn, p0, p1):
    return [np.sort(nbr[:nn[i], i].astype(np.int64) - p0) for i in range(p0, p1)]


def check_lists(b, r, pos_ref, nbr, nn):
    """Replica r's Verlet lists equal the oracle's neighbour sets of the
    positions they were built from."""
    p0, p1 = b.replica_range(r)
    offs, onbr = oracle.neighbors(pos_ref[p0:p1], b.L[r], PER, b.r_list)
    assert np.array_equal(nn[p0:p1].astype(np.int64), np.diff(offs)), r
    got = replica_sets(nbr, nn, p0, p1)
    for i in range(p1 - p0):
        assert np.array_equal(got[i], np.sort(onbr[offs[i]:offs[i + 1]].astype(np.int64))), (r, i)


def abs_virial(x, L, rc):
    """sum_{i<j, r<rc} |r_ij . F_ij| for sigma = eps = 1 (the scale of the
    virial's rounding error), from the oracle's neighbour sets."""
    offs, nbr = oracle.neighbors(x, L, PER, rc)
    i = np.repeat(np.arange(x.shape[0]), np.diff(offs))
    d = x[i, :3].astype(np.float64) - x[nbr.astype(np.int64), :3]
    d -= L * np.rint(d / L)
    ir6 = 1.0 / np.sum(d * d, axis=1) ** 3
    return 0.5 * np.sum(np.abs(24.0 * (2.0 * ir6 * ir6 - ir6)))


def check_forces(b, r, pos, force, energy):
    p0, p1 = b.replica_range(r)
    fref, U, W, pairs = oracle.lj_forces(pos[p0:p1].astype(np.float64), fbox(b.L[r]), PER, b.eps, b.sigma, b.rc,
                                         mask_f32=True)
    err = force_error(force[p0:p1].astype(np.float64), fref)
    assert err <= TOL_F, (r, err)
    assert abs(energy[r, 0] - U) <= TOL_E * abs(U), (r, energy[r, 0], U)
    wscale = abs_virial(pos[p0:p1], fbox(b.L[r]), b.rc)
    assert abs(energy[r, 1] - W) <= TOL_E * wscale, (r, energy[r, 1], W, wscale)
    assert int(round(energy[r, 2])) == pairs, r
    return err


@pytest.mark.parametrize("tile_target,sweep_blocks", [(0, 0), (96, -1), (256, 0), (128, 300)])
def test_batch_build_and_forces_match_oracle(cuda, tile_target, sweep_blocks):
    reps = small_ensemble()
    b = LJBatch(reps, tile_target=tile_target)
    b.set_sweep_blocks(sweep_blocks)
    b.compute_forces()
    torch.cuda.synchronize()
    b.check_status()
    pos, _, ids = b.state_numpy()
    cs, perm = u32(b.cell_start), u32(b.perm)
    nbr, nn = b.neighbor_lists()
    force, energy = b.force.cpu().numpy(), b.energies()
    modes = set()
    for r, (x, v, L) in enumerate(reps):
        p0, p1 = b.replica_range(r)
        o = oracle.celllist_build(x.astype(np.float32), L, PER, b.r_list)
        c0, ncell = b.reps[r].c0, b.reps[r].grid.ncell
        assert ncell == int(np.prod(o["nc"]))
        modes.add(int(o["nc"][0]))
        assert np.array_equal(cs[c0:c0 + ncell + 1].astype(np.int64) - p0, o["cell_start"].astype(np.int64)), r
        assert np.array_equal(perm[p0:p1].astype(np.int64) - p0, o["perm"].astype(np.int64)), r
        assert np.array_equal(ids[p0:p1].astype(np.int64) - p0, o["perm"].astype(np.int64)), r
        assert np.array_equal(pos[p0:p1, :3], o["pos"][:, :3]), r
        check_lists(b, r, pos, nbr, nn)
        check_forces(b, r, pos, force, energy)
    assert 1 in modes and 3 in modes  # all-pairs and stencil replicas both covered


def test_batch_forces_deterministic(cuda):
    b = LJBatch(small_ensemble(seed=9))
    f1, e1 = b.force.clone(), b.energy.clone()
    b.compute_forces()
    assert torch.equal(f1, b.force) and torch.equal(e1, b.energy)


def test_batch_gated_rebuild_touches_only_flagged_replicas(cuda):
    reps = small_ensemble(seed=7)
    b = LJBatch(reps)
    R = b.R
    flagged = [1, 3, R - 1]
    # move the flagged replicas' particles so that their cells change
    for r in flagged:
        p0, p1 = b.replica_range(r)
        b.pos[p0:p1, 0] += 0.9
    torch.cuda.synchronize()
    cs0, pos0 = u32(b.cell_start).copy(), b.pos.cpu().numpy().copy()
    nbr0, nn0 = b.neighbor_lists()
    nr0 = fpm.read_status(b.status).nrebuild
    f = torch.zeros(R, dtype=torch.int32, device="cuda")
    f[flagged] = 1
    b.flags.copy_(f)
    b.rebuild(gated=True)
    b.compute_forces()
    torch.cuda.synchronize()
    st = b.check_status()
    assert st.nrebuild - nr0 == len(flagged)
    assert int(b.flags.abs().sum().item()) == 0
    cs, pos = u32(b.cell_start), b.pos.cpu().numpy()
    nbr, nn = b.neighbor_lists()
    pref = b.pos_ref.cpu().numpy()
    force, energy = b.force.cpu().numpy(), b.energies()
    for r in range(R):
        p0, p1 = b.replica_range(r)
        c0, ncell = b.reps[r].c0, b.reps[r].grid.ncell
        if r in flagged:
            o = oracle.celllist_build(pos0[p0:p1], b.L[r], PER, b.r_list)
            assert np.array_equal(cs[c0:c0 + ncell + 1].astype(np.int64) - p0, o["cell_start"].astype(np.int64))
            assert np.array_equal(pos[p0:p1, :3], o["pos"][:, :3])
            assert np.array_equal(pref[p0:p1], pos[p0:p1])
        else:
            assert np.array_equal(cs[c0:c0 + ncell + 1], cs0[c0:c0 + ncell + 1]), r
            assert np.array_equal(pos[p0:p1], pos0[p0:p1]), r
            assert np.array_equal(nn[p0:p1], nn0[p0:p1]), r
            assert np.array_equal(nbr[:, p0:p1], nbr0[:, p0:p1]), r  # the list entries are untouched
        check_lists(b, r, pref, nbr, nn)
        check_forces(b, r, pos, force, energy)


def test_batch_steps_keep_lists_valid(cuda):
    """Steps under a CUDA graph: replicas rebuild on their own schedule; after
    the run every replica's list equals the oracle's sets at its reference
    positions and the forces equal the oracle's at the current positions."""
    b = LJBatch(small_ensemble(seed=11))
    b.step(3)
    b.capture(steps_per_graph=2)
    nr0 = fpm.read_status(b.status).nrebuild
    b.run(60)
    torch.cuda.synchronize()
    st = b.check_status()
    assert st.nrebuild > nr0  # some replicas were rebuilt
    assert int(b.flags.abs().sum().item()) == 0
    pos, vel, _ = b.state_numpy()
    pref = b.pos_ref.cpu().numpy()
    nbr, nn = b.neighbor_lists()
    force, energy = b.force.cpu().numpy(), b.energies()
    for r in range(b.R):
        p0, p1 = b.replica_range(r)
        # every particle within skin/2 of its reference (else it would have been rebuilt)
        d = pos[p0:p1, :3].astype(np.float64) - pref[p0:p1, :3]
        assert np.max(np.sum(d * d, axis=1)) <= (0.5 * b.skin) ** 2 * (1 + 1e-5)
        check_lists(b, r, pref, nbr, nn)
        check_forces(b, r, pos, force, energy)
        # momentum of each replica stays ~0 (pairwise forces, zero initial momentum)
        assert np.max(np.abs(vel[p0:p1, :3].astype(np.float64).sum(0))) < 1e-3 * (p1 - p0) ** 0.5


@pytest.mark.parametrize("config", ["tuned", "bench"])
def test_batch_full_ensemble_sampled(cuda, config):
    """The 512-replica ensemble (about 1.9M particles) under a CUDA graph,
    in the autotuned launch configuration ("tuned") and in the one the
    benchmark's tuner picks on GB300 ("bench": 230 particles per tile, one
    block per tile): sampled replicas (smallest, largest and three random)
    against the oracle after 20 steps."""
    reps, N, rho, T = inputs.ensemble()
    b = LJBatch(reps)
    if config == "tuned":
        res = autotune.tune_batch(b, steps=6, warmup=2, tile_targets=(128, 170), sweep_blocks=(0, -1),
                                  use_cache=False)
        assert res["config"]["tile_target"] in (128, 170)
    else:
        b.plan(230, -1)
    b.step(2)
    b.capture(steps_per_graph=1)
    b.run(20)
    torch.cuda.synchronize()
    b.check_status()
    pos, _, _ = b.state_numpy()
    pref = b.pos_ref.cpu().numpy()
    nbr, nn = b.neighbor_lists()
    force, energy = b.force.cpu().numpy(), b.energies()
    rng = np.random.default_rng(3)
    sample = sorted({int(np.argmin(N)), int(np.argmax(N)), *rng.choice(b.R, 3, replace=False).tolist()})
    for r in sample:
        check_lists(b, r, pref, nbr, nn)
        check_forces(b, r, pos, force, energy)


def test_batch_edge_cases(cuda):
    """A replica with no particles between two others, a batch of one
    replica, and a replica whose box is just above the smallest legal one
    (L = 5.61 > 2 r_list (1 + 2^-10) = 5.6055: one cell, all pairs): lists and
    forces still match the oracle and the empty replica's energies are zero."""
    L = 5.61
    tiny = inputs.replica_state(64, 64 / L ** 3, 1.0, 5)
    big = inputs.replica_state(300, 0.9, 1.0, 6)
    empty = (np.zeros((0, 4)), np.zeros((0, 4)), np.array([8.0, 8.0, 8.0]))
    for reps in ([big, empty, tiny], [big]):
        b = LJBatch(reps)
        b.step(2)
        b.compute_forces()
        torch.cuda.synchronize()
        b.check_status()
        pos, _, _ = b.state_numpy()
        pref = b.pos_ref.cpu().numpy()
        nbr, nn = b.neighbor_lists()
        force, energy = b.force.cpu().numpy(), b.energies()
        for r in range(b.R):
            p0, p1 = b.replica_range(r)
            if p1 == p0:
                assert np.all(energy[r] == 0.0)
                continue
            check_lists(b, r, pref, nbr, nn)
            check_forces(b, r, pos, force, energy)


def test_batch_forces_kick_equals_split(cuda):
    """fpm_batch_lj_forces_kick writes the forces and energies of
    fpm_batch_lj_forces and the velocities of a separate half-kick, bit for
    bit (replicas with walls on every side and all-pairs replicas included)."""
    b = LJBatch(small_ensemble())
    b.compute_forces()
    torch.cuda.synchronize()
    f0, e0, v0 = b.force.clone(), b.energy.clone(), b.vel.clone()
    fpm.fpm_vv_step(b.boxes[0], b.n, fpm.FPM_F32, 1, b.dt, None, b.vel, b.force)
    v_split = b.vel.clone()
    b.vel.copy_(v0)
    b.force.zero_()
    b.forces_and_kick()
    torch.cuda.synchronize()
    b.check_status()
    assert torch.equal(b.force, f0) and torch.equal(b.energy, e0) and torch.equal(b.vel, v_split)


@pytest.mark.parametrize("threads", [128, 512])
def test_batch_sweep_threads(cuda, threads):
    """The force sweep's block size is a launch shape only: 128 or 512 threads
    per block give the forces of the default 256 bit for bit (one thread per
    particle, the same list order) and the energies within rounding (the
    per-thread partial sums group differently when a tile is larger than the
    block)."""
    b = LJBatch(small_ensemble())
    b.compute_forces()
    torch.cuda.synchronize()
    f0, e0 = b.force.clone(), b.energy.clone()
    b.set_sweep_threads(threads)
    b.force.zero_()
    b.compute_forces()
    torch.cuda.synchronize()
    b.check_status()
    assert torch.equal(b.force, f0)
    e, e0 = b.energy.cpu().numpy(), e0.cpu().numpy()
    assert np.all(np.abs(e[:, 0] - e0[:, 0]) <= 1e-6 * np.abs(e0[:, 0]))
    assert np.array_equal(e[:, 2], e0[:, 2])


def batch_state(b):
    """Everything a step writes, as host arrays (the list object from byte 64:
    its header holds launch counters and the grid barrier's generation)."""
    torch.cuda.synchronize()
    out = {k: getattr(b, k).cpu().numpy().copy() for k in
           ("pos", "vel", "force", "pos_ref", "ids", "perm", "cell_start", "nn", "energy", "flags")}
    nbr = b.nbr.cpu().numpy()
    out["list"] = nbr[64:].copy()
    out["nwork"] = nbr[:4].copy()
    return out


@pytest.mark.parametrize("skin,sweep_blocks,minb", [(0.3, 0, 0), (0.05, 0, 2), (0.05, 7, 3)])
def test_batch_one_launch_step_equals_split(cuda, skin, sweep_blocks, minb):
    """fpm_batch_step (one cooperative launch: drift, gated cell lists and
    Verlet lists, forces and the closing kick, separated by grid barriers)
    leaves every array exactly as the four separate calls do, over eager and
    graph-captured steps in which replicas rebuild on their own schedule (a
    small skin rebuilds most replicas most steps), with a grid of a few
    blocks (each taking many replicas, cells and tiles), and over steps in
    which no replica is flagged (the rebuild phases skipped)."""
    reps = small_ensemble(seed=13)
    a = LJBatch(reps, skin=skin, fused=True)
    b = LJBatch(reps, skin=skin, fused=False)
    a.batch.sweep_blocks = sweep_blocks
    a.set_step_blocks_per_sm(minb)
    st0 = fpm.read_status(a.status).nrebuild
    for _ in range(4):
        a.step(1)
        b.step(1)
    sa, sb = batch_state(a), batch_state(b)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    a.capture(steps_per_graph=2)
    b.capture(steps_per_graph=2)
    a.run(8)
    b.run(8)
    sa, sb = batch_state(a), batch_state(b)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    ta, tb = a.check_status(), b.check_status()
    assert ta.nrebuild == tb.nrebuild and ta.nrebuild > st0
    assert ta.max_nn == tb.max_nn
    assert not sa["flags"].any()
    # steps in which no replica is flagged (dt = 0: nobody moves)
    a.dt = b.dt = 0.0
    for _ in range(2):
        a.step(1)
        b.step(1)
    sa, sb = batch_state(a), batch_state(b)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    assert a.check_status().nrebuild == ta.nrebuild


def test_batch_one_launch_step_barrier_timeout(cuda):
    """A grid barrier that can never complete (its arrival counter planted far
    past the grid size, so no block is ever the last) gives up after its
    bounded wait: the launch returns with FPM_FLAG_TIMEOUT latched and the
    context still usable; after the documented recovery (workspaces
    zero-filled, full cell and Verlet builds, which reset the barrier) the
    next steps again equal the separate calls."""
    reps = small_ensemble(seed=17, extra=2)
    a = LJBatch(reps, fused=True)
    b = LJBatch(reps, fused=False)
    hdr = a.nbr[:64].view(torch.int32)
    hdr[8] = 1 << 30
    a.step(1)
    torch.cuda.synchronize()
    st = fpm.read_status(a.status)
    assert st.flags & fpm.FPM_FLAG_TIMEOUT
    assert fpm.fpm_status_from_device(st) == fpm.FPM_ERR_TIMEOUT
    for k in ("pos", "vel", "force", "ids"):
        getattr(a, k).copy_(getattr(b, k))
    a.status.zero_()
    a.flags.zero_()
    a.ws_cell.zero_()
    a.ws_red.zero_()
    a.rebuild()
    a.compute_forces()
    b.rebuild()
    b.compute_forces()
    assert int(hdr[8].item()) == 0
    for _ in range(3):
        a.step(1)
        b.step(1)
    sa, sb = batch_state(a), batch_state(b)
    for k in ("pos", "vel", "force", "ids", "energy", "nn", "list"):
        assert np.array_equal(sa[k], sb[k]), k
    a.check_status()


def test_batch_one_launch_step_many_flagged_replicas(cuda):
    """Hundreds of replicas flagged in one step, more than the per-block
    tables of flagged replicas hold in shared memory: the step's binning,
    scatter and gather then walk every particle and cell of the batch (the
    replica of each read from the cell workspace) instead, with the same
    results as the separate calls; tiles beyond the staging capacity read
    their neighbourhoods from global memory on both sides."""
    reps = [inputs.replica_state(256, 0.9, 1.0, 900 + r) for r in range(700)]
    reps += [inputs.replica_state(3000, 0.8, 1.0, 1900 + r) for r in range(20)]
    a = LJBatch(reps, skin=0.02, fused=True)
    b = LJBatch(reps, skin=0.02, fused=False)
    # a small staging capacity (the larger replicas' tiles then read their
    # neighbourhoods from global memory), which also bounds the tables
    a.batch.stage_cap = b.batch.stage_cap = 384
    nr0 = fpm.read_status(a.status).nrebuild
    for _ in range(3):
        a.step(1)
        b.step(1)
    sa, sb = batch_state(a), batch_state(b)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    ta = a.check_status()
    per_step = (ta.nrebuild - nr0) / 3
    # the tables: 12 B per flagged replica (+ 8 B) after B2's counters, within
    # the step's dynamic shared memory (the larger of the counters and the staging)
    stage = min((a.batch.stage_cap + 31) // 32 * 32, 200 * 1024 // 16 // 32 * 32) * 16
    cnt = (a.batch.max_ncell + 1) * 4
    capacity = (max(stage, cnt) - cnt - 16 - 8) // 12
    assert per_step > capacity, (per_step, capacity)
    assert ta.spilled > 0
