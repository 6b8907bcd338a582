"""Request server and batched solves (continuous batching over workspace
slots): every result is the same alone and in the mix.

Requests for two meshes with different actuations and start states are
submitted together to a server whose workers solve them concurrently; each
result is compared with the same request solved alone through
fsim_solve_frame on the mesh's own workspace.  The order of floating-point
atomics differs between any two runs, so positions are compared at the
frame tolerances (1e-9 of the bounding-box diagonal in float64, 1e-6 in
mixed precision), and the iteration counts must match.
"""
import numpy as np
import pytest

from paper_2312_02999_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2312_02999_gb300 import build
    build.build()
    from paper_2312_02999_gb300 import fsim
    ctx = fsim.Context(0)
    meshes = []
    for (nx, ny, nz, seed) in ((4, 4, 2, 11), (5, 4, 2, 12)):
        mesh = I.two_slabs(nx, ny, nz, gap=0.004)
        m = ctx.upload(mesh)
        m.prefactor(fsim.params_for(mesh))
        acts = [I.slab_actuation(mesh, seed=seed + 10 * k) for k in range(3)]
        meshes.append((mesh, m, acts))
    yield fsim, ctx, meshes
    ctx.close()


def _diag(mesh):
    return float(np.linalg.norm(mesh.rest.max(0) - mesh.rest.min(0)))


def _requests(meshes):
    reqs = []
    rng = np.random.default_rng(5)
    for mi, (mesh, m, acts) in enumerate(meshes):
        for k, act in enumerate(acts):
            x0 = None
            if k == 2:    # an explicit, perturbed start state
                x0 = mesh.rest.copy()
                free = mesh.pinned == 0
                x0[free] += 1e-4 * rng.standard_normal((int(free.sum()), 3))
            for prec in (0, 1):
                reqs.append((mi, act, x0, prec))
    return reqs


def _alone(fsim, meshes, req):
    mi, act, x0, prec = req
    mesh, m, _ = meshes[mi]
    m.set_actuation(act.fiber, act.stretch)
    rc, st = m.solve_frame(x_init=mesh.rest if x0 is None else x0, precision=prec)
    return rc, m.positions(), st


def _tol(mesh, prec):
    return (1e-9 if prec == 0 else 1e-6) * _diag(mesh)


def test_server_results_match_solo_solves(setup):
    fsim, ctx, meshes = setup
    reqs = _requests(meshes)
    solo = [_alone(fsim, meshes, r) for r in reqs]
    with fsim.Server(ctx, workers=3) as srv:
        tickets = [srv.submit(meshes[mi][1], act.fiber, act.stretch, x0, prec)
                   for (mi, act, x0, prec) in reqs]
        outs = [srv.wait(t) for t in tickets]
        info = srv.info()
    assert info["completed"] == len(reqs) and info["queued"] == 0
    assert info["peak_running"] >= 2          # solves really overlapped
    for (mi, act, x0, prec), (rc0, x_solo, st0), (rc, x, st, lat, q) in zip(reqs, solo, outs):
        mesh = meshes[mi][0]
        assert rc == 0 and rc0 == 0
        assert st["iterations"] == st0["iterations"]
        assert np.abs(x - x_solo).max() <= _tol(mesh, prec)
        assert lat >= q >= 0.0


def test_memory_budget_serialises_slots(setup):
    fsim, ctx, meshes = setup
    reqs = _requests(meshes)[:4]
    solo = [_alone(fsim, meshes, r) for r in reqs]
    # a budget of one slot: requests of the other mesh evict it; all finish
    ws = max(mesh_m.info()["workspace_bytes"] for (_, mesh_m, _) in meshes)
    with fsim.Server(ctx, workers=2, mem_budget_bytes=int(1.5 * ws)) as srv:
        tickets = [srv.submit(meshes[mi][1], act.fiber, act.stretch, x0, prec)
                   for (mi, act, x0, prec) in reqs]
        outs = [srv.wait(t) for t in tickets]
        info = srv.info()
    assert info["peak_slots"] == 1 and info["peak_running"] == 1
    for (mi, _, _, prec), (_, x_solo, _), (rc, x, _, _, _) in zip(reqs, solo, outs):
        assert rc == 0
        assert np.abs(x - x_solo).max() <= _tol(meshes[mi][0], prec)


def test_solve_frames_batched_form(setup):
    fsim, ctx, meshes = setup
    reqs = _requests(meshes)
    solo = [_alone(fsim, meshes, r) for r in reqs]
    batch = [(meshes[mi][1], act.fiber, act.stretch, x0, prec) for (mi, act, x0, prec) in reqs]
    rc, xs, stats = fsim.solve_frames(ctx, batch, workers=4)
    assert rc == 0
    for (mi, _, _, prec), (_, x_solo, st0), x, st in zip(reqs, solo, xs, stats):
        assert st["status"] == 0 and st["iterations"] == st0["iterations"]
        assert np.abs(x - x_solo).max() <= _tol(meshes[mi][0], prec)


def test_server_rejects_bad_requests(setup):
    fsim, ctx, meshes = setup
    mesh, m, acts = meshes[0]
    bad = acts[0].stretch.copy()
    bad[3] = -1.0
    with fsim.Server(ctx, workers=1, mem_budget_bytes=1024) as small:
        with pytest.raises(fsim.FsimError) as e:     # one workspace exceeds the budget
            small.submit(m, acts[0].fiber, acts[0].stretch)
        assert e.value.status == fsim.FSIM_ENOMEM
    raw = fsim.Server(ctx, workers=1)
    try:
        with pytest.raises(fsim.FsimError) as e:
            raw.submit(m, acts[0].fiber, bad)
        assert e.value.status == fsim.FSIM_ENONFINITE
        other = I.two_slabs(3, 3, 2, gap=0.004)
        m2 = ctx.upload(other)                  # not prefactored
        a2 = I.slab_actuation(other, seed=1)
        with pytest.raises(fsim.FsimError) as e:
            raw.submit(m2, a2.fiber, a2.stretch)
        assert e.value.status == fsim.FSIM_ENOT_READY
    finally:
        raw.close()


def test_batch_server_results_match_solo_solves(setup):
    # batch workers: lock-step batches of up to 3 frames per mesh; the six
    # mixed requests of each mesh pass through three slots, so later requests
    # are admitted into the slots of finished frames at iteration boundaries
    fsim, ctx, meshes = setup
    reqs = [r for r in _requests(meshes) if r[3] == 1] * 2
    solo = [_alone(fsim, meshes, r) for r in reqs]
    with fsim.Server(ctx, workers=2, batch_frames=3) as srv:
        tickets = [srv.submit(meshes[mi][1], act.fiber, act.stretch, x0, prec)
                   for (mi, act, x0, prec) in reqs]
        outs = [srv.wait(t) for t in tickets]
        info = srv.info()
        # a batch server serves the mixed precision only
        mesh, m, acts = meshes[0]
        with pytest.raises(fsim.FsimError) as e:
            srv.submit(m, acts[0].fiber, acts[0].stretch, None, fsim.FP64)
        assert e.value.status == fsim.FSIM_EINVAL
    assert info["completed"] == len(reqs) and info["queued"] == 0
    for (mi, act, x0, prec), (rc0, x_solo, st0), (rc, x, st, lat, q) in zip(reqs, solo, outs):
        mesh = meshes[mi][0]
        assert rc == 0 and rc0 == 0
        assert abs(st["iterations"] - st0["iterations"]) <= 2
        assert np.abs(x - x_solo).max() <= _tol(mesh, prec)
        assert lat >= q >= 0.0
