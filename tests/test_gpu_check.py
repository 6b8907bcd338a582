"""The bounds-checked build (-DFSIM_CHECK, libfsim_check.so) on real solves.

The checked library tests its data-dependent indices before use. These are
the force gather's tet slots, the supernodal solves' off-diagonal rows and
the contact-list entries of the reduced systems. It records the first
failure in a status word instead of trapping.

The test runs these solves through the checked library:

* a single-frame float64 solve;
* a single-frame mixed solve;
* a lock-step batch.

Each must leave the word at 0 and give the frames of the normal library.
The normal library reports that it has no checks.
"""
import numpy as np
import pytest

from paper_2312_02999_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsim():
    from paper_2312_02999_gb300 import build
    build.build()
    build.build(check=True)
    from paper_2312_02999_gb300 import fsim as f
    return f


def _solves(fsim, ctx, mesh):
    act = I.slab_actuation(mesh, seed=3)
    rng = np.random.default_rng(4)
    x0 = mesh.rest.copy()
    free = mesh.pinned == 0
    x0[free] += 1e-4 * rng.standard_normal((int(free.sum()), 3))
    x0[(mesh.rest[:, 2] > mesh.rest[:, 2].mean()) & free, 2] -= 0.0033
    m = ctx.upload(mesh)
    m.prefactor(fsim.params_for(mesh))
    m.set_actuation(act.fiber, act.stretch)
    out = []
    for prec in (fsim.FP64, fsim.MIXED):
        rc, st = m.solve_frame(x_init=x0, precision=prec)
        assert rc == 0 and st["contacts"] > 0
        out.append(m.positions())
    rc, xs, sts = fsim.solve_batch(ctx, [(m, act.fiber, act.stretch, x0)] * 3, max_frames=2)
    assert rc == 0 and all(s["status"] == 0 for s in sts)
    out += xs
    return out


def test_checked_build_runs_clean_and_matches(fsim):
    mesh = I.two_slabs(6, 6, 2, gap=0.004)
    ctx = fsim.Context(0)
    try:
        assert ctx.check_status() == (False, 0)
        ref = _solves(fsim, ctx, mesh)
    finally:
        ctx.close()
    cctx = fsim.Context(0, lib_path=fsim.LIB_PATH.replace("libfsim.so", "libfsim_check.so"))
    try:
        assert cctx.check_status() == (True, 0)
        got = _solves(fsim, cctx, mesh)
        enabled, word = cctx.check_status()
    finally:
        cctx.close()
    assert enabled and word == 0, hex(word)
    diag = float(np.linalg.norm(mesh.rest.max(0) - mesh.rest.min(0)))
    for a, b in zip(got, ref):
        assert np.abs(a - b).max() <= 1e-12 * diag
