"""A frame solved on an automatically selected collision region, GPU against oracle.

fsim_select_region picks the proxy of the 5k-vertex face (the two lips across
the mouth slit, 2 mm radius, 4 surface rings); the GPU solves frame 20 of
sequence 3 from the rest pose on that proxy, float64 and mixed, and the oracle
solves the same frame on the same proxy (its own selection, which the CPU
tests show equal to the library's).  Positions must agree within 1e-9
(float64) and 1e-6 (mixed) of the bounding-box diagonal, iteration counts
within 2.
"""
import dataclasses

import numpy as np
import pytest

from oracle import region as R
from oracle import solver as S
from paper_2312_02999_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_frame_on_the_automatic_region_matches_the_oracle():
    from paper_2312_02999_gb300 import build
    build.build()
    from paper_2312_02999_gb300 import fsim
    mesh = I.face_shell(n_target=5000)
    tris, verts = fsim.select_region(mesh.rest, mesh.tets, mesh.pinned, 0.002, 4)
    to, vo = R.select_region(mesh.rest, mesh.tets, mesh.pinned, 0.002, 4)
    assert np.array_equal(tris, to) and np.array_equal(verts, vo) and len(verts) > 0
    auto = dataclasses.replace(mesh, proxy_tris=tris,
                               W_rowptr=np.arange(len(verts) + 1, dtype=np.int64),
                               W_col=verts.astype(np.int32), W_val=np.ones(len(verts)))
    field = I.bump_field(mesh, seed=2)
    act = I.bump_actuation(field, I.keyframe_coeffs(seed=3)[20])
    pr = S.Problem(auto.rest, auto.tets, auto.pinned, auto.proxy_tris, auto.W_rowptr, auto.W_col,
                   auto.W_val, S.Params(dhat=mesh.dhat, tol_abs=mesh.tol_abs, tol_rel=mesh.tol_rel))
    pr.set_actuation(act.fiber, act.stretch)
    xo, so = pr.solve_frame(mesh.rest)
    assert so.status == 0 and max(so.contacts) > 0
    diag = float(np.linalg.norm(mesh.rest.max(0) - mesh.rest.min(0)))
    with fsim.Context(0) as ctx:
        m = ctx.upload(auto)
        m.prefactor(fsim.params_for(auto))
        assert abs(m.info()["kappa"] - pr.kappa) <= 1e-12 * pr.kappa
        m.set_actuation(act.fiber, act.stretch)
        for prec, tol in ((fsim.FP64, 1e-9), (fsim.MIXED, 1e-6)):
            rc, st = m.solve_frame(x_init=mesh.rest, precision=prec)
            assert rc == 0 and st["n_c_max"] > 0
            err = float(np.abs(m.positions() - xo).max()) / diag
            assert err <= tol, (prec, err)
            assert abs(st["iterations"] - so.iterations) <= 2
