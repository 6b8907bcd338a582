"""GPU parity at the full 30k-vertex face size (the bench workload).

The oracle cannot afford a whole face frame (~90 sparse LU factorisations of
77k DOFs), so these tests check, at the positions the GPU converges to,
properties that the oracle can evaluate at any size: its own stopping test
of Algorithm 1 (gradient norm), the exact constraint set, the energy, the
per-tet projections, and the global step's backward error at a contact state.
"""
import numpy as np
import pytest

from oracle import contact as OC
from oracle import fem as OF
from oracle import solver as S
from paper_2312_02999_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def face():
    from paper_2312_02999_gb300 import build
    build.build()
    from paper_2312_02999_gb300 import fsim
    mesh = I.face_shell()
    field = I.bump_field(mesh, seed=2)
    coeffs = I.keyframe_coeffs(seed=3)
    act = I.bump_actuation(field, coeffs[30])
    ctx = fsim.Context(0)
    m = ctx.upload(mesh)
    m.prefactor(fsim.params_for(mesh))
    m.set_actuation(act.fiber, act.stretch)
    kappa = m.info()["kappa"]
    pr = S.Problem(mesh.rest, mesh.tets, mesh.pinned, mesh.proxy_tris, mesh.W_rowptr, mesh.W_col,
                   mesh.W_val, S.Params(dhat=mesh.dhat, tol_abs=mesh.tol_abs,
                                        tol_rel=mesh.tol_rel, kappa=kappa))
    pr.set_actuation(act.fiber, act.stretch)
    out = {"mesh": mesh, "m": m, "pr": pr, "fsim": fsim, "ctx": ctx}
    for name, prec in (("fp64", fsim.FP64), ("mixed", fsim.MIXED)):
        rc, st = m.solve_frame(x_init=mesh.rest, precision=prec)
        out[name] = (m.positions(), st)
    yield out
    ctx.close()


def _oracle_grad_norm(pr, x):
    ev = pr.evaluate(x)
    g = pr.gradient(x, ev).ravel()[pr.free_dofs]
    return float(np.linalg.norm(g)), ev


@pytest.mark.parametrize("name", ["fp64", "mixed"])
def test_face_frame_meets_the_oracle_stopping_test(face, name):
    mesh, pr = face["mesh"], face["pr"]
    x, st = face[name]
    assert st["status"] == 0 and st["iterations"] > 10
    assert st["contacts"] > 0 and st["n_c_max"] > 0       # the lips really touch
    gn, ev = _oracle_grad_norm(pr, x)
    g0, _ = _oracle_grad_norm(pr, mesh.rest)
    tol = max(mesh.tol_abs, mesh.tol_rel * g0)
    assert gn <= 1.5 * tol, (gn, tol)
    assert abs(gn - st["grad_norm"]) <= 1e-6 * tol + 1e-9 * gn
    assert abs(ev["E"] + ev["B"] - st["energy"]) <= 1e-10 * abs(st["energy"])
    # proxy never touches
    s = pr.W @ x
    typ, i, j = OC.candidate_pairs(s, pr.tris, pr.edges, 10 * mesh.dhat)
    V = OC.pair_vertices(typ, i, j, pr.tris, pr.edges)
    assert OC.distance(s[V], typ == 1).min() > 0.0


def test_face_mixed_and_fp64_positions_agree(face):
    mesh = face["mesh"]
    xa, _ = face["fp64"]
    xb, _ = face["mixed"]
    diag = float(np.linalg.norm(mesh.rest.max(0) - mesh.rest.min(0)))
    assert np.abs(xa - xb).max() / diag <= 1e-6


def test_face_contact_set_and_local_step(face):
    mesh, m, pr = face["mesh"], face["m"], face["pr"]
    x, _ = face["fp64"]
    keys = m.contacts()
    s = pr.W @ x
    typ, i, j, d = OC.constraint_set(s, pr.tris, pr.edges, mesh.dhat)
    assert set(map(tuple, keys.tolist())) == set(zip(typ.tolist(), i.tolist(), j.tolist()))
    E, g, P = m.eval_elastic(x, precision=0, want_proj=True)
    F = OF.deformation_gradients(x, pr.tets, pr.G)
    _, Po = OF.local_step(F, pr.A)
    assert np.abs(P - Po.reshape(-1, 9)).max() <= 1e-10 * np.abs(Po).max()
    assert abs(E - OF.elastic_energy(F, Po, pr.w)) <= 1e-10 * E


@pytest.mark.parametrize("prec,tol", [(0, 1e-6), (1, 1e-4)])
def test_face_global_step_backward_error(face, prec, tol):
    mesh, m, pr = face["mesh"], face["m"], face["pr"]
    x, _ = face["fp64"]
    # the converged contact state of frame 30 (n_c there exercises the
    # multi-CTA reduced solve of the mixed form)
    dx = m.eval_global_step(x, precision=prec)
    ev = pr.evaluate(x)
    assert ev["C"][0].size > 0
    g = pr.gradient(x, ev).ravel()[pr.free_dofs]
    Hh = pr.H + pr.free_part(pr.barrier_hessian(ev))
    res = np.linalg.norm(Hh @ dx.ravel()[pr.free_dofs] + g) / np.linalg.norm(g)
    # cond(H) of the face is ~1.6e3, but stiff contact pairs make the low-rank
    # correction z2 = u - Sigma^-1 Q^T v a difference of two large terms, so
    # the backward error of this (not backward-stable) route is well above
    # eps; measured 1.9e-7 in float64.  The mixed form's float32 solves of
    # K11 and Sigma bound it near 1e-5 (same bound as the slab test).  The
    # outer loop's float64 gradient absorbs either.
    assert res <= tol, res
