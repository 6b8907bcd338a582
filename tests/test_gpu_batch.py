"""Lock-step batched frame solves (fsim_solve_batch) against solo solves and the oracle.

A batch advances up to max_frames frames of one mesh together through
Algorithm 1 (batched launches, one multi-right-hand-side pass over the
factor, reduced systems side by side); more requests than slots exercise the
continuous admission of pending requests into the slots of finished frames.
Every frame must equal the same request solved alone (mixed precision) within
the mixed-precision bar, 1e-6 of the bounding-box diagonal, with iteration
counts within 4; the face frames are also compared with the stored oracle
frames (tests/golden).
"""
import os

import numpy as np
import pytest

from paper_2312_02999_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                    "face_seq3_f20_f21.npz")


@pytest.fixture(scope="module")
def fsim():
    from paper_2312_02999_gb300 import build
    build.build()
    from paper_2312_02999_gb300 import fsim as f
    return f


@pytest.fixture(scope="module")
def ctx(fsim):
    c = fsim.Context(0)
    yield c
    c.close()


def _diag(mesh):
    return float(np.linalg.norm(mesh.rest.max(0) - mesh.rest.min(0)))


def _pressed(mesh, seed, scale=1e-4, shift=0.0033):
    rng = np.random.default_rng(seed)
    x = mesh.rest.copy()
    free = mesh.pinned == 0
    x[free] += scale * rng.standard_normal((int(free.sum()), 3))
    top = mesh.rest[:, 2] > mesh.rest[:, 2].mean()
    x[top & free, 2] -= shift
    return x


@pytest.mark.parametrize("nx,max_frames,one_cta_max,path", [
    (4, 3, 0, "CLUSTER"), (4, 3, 96, "ONE_CTA"), (6, 4, 0, "CLUSTER"), (8, 2, 0, "COOPERATIVE")])
def test_batch_equals_solo_solves(fsim, ctx, nx, max_frames, one_cta_max, path):
    # two slabs pressed together: n_c ~ 50, ~98 and ~162; five requests with
    # their own actuation and start state, more than the batch's slots.  A
    # batch solves every 0 < n_c <= 128 on the 4-CTA cluster path unless the
    # mesh sets reduced_one_cta_max (then n_c up to it takes the one-CTA
    # path); larger n_c take the cooperative kernel
    mesh = I.two_slabs(nx, nx, 2, gap=0.004)
    m = ctx.upload(mesh)
    m.prefactor(fsim.params_for(mesh, reduced_one_cta_max=one_cta_max))
    reqs, solo = [], []
    for k in range(5):
        act = I.slab_actuation(mesh, seed=20 + k)
        x0 = _pressed(mesh, seed=40 + k)
        reqs.append((m, act.fiber, act.stretch, x0))
        m.set_actuation(act.fiber, act.stretch)
        rc, st = m.solve_frame(x_init=x0, precision=fsim.MIXED)
        assert rc == 0
        solo.append((m.positions(), st))
    rc, xs, sts = fsim.solve_batch(ctx, reqs, max_frames=max_frames)
    assert rc == 0
    diag = _diag(mesh)
    paths = np.zeros(4, dtype=int)
    for (xo, so), x, st in zip(solo, xs, sts):
        assert st["status"] == 0
        assert np.abs(x - xo).max() <= 1e-6 * diag, np.abs(x - xo).max() / diag
        # the two solves round differently (batched vs single-frame reduced
        # paths, and the order of the float64 atomic sums of B-check and g),
        # which can flip a line-search acceptance at the 1e-12 energy margin:
        # iteration counts agree within 4
        assert abs(st["iterations"] - so["iterations"]) <= 4, (st["iterations"], so["iterations"])
        assert st["contacts"] > 0
        paths += np.array(st["reduced_steps"])
    # the batch really took the reduced-system path of this contact size
    assert paths[getattr(fsim, "REDUCED_" + path)] > 0, paths


@pytest.mark.slow
def test_batch_face_frames_match_the_oracle(fsim, ctx):
    gold = dict(np.load(GOLD))
    mesh = I.face_shell()
    field = I.bump_field(mesh, seed=int(gold["field_seed"]))
    coeffs = I.keyframe_coeffs(seed=int(gold["seq_seed"]))
    m = ctx.upload(mesh)
    m.prefactor(fsim.params_for(mesh))
    f20, f21 = gold["frames"].tolist()
    a20 = I.bump_actuation(field, coeffs[f20])
    a21 = I.bump_actuation(field, coeffs[f21])
    # frame 20 from rest and frame 21 from the oracle's frame-20 result, in one batch
    rc, xs, sts = fsim.solve_batch(ctx, [(m, a20.fiber, a20.stretch, None),
                                         (m, a21.fiber, a21.stretch, gold["x0"])], max_frames=2)
    assert rc == 0
    diag = _diag(mesh)
    for k, (x, st) in enumerate(zip(xs, sts)):
        assert st["status"] == 0 and st["n_c_max"] > 0
        err = np.abs(x - gold[f"x{k}"]).max() / diag
        assert err <= 1e-6, (k, err)
        assert abs(st["iterations"] - int(gold[f"iterations{k}"])) <= 2


def test_headline_batch_frames_match_the_oracle(fsim, ctx):
    # the launch configuration of the headline: one 32-frame lock-step batch
    # (96 multi-RHS columns, tensor-core Sigma^-1 product, lane-per-pair
    # barrier) on the full 30k face; two of its frames are the stored oracle
    # frames (frame 20 from rest, frame 21 from the oracle's frame 20), the
    # other 30 are further frames of the sequence from rest, which must
    # converge.  The oracle frames are placed in the middle of the batch.
    gold = dict(np.load(GOLD))
    mesh = I.face_shell()
    field = I.bump_field(mesh, seed=int(gold["field_seed"]))
    coeffs = I.keyframe_coeffs(seed=int(gold["seq_seed"]))
    m = ctx.upload(mesh)
    m.prefactor(fsim.params_for(mesh))
    f20, f21 = gold["frames"].tolist()
    reqs = []
    for k in range(32):
        fr = 22 + k if k not in (13, 14) else (f20 if k == 13 else f21)
        a = I.bump_actuation(field, coeffs[fr])
        reqs.append((m, a.fiber, a.stretch, gold["x0"] if k == 14 else None))
    rc, xs, sts = fsim.solve_batch(ctx, reqs, max_frames=32)
    assert rc == 0
    assert all(st["status"] == 0 for st in sts)
    diag = _diag(mesh)
    for k, slot in ((0, 13), (1, 14)):
        err = np.abs(xs[slot] - gold[f"x{k}"]).max() / diag
        assert err <= 1e-6, (k, err)
        assert abs(sts[slot]["iterations"] - int(gold[f"iterations{k}"])) <= 4


def test_batch_argument_errors(fsim, ctx):
    mesh = I.two_slabs(3, 3, 2)
    m = ctx.upload(mesh)
    m.prefactor(fsim.params_for(mesh))
    act = I.slab_actuation(mesh, seed=1)
    rc, _, _ = fsim.solve_batch(ctx, [(m, act.fiber, act.stretch, None)], max_frames=0)
    assert rc == fsim.FSIM_EINVAL
    bad = act.stretch.copy()
    bad[0] = -1.0
    rc, _, sts = fsim.solve_batch(ctx, [(m, act.fiber, bad, None),
                                        (m, act.fiber, act.stretch, None)], max_frames=2)
    assert rc == fsim.FSIM_ENONFINITE
    assert sts[0]["status"] == fsim.FSIM_ENONFINITE and sts[1]["status"] == 0


def test_batch_stiff_requests_switch_to_float64(fsim, ctx):
    # The 2k-vertex face under requests that press the lips together hard:
    # a frame whose float32 reduced factor loses positive definiteness
    # redoes that step with float64 pair eigen-solves and factors on its own
    # workspace and keeps them for the rest of the frame, inside the batch.
    # Every frame must converge and agree with its float64 solve.  Some of
    # these requests have two equilibria a few 1e-5 of the diagonal apart
    # with energies within 1e-6 (relative; 4e-9 to 4e-7 seen) of each other,
    # and rounding decides which one a solve reaches; at most four frames may
    # end at another one, as stationary points of nearly the same energy.
    mesh = I.face_shell(n_target=2000)
    field = I.bump_field(mesh, n_bumps=64, seed=11)
    coeffs = I.request_coeffs(48 * 8, n_bumps=64, seed=5)
    m = ctx.upload(mesh)
    m.prefactor(fsim.params_for(mesh))
    reqs, ref = [], []
    for ci in (16, 188, 189, 195, 235, 270, 303, 344, 359, 0, 3, 40):
        a = I.bump_actuation(field, coeffs[ci])
        m.set_actuation(a.fiber, a.stretch)
        rc, st64 = m.solve_frame(x_init=mesh.rest, precision=fsim.FP64, check=False)
        assert rc == 0
        ref.append((m.positions(), st64))
        reqs.append((m, a.fiber, a.stretch, None))
    rc, xs, sts = fsim.solve_batch(ctx, reqs, max_frames=8)
    assert rc == 0
    diag = _diag(mesh)
    other = 0
    for x, (xr, s64), st in zip(xs, ref, sts):
        assert st["status"] == 0
        assert st["grad_norm"] <= mesh.tol_rel * st["grad_norm0"] + mesh.tol_abs
        err = np.abs(x - xr).max() / diag
        if err > 1e-6:
            other += 1
            assert err <= 1e-3
            assert abs(st["energy"] - s64["energy"]) <= 1e-6 * abs(s64["energy"])
    assert other <= 4
    assert sum(st["fp64_steps"] for st in sts) > 0
