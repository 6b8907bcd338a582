#!/usr/bin/env python3
"""Write the face-frame expected values (tests/golden/face_seq3_f20_f21.npz).

Only the float64 CPU oracle (``oracle/``) and the seeded input generator
(``paper_2312_02999_gb300.inputs``, which holds none of the method's
arithmetic) are used: no value here comes from the CUDA path.

Workload: the synthetic 30k-vertex face shell, actuation field seed 2,
keyframe sequence seed 3 (the first of the benchmark's request streams).
Frame 20 is solved by Algorithm 1 from the rest pose; frame 21 is solved
from frame 20's result (the warm start a served sequence uses).  Stored per
frame: converged positions, the constraint set at them (sorted keys
type, i, j), accepted iterations, the gradient norm at the start and at the
end, the energy, and the per-iteration n_c.  The barrier stiffness is the
oracle's automatic one (mean diagonal entry of H over the free DOFs).

Usage:  python tests/golden/make_face_golden.py   (about 15 min on one core)
"""
from __future__ import annotations

import os
import sys
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import contact as OC  # noqa: E402
from oracle import solver as S  # noqa: E402
from paper_2312_02999_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "face_seq3_f20_f21.npz")
SEQ_SEED, FIELD_SEED, FIRST = 3, 2, 20


def main():
    mesh = I.face_shell()
    field = I.bump_field(mesh, seed=FIELD_SEED)
    coeffs = I.keyframe_coeffs(seed=SEQ_SEED)
    pr = S.Problem(mesh.rest, mesh.tets, mesh.pinned, mesh.proxy_tris, mesh.W_rowptr,
                   mesh.W_col, mesh.W_val,
                   S.Params(dhat=mesh.dhat, tol_abs=mesh.tol_abs, tol_rel=mesh.tol_rel))
    out = {"n": mesh.n, "T": mesh.T, "kappa": pr.kappa, "dhat": mesh.dhat,
           "tol_abs": mesh.tol_abs, "tol_rel": mesh.tol_rel,
           "frames": np.array([FIRST, FIRST + 1]), "seq_seed": SEQ_SEED,
           "field_seed": FIELD_SEED}
    x = mesh.rest
    for k, f in enumerate((FIRST, FIRST + 1)):
        act = I.bump_actuation(field, coeffs[f])
        pr.set_actuation(act.fiber, act.stretch)
        t0 = time.perf_counter()
        x, st = pr.solve_frame(x)
        dt = time.perf_counter() - t0
        if st.status != S.STATUS_OK:
            raise SystemExit(f"frame {f}: oracle status {st.status}")
        typ, i, j, _ = OC.constraint_set(pr.W @ x, pr.tris, pr.edges, mesh.dhat)
        keys = np.stack([typ, i, j], axis=1).astype(np.int64)
        keys = keys[np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))]
        out[f"x{k}"] = x
        out[f"keys{k}"] = keys
        out[f"iterations{k}"] = st.iterations
        out[f"grad_norm0_{k}"] = st.grad_norms[0]
        out[f"grad_norm{k}"] = st.grad_norms[-1]
        out[f"energy{k}"] = st.energies[-1]
        out[f"n_c{k}"] = np.array(st.n_c, dtype=np.int32)
        out[f"seconds{k}"] = dt
        print(f"frame {f}: {st.iterations} iterations, |C| {len(keys)}, "
              f"max n_c {max(st.n_c) if st.n_c else 0}, {dt:.0f} s", flush=True)
    np.savez_compressed(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
