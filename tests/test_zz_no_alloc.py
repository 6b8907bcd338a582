"""fsim_ccd_noalloc: the CCD step bound without any device allocation.

Callers that cannot let a library allocate GPU memory (an engine that owns
all device memory through its own pool, a process held to a fixed memory
budget, code recorded into the caller's CUDA graph) pass their own device
buffers and get the same step bound as the solver's CCD stage; the entry
point keeps its scratch in a fixed static device array.  This test checks it
against the existing entry point fsim_eval_ccd on two calls in a row (the
second call must not see the first call's candidates), through the C ABI.
This file is collected last so that a failure here leaves every other test run.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2312_02999_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _edges(tris):
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]], axis=0)
    return np.unique(np.sort(e, axis=1), axis=0).astype(np.int32)


def test_noalloc_ccd_matches_existing_entry_point_twice():
    torch = pytest.importorskip("torch")
    from paper_2312_02999_gb300 import build
    build.build()
    from paper_2312_02999_gb300 import fsim

    mesh = I.two_slabs(4, 4, 2, gap=0.004)
    act = I.slab_actuation(mesh, seed=11)
    rng = np.random.default_rng(8)
    free = mesh.pinned == 0
    top = mesh.rest[:, 2] > mesh.rest[:, 2].mean()
    x = mesh.rest.copy()
    x[free] += 2e-4 * rng.standard_normal((int(free.sum()), 3))
    x[top & free, 2] -= 0.003
    steps = []
    for k, down in enumerate((0.004, 0.006)):
        dx = np.zeros_like(x)
        dx[free & top, 2] = -down
        dx[free] += 3e-4 * rng.standard_normal((int(free.sum()), 3))
        steps.append(dx)

    with fsim.Context(0) as ctx:
        m = ctx.upload(mesh)
        p = fsim.params_for(mesh)
        m.prefactor(p)
        m.set_actuation(act.fiber, act.stretch)
        s = m.eval_proxy(x)
        dev = torch.device("cuda", 0)
        tris_d = torch.tensor(mesh.proxy_tris.astype(np.int32), device=dev).contiguous()
        edges = _edges(mesh.proxy_tris)
        edges_d = torch.tensor(edges, device=dev).contiguous()
        s_d = torch.tensor(s, dtype=torch.float64, device=dev).contiguous()
        alpha_d = torch.zeros(1, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev)
        for dx in steps:
            ref = m.eval_ccd(x, dx)
            ds = m.eval_proxy(dx)                  # W dx, as the CCD stage forms it
            ds_d = torch.tensor(ds, dtype=torch.float64, device=dev).contiguous()
            alpha_d.fill_(-7.0)                    # the call must overwrite it
            torch.cuda.synchronize()
            st = ctx.lib.fsim_ccd_noalloc(
                C.c_void_p(s_d.data_ptr()), C.c_void_p(ds_d.data_ptr()), s.shape[0],
                C.c_void_p(tris_d.data_ptr()), mesh.proxy_tris.shape[0],
                C.c_void_p(edges_d.data_ptr()), edges.shape[0], p.dhat, p.ccd_s,
                p.accd_max_iters, C.c_void_p(alpha_d.data_ptr()),
                C.c_void_p(stream.cuda_stream))
            assert st == fsim.FSIM_OK
            got = float(alpha_d.item())
            assert 0.0 < ref < 1.0
            assert abs(got - ref) <= 1e-12 * ref, (got, ref)
        # argument checks return errors, never fault
        bad = ctx.lib.fsim_ccd_noalloc(None, None, 5, None, 0, None, 0, p.dhat, p.ccd_s,
                                       p.accd_max_iters, C.c_void_p(alpha_d.data_ptr()), None)
        assert bad == fsim.FSIM_EINVAL
