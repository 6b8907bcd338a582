"""fsim_ccd_noalloc: the CCD step bound without any device allocation.

Callers that cannot let a library allocate GPU memory (an engine that owns
all device memory through its own pool, a process held to a fixed memory
budget) pass their own device buffers and get the same step bound as the
solver's CCD stage; the entry point keeps its scratch in a fixed static
device array.  This test checks it against the existing entry point
fsim_eval_ccd on two calls in a row (the second call must not see the first
call's candidates), through the C ABI; then a call with more candidates than
the static array holds (FSIM_ECONTACT_OVERFLOW) and a call with a triangle
index out of range (FSIM_EINVAL), each followed by a normal call that must
again match the existing entry point.
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

        def call(s_t, ds_t, tris_t, edges_t, dhat):
            alpha_d.fill_(-7.0)
            torch.cuda.synchronize()
            return ctx.lib.fsim_ccd_noalloc(
                C.c_void_p(s_t.data_ptr()), C.c_void_p(ds_t.data_ptr()), s_t.shape[0],
                C.c_void_p(tris_t.data_ptr()), tris_t.shape[0],
                C.c_void_p(edges_t.data_ptr()), edges_t.shape[0], dhat, p.ccd_s,
                p.accd_max_iters, C.c_void_p(alpha_d.data_ptr()),
                C.c_void_p(stream.cuda_stream))

        ds_last = torch.tensor(m.eval_proxy(steps[-1]), dtype=torch.float64, device=dev)
        ref_last = m.eval_ccd(x, steps[-1])
        # more candidates than the static array holds: with dhat far larger than
        # the mesh every non-adjacent pair is a candidate (16x16 faces: about
        # 0.6M point-triangle and 1.3M edge-edge pairs > 2^20)
        big = I.two_slabs(16, 16, 2, gap=0.004)
        sb = big.rest[big.W_col]                      # selection proxy: s = W x
        assert np.array_equal(np.diff(big.W_rowptr), np.ones(sb.shape[0], dtype=np.int64))
        sb_d = torch.tensor(sb, dtype=torch.float64, device=dev).contiguous()
        dsb_d = torch.full_like(sb_d, 1e-4)
        trb_d = torch.tensor(big.proxy_tris.astype(np.int32), device=dev).contiguous()
        edb_d = torch.tensor(_edges(big.proxy_tris), device=dev).contiguous()
        assert call(sb_d, dsb_d, trb_d, edb_d, 100.0) == fsim.FSIM_ECONTACT_OVERFLOW
        assert call(s_d, ds_last, tris_d, edges_d, p.dhat) == fsim.FSIM_OK
        assert abs(float(alpha_d.item()) - ref_last) <= 1e-12 * ref_last
        # a triangle naming a vertex outside [0, Ns) is reported, not read
        tris_bad = tris_d.clone()
        tris_bad[3, 1] = s.shape[0]
        assert call(s_d, ds_last, tris_bad, edges_d, p.dhat) == fsim.FSIM_EINVAL
        assert call(s_d, ds_last, tris_d, edges_d, p.dhat) == fsim.FSIM_OK
        assert abs(float(alpha_d.item()) - ref_last) <= 1e-12 * ref_last
