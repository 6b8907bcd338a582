"""The tensor-core product u = Sigma^-1 y2 of the lock-step batches against the oracle.

Sigma is the Schur complement of Eq. 8 (Sec. 3.2): the oracle forms it
densely from its own PD matrix (K (x) I_3 over the free vertices) and inverts
it in float64.  The kernel (tcgen05, kind::tf32) multiplies TF32 head/tail
splits of float32 Sigma^-1 and float32 y.  Its error per product term, in
units of |Sigma^-1_ik| |y_kc|, is:

* 2^-24 from rounding Sigma^-1 to float32;
* 2 x 2^-20 from the head/tail truncation of the two operands;
* 2^-20 from the dropped tail x tail term.

A float32 accumulation over n2 terms adds at most n2 2^-23.  The test bound
is the sum of these, applied to |Sigma^-1| |y|.  A TF32-only product, which
has errors near 2^-11, fails this bound.

The mesh is two slabs with n2 = 162 x2 vertices: two 128-row tiles, the
second one ragged, and six k stages, the last one ragged.
"""
import numpy as np
import pytest

from oracle import solver as S
from paper_2312_02999_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def slabs(fsim, ctx):
    mesh = I.two_slabs(8, 8, 2, gap=0.004)
    m = ctx.upload(mesh)
    p = fsim.params_for(mesh)
    m.prefactor(p)
    op = S.Params(dhat=mesh.dhat, tol_abs=p.tol_abs, tol_rel=p.tol_rel,
                  weight_scale=mesh.weight_scale)
    pr = S.Problem(mesh.rest, mesh.tets, mesh.pinned, mesh.proxy_tris, mesh.W_rowptr,
                   mesh.W_col, mesh.W_val, op, region=mesh.region)
    i1, i2 = pr.split_dofs()
    sig = S.schur_complement(pr.H.toarray(), i1, i2)
    # Sigma = Sigma_v (x) I_3: the x, y, z blocks are equal and uncoupled
    assert np.abs(sig[0::3, 1::3]).max() <= 1e-12 * np.abs(sig).max()
    assert np.allclose(sig[0::3, 0::3], sig[2::3, 2::3], rtol=0, atol=1e-12 * np.abs(sig).max())
    sinv = np.linalg.inv(sig[0::3, 0::3])
    return m, sinv


def _bound(sinv, y32):
    n2 = sinv.shape[0]
    unit = 2.0 ** -24 + 3 * 2.0 ** -20 + n2 * 2.0 ** -23
    return unit * (np.abs(sinv) @ np.abs(y32))


@pytest.mark.parametrize("ncols", [96, 32, 7, 192])
def test_sigma_inv_product_tensor_cores(slabs, ncols):
    m, sinv = slabs
    n2 = sinv.shape[0]
    assert n2 > 128 and n2 % 128 != 0 and n2 % 32 != 0
    y = np.random.default_rng(ncols).standard_normal((n2, ncols))
    y32 = y.astype(np.float32).astype(np.float64)
    ref = sinv @ y32
    u = m.eval_sigma_inv_mr(y, tensor_cores=True)
    assert np.all(np.abs(u - ref) <= _bound(sinv, y32))


def test_sigma_inv_product_simt_matches(slabs):
    m, sinv = slabs
    n2 = sinv.shape[0]
    y = np.random.default_rng(5).standard_normal((n2, 64))
    y32 = y.astype(np.float32).astype(np.float64)
    ref = sinv @ y32
    u = m.eval_sigma_inv_mr(y, tensor_cores=False)
    bound = (2.0 ** -24 + n2 * 2.0 ** -24) * (np.abs(sinv) @ np.abs(y32))
    assert np.all(np.abs(u - ref) <= bound)


def test_sigma_inv_product_structure(slabs):
    # linear in y, and zero columns stay zero (no cross-talk between frames'
    # columns or from stale shared-memory tiles)
    m, sinv = slabs
    n2 = sinv.shape[0]
    rng = np.random.default_rng(9)
    y = np.zeros((n2, 96))
    y[:, 3:6] = rng.standard_normal((n2, 3))
    u = m.eval_sigma_inv_mr(y, tensor_cores=True)
    assert np.all(u[:, :3] == 0.0) and np.all(u[:, 6:] == 0.0)
    e = np.zeros((n2, 32))
    e[np.arange(32) * 5, np.arange(32)] = 1.0        # unit vectors: columns of Sigma^-1
    u = m.eval_sigma_inv_mr(e, tensor_cores=True)
    col = sinv[:, np.arange(32) * 5]
    assert np.all(np.abs(u - col) <= (2.0 ** -24 + 3 * 2.0 ** -20 + 2.0 ** -23) * np.abs(col)
                  + 1e-30)
