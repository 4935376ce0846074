"""The randomized SVD's products on the dense count table (LNE_OPT_DENSE_PRODUCT:
the tcgen05 tensor-core product with TF32 hi / lo splitting) against the same
products on the CSR: the same values and FP32-accurate sums in another order,
so embeddings agree to FP32 rounding (1e-5 on the leading subspace), and both
stay within the oracle's 1e-3 subspace bound; c from 40 (padded to the MMA's
48 columns) to 144 (the benchmark's width)."""
import numpy as np
import pytest

import oracle
from paper_2302_07084_gb300 import lne, synth
from gpu_common import assert_subspace, make_params, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("d,q", [(32, 1), (24, 2), (128, 1)])
def test_dense_table_products_match_csr_products(ctx, d, q):
    g = synth.sbm_small()
    s = np.full(10, 0.1)
    p = make_params(10, s, 10.0 * g.n_arcs, d=d, q=q, k=10, seed=1)
    dg = lne.DeviceGraph.from_graph(g)
    ctx.set_option(lne.OPT_AGGREGATION, lne.AGG_TABLE)
    out = {}
    for mode in (1, 2):
        ctx.set_option(lne.OPT_DENSE_PRODUCT, mode)
        out[mode] = to_np(ctx.embed(dg, p)).astype(np.float64)
    ctx.set_option(lne.OPT_DENSE_PRODUCT, 0)
    ctx.set_option(lne.OPT_AGGREGATION, lne.AGG_AUTO)
    lead = 4
    # two FP32 paths summing in different orders: the leading directions agree
    # to 1e-5, the whole d-column span (small gap at d) to 1e-4
    assert_subspace(out[1], out[2], lead, 1e-5, 1e-4, tag=f"table vs csr d={d} q={q}")
    ref = oracle.embed(g.indptr, g.indices, 10, s, p.samples, d, q, 10, 0.5, 0.2, 1)
    for mode in (1, 2):
        assert_subspace(out[mode], ref["X"], lead, tag=f"mode {mode} vs oracle d={d} q={q}")


def test_dense_product_mode_is_validated(ctx):
    with pytest.raises(lne.LneError):
        ctx.set_option(lne.OPT_DENSE_PRODUCT, 3)
