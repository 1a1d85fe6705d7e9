"""Bounded waits of the split-precision kernel report DSRG_ERR_TIMEOUT.

The tensor-core kernel waits on shared-memory barriers for its own bulk
copies and tensor-core products.  Each wait has a budget in SM clock cycles
(dsrg_options.wait_limit).  With a budget of one cycle the first wait of
every tile runs out while its copies are still in flight: the kernel then
waits (with the fixed default budget) for what it has in flight, frees its
tensor memory and sets the error flag, and the call returns
DSRG_ERR_TIMEOUT.  The context stays usable: the same energy with the
default budget afterwards matches the FP64 path.
"""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_02011_gb300 import build
    build.build()
    import paper_1701_02011_gb300 as g
    g.load_library()
    return g


def test_wait_budget_runs_out_then_context_is_usable(lib):
    # large enough that the DF ladder build (M = N = 34^2, K = 120) runs as a split product
    inst = synth.make_instance(2, 4, 4, 30, 120, 0.5, seed=5)
    h = lib.Dsrg(inst, precision=lib.DSRG_PREC_SPLIT, slices=6, wait_limit=1)
    try:
        with pytest.raises(lib.DsrgError) as ex:
            h.pt3()
        assert ex.value.code == lib.DSRG_ERR_TIMEOUT
        assert "bounded wait" in str(ex.value)
    finally:
        h.close()
    ref = lib.Dsrg(inst)
    try:
        e64 = ref.pt3()
    finally:
        ref.close()
    h = lib.Dsrg(inst, precision=lib.DSRG_PREC_SPLIT, slices=6)
    try:
        e = h.pt3()
    finally:
        h.close()
    for k in ("e2", "e3a", "e3b", "e3"):
        assert abs(e[k] - e64[k]) < 1e-6, (k, e[k], e64[k])


def test_negative_wait_limit_is_an_argument_error(lib):
    inst = synth.make_instance(1, 2, 2, 2, 4, 0.5, seed=1)
    with pytest.raises(lib.DsrgError) as ex:
        lib.Dsrg(inst, precision=lib.DSRG_PREC_SPLIT, slices=6, wait_limit=-5)
    assert ex.value.code == lib.DSRG_ERR_ARG
