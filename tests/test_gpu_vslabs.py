"""Two-body classes built on demand: with a tiny memory budget no class of V
is stored, and every term that reads V builds it from B on the term's own
intervals, a slab of the first slot at a time.  Energies and intermediates
must not change beyond summation order."""
import os

import numpy as np
import pytest

import synth
from oracle import dsrg

pytestmark = pytest.mark.gpu

KEYS = ("e2", "e3a", "e3b", "e3")


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


def _run(lib, inst, budget_mb, **kw):
    old = os.environ.get("DSRG_V_CLASS_BUDGET_MB")
    if budget_mb is None:
        os.environ.pop("DSRG_V_CLASS_BUDGET_MB", None)
    else:
        os.environ["DSRG_V_CLASS_BUDGET_MB"] = str(budget_mb)
    try:
        h = lib.Dsrg(inst, **kw)
        try:
            e = h.pt3()
            inter = {k: h.fetch(k) for k in ("T2b", "O2")}
        finally:
            h.close()
    finally:
        if old is None:
            os.environ.pop("DSRG_V_CLASS_BUDGET_MB", None)
        else:
            os.environ["DSRG_V_CLASS_BUDGET_MB"] = old
    return e, inter


@pytest.mark.parametrize("shape", [(3, 4, 4, 21, 50), (2, 4, 4, 12, 60), (1, 3, 2, 2, 5)])
def test_on_demand_classes_match_stored_and_oracle(lib, shape):
    nc, na, nel, nv, naux = shape
    inst = synth.make_instance(nc, na, nel, nv, naux, 0.5, seed=sum(shape) + 31)
    e_lazy, i_lazy = _run(lib, inst, 0.05)     # every class over budget: slabs
    e_full, i_full = _run(lib, inst, None)     # every class stored
    ref = dsrg.dsrg_pt3(inst)
    for k in KEYS:
        assert abs(e_lazy[k] - ref[k]) < 1e-9, (k, e_lazy[k], ref[k])
        assert abs(e_lazy[k] - e_full[k]) < 1e-11 * max(1.0, abs(e_full[k])), k
    for k in i_full:
        scale = max(1.0, float(np.abs(i_full[k]).max()))
        assert np.abs(i_lazy[k] - i_full[k]).max() < 1e-11 * scale, k


def test_on_demand_classes_split_precision(lib):
    inst = synth.make_instance(3, 4, 4, 21, 50, 0.5, seed=77)
    e_lazy, _ = _run(lib, inst, 0.05, precision=lib.DSRG_PREC_SPLIT, slices=6)
    ref = dsrg.dsrg_pt3(inst)
    for k in KEYS:
        assert abs(e_lazy[k] - ref[k]) < 1e-9, (k, e_lazy[k], ref[k])
