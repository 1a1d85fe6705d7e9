"""The large-active regime (the lambda3 terms of order N_A^6 N_V that the
paper names as the cost of large active spaces, Eq. E_cumulant): synthetic
symmetry-respecting references (synth.synthetic_reference) for active spaces
whose exact CI is out of reach.  CAS(12,12)-sized: the GPU FP64 path against
the block oracle within 1e-9 Eh per component.  16 active orbitals (the
library's limit): the split path against the FP64 path within 1e-6 Eh."""
import pytest

import synth
from oracle import dsrg_df

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


def test_twelve_active_orbitals_against_oracle(lib):
    inst = synth.make_synthetic_instance(1, 12, 3, 12, seed=12)
    ref = dsrg_df.dsrg_pt3(inst)
    h = lib.Dsrg(inst)
    try:
        e = h.pt3()
    finally:
        h.close()
    for k in ("e2", "e3a", "e3b", "e3"):
        assert abs(e[k] - ref[k]) < 1e-9, (k, e[k], ref[k])


def test_sixteen_active_orbitals_split_against_fp64(lib):
    inst = synth.make_synthetic_instance(2, 16, 24, 60, seed=16)
    out = {}
    for prec, sl in ((lib.DSRG_PREC_FP64, 0), (lib.DSRG_PREC_SPLIT, 6)):
        h = lib.Dsrg(inst, precision=prec, slices=sl)
        try:
            out[prec] = h.pt3()
        finally:
            h.close()
    for k in ("e2", "e3a", "e3b", "e3"):
        assert abs(out[lib.DSRG_PREC_SPLIT][k] - out[lib.DSRG_PREC_FP64][k]) < 1e-6, k
