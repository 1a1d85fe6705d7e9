"""The density-fitted particle-particle ladder through its C entry point,
against the oracle's definition (Eq. scaling_problem with Eq. int_fact)."""
import numpy as np
import pytest

from oracle import dsrg

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


@pytest.mark.parametrize("n,naux,p0,npart,nh", [(7, 5, 2, 5, 3), (40, 33, 5, 35, 9), (70, 20, 3, 67, 2)])
def test_df_ladder_matches_definition(lib, n, naux, p0, npart, nh):
    import torch
    rng = np.random.default_rng(n + naux)
    B = rng.standard_normal((naux, n, n))
    B = 0.5 * (B + np.transpose(B, (0, 2, 1)))
    t = rng.standard_normal((npart, npart, nh, nh))
    ref = dsrg.df_ladder(B, t, p0)
    Bd = torch.from_numpy(B).cuda()
    td = torch.from_numpy(t).cuda()
    L = torch.full((npart, npart, nh, nh), 7.0, dtype=torch.float64, device="cuda")
    lib.dsrg_df_ladder(Bd, td, L, p0)
    got = L.cpu().numpy()
    assert np.abs(got - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())


def test_df_ladder_argument_errors(lib):
    import torch
    B = torch.zeros((2, 4, 4), dtype=torch.float64, device="cuda")
    t = torch.zeros((3, 3, 2, 2), dtype=torch.float64, device="cuda")
    L = torch.zeros((3, 3, 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.DsrgError) as ex:
        lib.dsrg_df_ladder(B, t, L, p0=2)  # p0 + np > n
    assert ex.value.code == -1
