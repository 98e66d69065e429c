"""GPU set-up (S0) vs the oracle: tet classification, linear IFE local data,
cut cells and the surface-charge target table."""
import numpy as np
import pytest

from tests.pairs import CASES, make_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", list(CASES))
def test_interface_tets_match_oracle(case):
    gpu, orc = make_pair(case)
    fs = orc.fs
    g = gpu.interface()
    # bit-exact: which tets are interface tets, in (cell, local tet) order
    assert np.array_equal(g["cell"], fs.it_cell) and np.array_equal(g["tet"], fs.it_t)
    h = fs.mesh.h
    V = h ** 3
    assert np.allclose(g["vol_plus"], fs.it_volp, rtol=0, atol=1e-13 * V)
    assert np.allclose(g["vol_minus"], fs.it_volm, rtol=0, atol=1e-13 * V)
    assert np.allclose(g["area"], fs.it_area, rtol=0, atol=1e-12 * h * h)
    kscale = np.abs(fs.it_K).max()
    assert np.abs(g["K"] - fs.it_K).max() <= 1e-10 * kscale
    cscale = np.abs(fs.it_c).max()
    assert np.abs(g["c"] - fs.it_c).max() <= 1e-10 * cscale
    cells, area = gpu.cut_cells()
    assert np.array_equal(cells, fs.cut_cells)
    assert np.allclose(area, fs.cut_area, rtol=1e-12, atol=0)
    assert np.array_equal(gpu.cell_target(), fs.cell_to_acc)
    gpu.close()
