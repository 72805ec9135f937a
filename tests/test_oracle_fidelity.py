"""The fidelity study composes the oracle's runs: on a coarse copy of the
paper layout its ROM approaches the slit fine grid as the ROM deepens, from
a point source and from an initial pulse."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import fidelity


@pytest.mark.slow
@pytest.mark.parametrize("start", ["source", "pulse"])
def test_rom_approaches_the_slit_grid_on_a_coarse_paper_layout(start):
    errs = []
    for k in (1, 2, 3):
        p = inputs.paper_layout(cells_per_unit=6, m=4, k=k)
        u0 = None if start == "source" else inputs.gaussian_pulse(p, p.src_xyz[0], 0.6)
        r = fidelity.trace_errors(p, 6.0, u0)
        assert all(np.isfinite(v) for v in r.values())
        errs.append(r["rom_vs_slit"])
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.2, errs
