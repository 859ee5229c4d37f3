"""Host-side argument checks of the binding (no GPU needed): a state solve with a
wrongly shaped output or slowness is refused with ValueError before any pointer reaches
the library, so the library never writes past a caller's buffer."""
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W


def test_state_solve_refuses_wrong_shapes_before_the_library():
    g = W.config1().grid
    dg = eik.DeviceGrid(g, device="cpu")
    s = torch.ones(g.N, dtype=torch.float64)
    with pytest.raises(ValueError):
        eik.eik_forward_noalloc(dg, s, [0, 1], torch.empty((2, g.N - 1), dtype=torch.float64))
    with pytest.raises(ValueError):
        eik.eik_forward_noalloc(dg, s, [0, 1], torch.empty((1, g.N), dtype=torch.float64))
    with pytest.raises(ValueError):
        eik.eik_forward_noalloc(dg, torch.ones(g.N + 1, dtype=torch.float64), [0], torch.empty((1, g.N), dtype=torch.float64))
    with pytest.raises(ValueError):
        eik.eik_forward(dg, s, [0], out=torch.empty((2, g.N), dtype=torch.float64))
