"""The state solve without device allocation (eik_forward_noalloc).

Some callers cannot call cudaMalloc: code running inside a framework whose caching
allocator owns all device memory, or inside a region where cudaMalloc/cudaFree are not
allowed because they synchronize the device.  eik_forward_noalloc gives them the state
solve with its scratch in one fixed device array inside the library.  These tests call
it through the C-ABI several times in a row on problems of different sizes (a smaller
one after a larger one, so a call runs over scratch an earlier call left behind), check
each result bit for bit against the allocating eik_forward (same kernels, same order),
check that a repeated call changes neither the device's free memory nor torch's
allocations, and check that an oversize request is refused."""
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _cases():
    wl = W.config1()
    g1 = wl.grid
    small = (g1, wl.s, [int(wl.src[0]), g1.index(40, 0)])
    g2 = W.graph_grid((21, 19, 11), 300.0)
    s2 = 1.0 / (2000.0 + 0.5 * g2.xyz[:, 2])
    large = (g2, s2, [g2.index(4, 4, 0), g2.index(15, 9, 0), g2.index(10, 14, 0)])
    return [large, small, large]


def test_noalloc_matches_allocating_state_solve_bitwise():
    assert eik.lib().eik_forward_noalloc_capacity() == 64 << 20
    for g, s, src in _cases():
        dg = eik.DeviceGrid(g)
        sd = torch.tensor(s, device=DEV)
        ref, cyc_ref = eik.eik_forward(dg, sd, src)
        out = torch.full_like(ref, float("nan"))
        got, cyc = eik.eik_forward_noalloc(dg, sd, src, out)
        torch.cuda.synchronize()
        assert cyc == cyc_ref
        assert torch.equal(got, ref)


def test_noalloc_allocates_nothing_on_repeated_calls():
    g, s, src = _cases()[0]
    dg = eik.DeviceGrid(g)
    sd = torch.tensor(s, device=DEV)
    out = torch.empty((len(src), g.N), dtype=torch.float64, device=DEV)
    eik.eik_forward_noalloc(dg, sd, src, out)       # loads the module and looks up the array
    first = out.clone()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):
        eik.eik_forward_noalloc(dg, sd, src, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.equal(out, first)


def test_noalloc_refuses_requests_beyond_its_scratch():
    wl = W.config3()
    dg = eik.DeviceGrid(wl.grid)
    sd = torch.tensor(wl.s, device=DEV)
    out = torch.empty((len(wl.src), wl.grid.N), dtype=torch.float64, device=DEV)
    with pytest.raises(eik.EikError) as e:
        eik.eik_forward_noalloc(dg, sd, wl.src, out)
    assert e.value.code == -1 and "scratch" in str(e.value)
