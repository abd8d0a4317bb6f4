"""The allocation-free brute-force entry point (irs_make_map_brute_noalloc).

It exists for callers that cannot allocate device memory -- code running
while another memory manager owns the device, plug-ins that must not trigger
cudaMalloc's device-wide synchronisation, latency-critical loops.  This file
checks, through the C ABI, that two calls in a row give the map of the
ordinary entry point (irs_make_map with a brute-force plan) within the tests'
misbinning bar, that the second call leaves the device's free memory
unchanged, and that lattices beyond its static scratch are refused before any
work is enqueued.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import oracle
from paper_2204_10871_gb300 import irs
from gpu_common import MISBIN_TOL, lenses_for, misbinned, params_pair, require_gpu, to_dev

pytestmark = pytest.mark.gpu

C1 = (0.3, 0.0, 0.3, (-2.5, 2.5, -2.5, 2.5), 128, 25.0)


def test_noalloc_matches_plan_entry_point_twice():
    torch = require_gpu()
    po, pl = params_pair(*C1, method=irs.IRS_BRUTE)
    qo = oracle.size(po)
    xy, m = lenses_for(qo, 150, seed=1, kappa_star=0.3)
    dxy, dm = to_dev(torch, xy, m)
    with irs.Plan(pl) as plan:
        ref, ref_mag = plan.make_map(dxy, dm)
        plan.sync()
    ref = ref.cpu().numpy()
    landed = int(ref.sum())
    counts = torch.full((128, 128), 7, dtype=torch.uint32, device="cuda")  # stale contents
    mag = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    free_after_first = None
    for call in range(2):
        if call == 1:
            torch.cuda.synchronize()
            free_after_first = torch.cuda.mem_get_info()[0]
        irs.irs_make_map_brute_noalloc(pl, dxy, dm, counts, mag)
        torch.cuda.synchronize()
        got = counts.cpu().numpy()
        assert misbinned(ref, got) <= MISBIN_TOL * landed, f"call {call}"
        assert np.allclose(mag.cpu().numpy(), ref_mag.cpu().numpy(), rtol=1e-6, atol=0)
    assert torch.cuda.mem_get_info()[0] == free_after_first


def test_noalloc_rejects_lattice_beyond_scratch():
    torch = require_gpu()
    _, pl = params_pair(0.45, 0.0, 0.45, (-10.0, 10.0, -10.0, 10.0), 2000, 100.0,
                        method=irs.IRS_BRUTE)
    xy = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    m = torch.ones(4, dtype=torch.float64, device="cuda")
    counts = torch.zeros((2000, 2000), dtype=torch.uint32, device="cuda")
    with pytest.raises(irs.IrsError) as err:
        irs.irs_make_map_brute_noalloc(pl, xy, m, counts)
    assert err.value.status == 6  # IRS_ERR_OVERFLOW
    _, pi = params_pair(*C1, method=irs.IRS_INTERP)
    small = torch.zeros((128, 128), dtype=torch.uint32, device="cuda")
    with pytest.raises(irs.IrsError) as err:
        irs.irs_make_map_brute_noalloc(pi, xy, m, small)
    assert err.value.status == 8  # IRS_ERR_UNSUPPORTED
