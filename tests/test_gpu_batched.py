"""irs_make_maps_batched: many uneven maps in one captured CUDA graph give the
same count maps as one irs_make_map per map, on the first call (capture) and
on replays, including replays after the lens values changed in place."""
import numpy as np
import pytest

import oracle
from paper_2204_10871_gb300 import irs
from gpu_common import lenses_for, params_pair, require_gpu, to_dev

pytestmark = pytest.mark.gpu

# (kappa_*, kappa_s, gamma, source side, npix, rays/px, N_*, method, variant)
MAPS = [
    (0.30, 0.00, 0.30, 4.0, 96, 16.0, 400, irs.IRS_INTERP, 0),
    (0.55, 0.25, 0.15, 3.0, 64, 25.0, 900, irs.IRS_INTERP, 1),
    (0.12, 0.08, 0.55, 5.0, 120, 9.0, 150, irs.IRS_INTERP, 2),
    (0.40, 0.10, 0.35, 2.5, 50, 36.0, 1500, irs.IRS_INTERP, 3),
    (0.20, 0.00, 0.10, 2.0, 40, 16.0, 60, irs.IRS_BRUTE, 0),
    (0.45, 0.05, 0.45, 3.0, 80, 20.0, 2000, irs.IRS_INTERP, 0),
]


def _setup(torch):
    plans, lens, counts = [], [], []
    for k, (ks, kss, g, S, npix, nav, nst, meth, var) in enumerate(MAPS):
        po, pl = params_pair(ks, kss, g, (-S / 2, S / 2, -S / 2, S / 2), npix, nav, method=meth,
                             n_star=nst, kernel_variant=var)
        qo = oracle.size(po)
        xy, m = lenses_for(qo, nst, shape="uniform", seed=40 + k, kappa_star=ks)
        plans.append(irs.Plan(pl))
        lens.append(to_dev(torch, xy, m))
        counts.append(torch.zeros((npix, npix), dtype=torch.uint32, device="cuda"))
    return plans, lens, counts


def _singles(torch, plans, lens):
    out = []
    for p, (xy, m) in zip(plans, lens):
        c, _ = p.make_map(xy, m, with_mag=False)
        out.append(c)
    torch.cuda.synchronize()
    return [c.cpu().numpy() for c in out]


def test_batched_graph_matches_single_maps():
    torch = require_gpu()
    plans, lens, counts = _setup(torch)
    try:
        handles = [p.handle for p in plans]
        xs = [l[0] for l in lens]
        ms = [l[1] for l in lens]
        for call in range(3):  # capture, then two replays
            for c in counts:
                c.fill_(123)
            irs.irs_make_maps_batched(handles, xs, ms, counts)
            torch.cuda.synchronize()
            ref = _singles(torch, plans, lens)
            for k, (c, r) in enumerate(zip(counts, ref)):
                assert np.array_equal(c.cpu().numpy(), r), f"map {k}, call {call}"
            if call == 1:  # new lens values behind the same pointers
                for xy, m in lens:
                    m.mul_(0.9)
                    xy.add_(0.01)
        for p in plans:
            p.sync()
    finally:
        for p in plans:
            p.close()


def test_batched_rejects_repeated_plan_and_mlp():
    torch = require_gpu()
    plans, lens, counts = _setup(torch)
    try:
        with pytest.raises(irs.IrsError) as e:
            irs.irs_make_maps_batched([plans[0].handle, plans[0].handle], [lens[0][0]] * 2,
                                      [lens[0][1]] * 2, [counts[0], counts[1]])
        assert e.value.status == 1
    finally:
        for p in plans:
            p.close()
