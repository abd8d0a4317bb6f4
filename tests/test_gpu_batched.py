"""irs_make_maps_batched: many uneven maps in one captured CUDA graph give the
same count maps as one irs_make_map per map, on the first call (capture) and
on replays, including replays after the lens values changed in place and
after a plan's lens buffers were reallocated; and every batched map matches
the FP64 oracle at the misbinning bar, a 500^2 map with 1e4 lenses among
them."""
import numpy as np
import pytest

import oracle
from paper_2204_10871_gb300 import irs
from gpu_common import MISBIN_TOL, lenses_for, misbinned, params_pair, require_gpu, to_dev

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


# Maps of the oracle comparison: uneven kappa, gamma, N_* and sizes, rays per
# pixel kept low enough that the oracle shoots all of them in ~25 s on 16
# cores; a 500^2 map with 1e4 lenses (the smallest maps of the 256-map
# batched workload have this size) and a map without lenses.
MAPS_ORACLE = [
    (0.30, 0.00, 0.30, 4.0, 96, 16.0, 400, irs.IRS_INTERP, 0),
    (0.55, 0.25, 0.15, 3.0, 64, 4.0, 900, irs.IRS_INTERP, 1),
    (0.12, 0.08, 0.55, 5.0, 120, 9.0, 150, irs.IRS_INTERP, 2),
    (0.40, 0.10, 0.35, 2.5, 50, 9.0, 1500, irs.IRS_INTERP, 3),
    (0.20, 0.00, 0.10, 2.0, 40, 16.0, 60, irs.IRS_BRUTE, 0),
    (0.45, 0.05, 0.45, 3.0, 80, 4.0, 2000, irs.IRS_INTERP, 0),
    (0.10, 0.00, 0.10, 10.0, 500, 4.0, 10000, irs.IRS_INTERP, 0),
    # no lenses: the smooth terms alone; at 10.25 rays per pixel every ray of
    # the regular lattice lands >= 5.8e-3 pixel from a pixel edge (checked
    # with the oracle's sizing: a lens-free ray on an edge goes to either side
    # by rounding, FP64 in the oracle, FP32 here)
    (0.20, 0.10, 0.20, 3.0, 48, 10.25, 0, irs.IRS_INTERP, 13),
]


def _setup(torch, maps=MAPS):
    plans, lens, counts = [], [], []
    for k, (ks, kss, g, S, npix, nav, nst, meth, var) in enumerate(maps):
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
                    xy.mul_(0.99)  # towards the plane centre (the origin): still inside
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


def test_batched_after_a_plan_reallocated_its_lens_buffers():
    """A batched call, then irs_make_map on one of the plans with more lenses
    than its buffers hold (they are reallocated), then the batched call again
    with the first lenses: the second call must not replay the graph captured
    on the freed buffers, and every map must equal the single-call map."""
    torch = require_gpu()
    plans, lens, counts = _setup(torch)
    try:
        handles = [p.handle for p in plans]
        xs = [l[0] for l in lens]
        ms = [l[1] for l in lens]
        irs.irs_make_maps_batched(handles, xs, ms, counts)
        torch.cuda.synchronize()
        ks, kss, g, S, npix, nav, nst, meth, var = MAPS[0]
        po, _ = params_pair(ks, kss, g, (-S / 2, S / 2, -S / 2, S / 2), npix, nav)
        qo = oracle.size(po)
        big_xy, big_m = lenses_for(qo, 4 * nst, shape="uniform", seed=99, kappa_star=ks)
        bxy, bm = to_dev(torch, big_xy, big_m)
        ws0 = plans[0].info.workspace_bytes
        plans[0].make_map(bxy, bm, with_mag=False)  # grows (moves) plan 0's lens buffers
        torch.cuda.synchronize()
        assert irs.irs_plan_info_get(plans[0].handle).workspace_bytes > ws0
        for c in counts:
            c.fill_(77)
        irs.irs_make_maps_batched(handles, xs, ms, counts)
        torch.cuda.synchronize()
        ref = _singles(torch, plans, lens)
        for k, (c, r) in enumerate(zip(counts, ref)):
            assert np.array_equal(c.cpu().numpy(), r), f"map {k}"
        for p in plans:
            p.sync()
    finally:
        for p in plans:
            p.close()


def test_batched_maps_match_the_oracle():
    """Every map of a batched call against the FP64 oracle's brute force on the
    same lenses (all rays, every lens), at the misbinning bar."""
    torch = require_gpu()
    plans, lens, counts = _setup(torch, MAPS_ORACLE)
    try:
        irs.irs_make_maps_batched([p.handle for p in plans], [l[0] for l in lens], [l[1] for l in lens],
                                  counts)
        torch.cuda.synchronize()
        for p in plans:
            p.sync()
        for k, (ks, kss, g, S, npix, nav, nst, meth, var) in enumerate(MAPS_ORACLE):
            po, _ = params_pair(ks, kss, g, (-S / 2, S / 2, -S / 2, S / 2), npix, nav)
            qo = oracle.size(po)
            xy, m = lenses_for(qo, nst, shape="uniform", seed=40 + k, kappa_star=ks)
            co, _, landed = oracle.make_map(po, qo, xy, m)
            bad = misbinned(co, counts[k].cpu().numpy())
            print(f"\nmap {k}: {npix}^2 px, {nst} lenses, {landed} rays landed, {bad} binned differently")
            assert bad <= max(1, MISBIN_TOL * landed), f"map {k}: {bad} of {landed} rays binned differently"
    finally:
        for p in plans:
            p.close()
