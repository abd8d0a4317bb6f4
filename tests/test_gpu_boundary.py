"""Errors the C ABI reports from the device (include/irs.h: irs_make_map,
irs_plan_sync): a lens outside the plan's lens region gives IRS_ERR_ARG
(Sec. 2.2: the rectangle is both the image plane and the lens plane, or the
circumscribed circle of the circular plane), and a 3 x 3 block of level-1
cells holding more lenses than the interpolated ray pass keeps in shared
memory gives IRS_ERR_OVERFLOW.  Both are status words read by irs_plan_sync;
the plan stays usable afterwards."""
import numpy as np
import pytest

import oracle
from paper_2204_10871_gb300 import irs
from gpu_common import lenses_for, params_pair, require_gpu, to_dev

pytestmark = pytest.mark.gpu

C1 = (0.3, 0.0, 0.3, (-2.5, 2.5, -2.5, 2.5), 64, 9.0)


def _sync_status(plan):
    try:
        plan.sync()
        return 0
    except irs.IrsError as e:
        return e.status


@pytest.mark.parametrize("method", [irs.IRS_BRUTE, irs.IRS_INTERP])
@pytest.mark.parametrize("where", ["right", "below", "nan"])
def test_lens_outside_the_rectangle_is_rejected(method, where):
    torch = require_gpu()
    po, pl = params_pair(*C1, method=method, n_star=150)
    qo = oracle.size(po)
    xy, m = lenses_for(qo, 150, seed=3, kappa_star=0.3)
    h = 1e-6 * (qo.a2 - qo.a1)
    bad = xy.copy()
    if where == "right":
        bad[77] = (qo.a2 + h, 0.5 * (qo.b1 + qo.b2))
    elif where == "below":
        bad[5] = (0.5 * (qo.a1 + qo.a2), qo.b1 - h)
    else:
        bad[149, 0] = np.nan
    with irs.Plan(pl) as plan:
        dxy, dm = to_dev(torch, bad, m)
        plan.make_map(dxy, dm)
        assert _sync_status(plan) == 1  # IRS_ERR_ARG
        # the same lenses moved back inside: the plan is still usable
        dxy, dm = to_dev(torch, xy, m)
        plan.make_map(dxy, dm)
        assert _sync_status(plan) == 0
        # lenses exactly on the rectangle's edges and corners are inside
        edge = xy.copy()
        edge[:4] = [(qo.a1, qo.b1), (qo.a2, qo.b2), (qo.a1, qo.b2), (qo.a2, 0.0)]
        dxy, dm = to_dev(torch, edge, m)
        plan.make_map(dxy, dm)
        assert _sync_status(plan) == 0


@pytest.mark.parametrize("method", [irs.IRS_BRUTE, irs.IRS_INTERP])
def test_lens_outside_the_circle_is_rejected(method):
    """Circular plane: a lens inside the circumscribed circle but outside the
    image rectangle is fine, one beyond the circle is not."""
    torch = require_gpu()
    po, pl = params_pair(*C1, method=method, n_star=150, plane=irs.IRS_PLANE_CIRCLE)
    qo = oracle.size(po)
    xy, m = lenses_for(qo, 150, seed=3, kappa_star=0.3, plane=irs.IRS_PLANE_CIRCLE)
    r = qo.circle_r
    inside = xy.copy()
    inside[0] = (qo.cx, qo.cy + 0.999 * r)  # above the rectangle, inside the circle
    outside = xy.copy()
    outside[0] = (qo.cx + 0.8 * r, qo.cy + 0.8 * r)  # 1.13 r from the centre
    with irs.Plan(pl) as plan:
        dxy, dm = to_dev(torch, inside, m)
        plan.make_map(dxy, dm)
        assert _sync_status(plan) == 0
        dxy, dm = to_dev(torch, outside, m)
        plan.make_map(dxy, dm)
        assert _sync_status(plan) == 1


def test_lens_check_in_batched_maps():
    torch = require_gpu()
    po, pl = params_pair(*C1, method=irs.IRS_INTERP, n_star=150)
    qo = oracle.size(po)
    xy, m = lenses_for(qo, 150, seed=3, kappa_star=0.3)
    bad = xy.copy()
    bad[10] = (qo.a1 - 0.5, qo.b1)
    plans = [irs.Plan(pl), irs.Plan(pl)]
    try:
        lens = [to_dev(torch, xy, m), to_dev(torch, bad, m)]
        counts = [torch.zeros((64, 64), dtype=torch.uint32, device="cuda") for _ in plans]
        irs.irs_make_maps_batched([p.handle for p in plans], [l[0] for l in lens], [l[1] for l in lens], counts)
        assert _sync_status(plans[0]) == 0
        assert _sync_status(plans[1]) == 1
    finally:
        for p in plans:
            p.close()


def test_crowded_block_reports_overflow():
    """More than 1024 lenses in one 3 x 3 block of level-1 cells (a plan sized
    for 150 lenses given 1100 in a clump 0.05 theta_E wide): the ray pass keeps
    the first 1024 of them and the plan reports IRS_ERR_OVERFLOW; a normal
    field afterwards syncs clean."""
    torch = require_gpu()
    po, pl = params_pair(*C1, method=irs.IRS_INTERP, n_star=150)
    qo = oracle.size(po)
    rng = np.random.default_rng(12)
    clump = np.stack([0.5 * (qo.a1 + qo.a2) + rng.uniform(-0.025, 0.025, 1100),
                      0.5 * (qo.b1 + qo.b2) + rng.uniform(-0.025, 0.025, 1100)], 1)
    mc = np.full(1100, 1e-3)
    with irs.Plan(pl) as plan:
        assert plan.info.cell_x > 0.2  # the clump sits in one cell and its neighbours
        dxy, dm = to_dev(torch, clump, mc)
        plan.make_map(dxy, dm)
        assert _sync_status(plan) == 6  # IRS_ERR_OVERFLOW
        xy, m = lenses_for(qo, 150, seed=3, kappa_star=0.3)
        dxy, dm = to_dev(torch, xy, m)
        plan.make_map(dxy, dm)
        assert _sync_status(plan) == 0


def test_size_limits_are_rejected_at_plan_time():
    """Limits that the kernels' index arithmetic and FP32 ranges need, checked
    by irs_plan before any allocation of note: the interpolated ray pass's
    pixel keys need maps below 2^21 pixels per side (IRS_ERR_OVERFLOW), and
    the default brute-force kernel's four-row reciprocal needs a plane
    diagonal of at most 1e4 theta_E (IRS_ERR_UNSUPPORTED; a variant with
    reciprocals shared by two rows serves such planes)."""
    require_gpu()
    _, pl = params_pair(0.3, 0.0, 0.3, (-1.0, 1.0, -1.0, 1.0), (1 << 21, 1), 1e-6, method=irs.IRS_INTERP)
    with pytest.raises(irs.IrsError) as e:
        irs.Plan(pl)
    assert e.value.status == 6
    big = (-5000.0, 5000.0, -5000.0, 5000.0)
    _, pb = params_pair(0.1, 0.0, 0.1, big, 16, 1e-3, method=irs.IRS_BRUTE)
    with pytest.raises(irs.IrsError) as e:
        irs.Plan(pb)
    assert e.value.status == 8
    _, pb11 = params_pair(0.1, 0.0, 0.1, big, 16, 1e-3, method=irs.IRS_BRUTE, kernel_variant=11)
    with irs.Plan(pb11) as plan:
        assert plan.info.circle_r * 2 > 1e4
