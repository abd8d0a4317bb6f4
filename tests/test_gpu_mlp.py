"""The learned far field: the tensor-core network kernels against the FP64
network reference (oracle/mlp_oracle.py), and what a trained network gains over
the same method without it.

Gradient bar: the GPU computes with BF16 operands and FP32 accumulation, so
the batch gradient must agree with the FP64 reference to 3e-2 in relative L2
norm (BF16 keeps 8 significant bits: ~4e-3 per operand, a few layers deep).
"""
import numpy as np
import pytest

import oracle
from oracle import mlp_oracle as mo
from paper_2204_10871_gb300 import irs
from gpu_common import lenses_for, params_pair, require_gpu, to_dev

pytestmark = pytest.mark.gpu

CFG = (0.4, 0.1, 0.35, (-2.0, 2.0, -2.0, 2.0), 64, 16.0)


def _mlp_plan(torch, n_star=0):
    po, pl = params_pair(*CFG, method=irs.IRS_MLP, n_star=n_star)
    return po, irs.Plan(pl)


def test_network_forward_and_gradient_match_reference():
    torch = require_gpu()
    rng = np.random.default_rng(3)
    theta = (mo.init_params(5) + rng.normal(0, 0.02, mo.N_PARAMS)).astype(np.float32)
    B = rng.normal(0, 2.0, (32, 2)).astype(np.float32)
    x = rng.uniform(-1, 1, (300, 2)).astype(np.float32)
    t = rng.normal(0, 1, (300, 8)).astype(np.float32)
    _, plan = _mlp_plan(torch)
    with plan:
        th_out, fr_out = irs.irs_mlp_params(plan.handle, theta, B)
        assert np.array_equal(th_out, theta) and np.array_equal(fr_out, B)
        dx = torch.from_numpy(x).cuda()
        dt = torch.from_numpy(t).cuda()
        y = irs.irs_mlp_forward(plan.handle, dx).cpu().numpy()
        grad, lsum = irs.irs_mlp_grad(plan.handle, dx, dt)
        plan.sync()
        grad = grad.cpu().numpy().astype(np.float64)
        lsum = float(lsum.cpu().numpy()[0])
    yo, _ = mo.forward(theta.astype(np.float64), B.astype(np.float64), x.astype(np.float64))
    assert np.abs(y - yo).max() <= 3e-2 * np.sqrt(np.mean(yo ** 2))
    lo = mo.loss(theta.astype(np.float64), B.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(lsum / (300 * 8) - lo) <= 1e-2 * lo
    go = mo.backward(theta.astype(np.float64), B.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    rel = np.linalg.norm(grad - go) / np.linalg.norm(go)
    assert rel <= 3e-2, f"gradient relative L2 error {rel:.3e}"
    # every parameter block moves in the same direction as the reference
    for name, k0, k1 in [("W1", 0, 4096), ("W2", 4160, 8256), ("W3", 8320, 12416), ("W4", 12480, 12992),
                         ("b4", 12992, 13000)]:
        c = grad[k0:k1] @ go[k0:k1] / (np.linalg.norm(grad[k0:k1]) * np.linalg.norm(go[k0:k1]))
        assert c > 0.999, name


# A field large enough that the network, not the exact corner-zone sums,
# carries most cells: 4000 lenses over a 137 x 24 theta_E plane (cells of
# 0.91 theta_E, 150 x 27 of them), R_f = 8 cells, so the corner zones (cells
# within 1.5 R_f of a corner) hold ~11 % of the cells.
CFG_FIELD = (0.4, 0.1, 0.35, (-4.0, 4.0, -4.0, 4.0), 128, 25.0)
N_FIELD = 4000
# Measured on one GB300 (seeded field and training): 0.19 on this field (0.56
# with the network zeroed); at the learned workload, 0.74-0.96 per-pixel
# magnification rel RMS from the brute force over split radii R_f of 4-32
# cells, the network's deflection error ~1e-2 theta_E at every R_f, four
# orders above the ~1e-6 theta_E that a 1e-3 map needs.  The bound below is
# the best the network reaches here, with room for the run-to-run spread of
# the training (atomic gradient sums).
LEARNED_BEST = 0.3


def test_trained_network_gains_over_the_method_without_it():
    """Train on a field, make maps with the network, with the network zeroed
    (its far-far remainder omitted) and with the exact series; judge all
    three against the GPU brute force (per-pixel magnification rel RMS over
    pixels with >= 100 rays).  The learned map must beat the one without the
    network and stay at the best error measured for it; the 1e-3 bar of the
    series form is out of its reach (see LEARNED_BEST)."""
    torch = require_gpu()
    po, pb = params_pair(*CFG_FIELD, method=irs.IRS_BRUTE)
    qo = oracle.size(po)
    xy, m = lenses_for(qo, N_FIELD, shape="equal", seed=21, kappa_star=CFG_FIELD[0])
    dxy, dm = to_dev(torch, xy, m)
    with irs.Plan(pb) as plan:
        ref, _ = plan.make_map(dxy, dm, with_mag=False)
        plan.sync()
    ref = ref.cpu().numpy().astype(np.float64)
    sel = ref >= 100
    assert sel.sum() > 5000

    def rms(c):
        c = c.cpu().numpy().astype(np.float64)
        r = (c[sel] - ref[sel]) / ref[sel]
        return float(np.sqrt(np.mean(r * r)))

    _, pi = params_pair(*CFG_FIELD, method=irs.IRS_INTERP, n_star=N_FIELD)
    with irs.Plan(pi) as plan:
        ci, _ = plan.make_map(dxy, dm, with_mag=False)
        plan.sync()
    _, pm = params_pair(*CFG_FIELD, method=irs.IRS_MLP, n_star=N_FIELD, window=8)
    with irs.Plan(pm) as plan:
        info = plan.info
        # share of ray cells in the corner zones (exact far-far sums there)
        h = info.cell_x
        cx = info.lens_x0 + (np.arange(info.ncell_x) + 0.5) * h
        cy = info.lens_y0 + (np.arange(info.ncell_y) + 0.5) * h
        X, Y = np.meshgrid(cx, cy)
        near = np.zeros_like(X, dtype=bool)
        for x0 in (info.lens_x0, info.lens_x1):
            for y0 in (info.lens_y0, info.lens_y1):
                near |= np.hypot(X - x0, Y - y0) < 1.5 * 8 * h
        assert near.mean() < 0.25, f"corner zones hold {near.mean():.0%} of the cells"
        fallback, _ = plan.make_map(dxy, dm, with_mag=False)  # untrained: exact series
        rep = irs.irs_mlp_train(plan.handle, dxy, dm, n_samples=1 << 18, steps=1500, seed=7)
        assert rep.trained == 1 and rep.loss_final < rep.loss_first
        assert 0.0 < rep.valid_rel_rms < 1.0
        cm, _ = plan.make_map(dxy, dm, with_mag=False)
        theta, B = irs.irs_mlp_params(plan.handle)
        irs.irs_mlp_params(plan.handle, np.zeros_like(theta), B)  # network zeroed
        c0, _ = plan.make_map(dxy, dm, with_mag=False)
        plan.sync()
    assert torch.equal(fallback, ci)
    e_interp, e_mlp, e_zero = rms(ci), rms(cm), rms(c0)
    print(f"\nrel RMS vs brute: interp {e_interp:.3e}, learned {e_mlp:.3e}, without network {e_zero:.3e}; "
          f"held-out rel error {rep.valid_rel_rms:.3f}, target rms {rep.target_rms:.3e}, "
          f"corner-zone cells {near.mean():.1%}")
    assert e_interp <= 1e-3
    assert e_mlp < e_zero, "the trained network must reduce the map error"
    assert e_mlp <= LEARNED_BEST, f"learned map rel RMS {e_mlp:.3e} above its measured best"
