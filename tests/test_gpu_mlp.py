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


def test_trained_network_gains_over_the_method_without_it():
    """Train on a field, make maps with the network, with the network zeroed
    (its far-far fluctuation omitted) and with the exact series; judge all
    three against the GPU brute force (per-pixel magnification rel RMS)."""
    torch = require_gpu()
    po, pb = params_pair(*CFG, method=irs.IRS_BRUTE)
    qo = oracle.size(po)
    n = int(round(qo.n_star_paper))
    xy, m = lenses_for(qo, n, shape="equal", seed=21, kappa_star=CFG[0])
    dxy, dm = to_dev(torch, xy, m)
    with irs.Plan(pb) as plan:
        ref, _ = plan.make_map(dxy, dm, with_mag=False)
        plan.sync()
    ref = ref.cpu().numpy().astype(np.float64)
    sel = ref >= 100

    def rms(c):
        c = c.cpu().numpy().astype(np.float64)
        r = (c[sel] - ref[sel]) / ref[sel]
        return float(np.sqrt(np.mean(r * r)))

    _, pi = params_pair(*CFG, method=irs.IRS_INTERP, n_star=n)
    with irs.Plan(pi) as plan:
        ci, _ = plan.make_map(dxy, dm, with_mag=False)
        plan.sync()
    _, plan = _mlp_plan(torch, n_star=n)
    with plan:
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
          f"held-out rel error {rep.valid_rel_rms:.3f}, target rms {rep.target_rms:.3e}")
    assert e_interp <= 1e-3
    assert e_mlp < e_zero, "the trained network must reduce the map error"
