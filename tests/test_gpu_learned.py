"""The learned relaxation weights on the GPU against the oracle: the weighted smoother with
fixed weights, the network's inference, the training loss and gradient, and the per-V-cycle
acceptance mode."""
import numpy as np
import pytest

import oracle as O
from oracle import learned as NL
from paper_1807_02137_gb300 import synth
from tests.gpu_common import gpu_solver, need_gpu, oracle_params, relmax, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def segmg():
    return need_gpu()


def _weights(shape, seed):
    return np.random.default_rng(seed).uniform(0.4, 1.6, shape)


def test_fixed_weights_match_oracle(segmg):
    img, mk, _ = synth.ellipses(150, 133, 6, (20, 70), 5, 0.05, 31)
    # FP64: per V-cycle against the oracle with the same weights on grids 0 and 1
    s, p = gpu_solver(segmg, img, mk, precision=segmg.MG_F64, levels=4, smoother=segmg.MG_SMOOTH_FUSED_VEC)
    s.set_bottom_kernel(False)
    o = O.Solver(img, mk, oracle_params(150, 133, p))
    for l in (0, 1):
        w = _weights((150 >> l, 133 >> l), 40 + l)
        s.set_omega(l, w)
        o.set_omega(l, w)
    s.begin_step(); o.begin_step()
    for _ in range(3):
        rg, ro = s.vcycle(), o.vcycle()
        assert abs(rg - ro) <= 1e-8 * ro
    assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-10
    # FP32: the TMA and vector-load sweeps agree bitwise with weights
    outs = []
    for sm in (segmg.MG_SMOOTH_FUSED, segmg.MG_SMOOTH_FUSED_VEC):
        s32, _ = gpu_solver(segmg, img.astype(np.float32), mk, precision=segmg.MG_F32, levels=4, smoother=sm)
        s32.set_bottom_kernel(False)
        for l in (0, 1):
            s32.set_omega(l, _weights((150 >> l, 133 >> l), 40 + l))
        s32.begin_step()
        for _ in range(3):
            s32.vcycle()
        outs.append(s32.phi().cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def _theta(seed):
    rng = np.random.default_rng(seed)
    th = rng.normal(0, 0.25, NL.NPARAM)
    th[-1] = 0.1
    return th


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_inference_matches_oracle(segmg, precision):
    # omega of the finest grid from the first snapshot of a V-cycle, against the oracle's
    # network on its own coefficients at the same state (BF16 storage emulated).  Both sides
    # round features and activations to BF16 (8-bit significand); a value whose FP32 (GPU,
    # tensor-core accumulation) and FP64 (oracle) evaluations fall on either side of a BF16
    # rounding boundary differs by one BF16 ulp (2^-8 relative), which moves omega = 2 sigmoid(z)
    # of the cells downstream by at most a few 1e-3 for this network; elsewhere the sides agree to
    # the FP32 accumulation error.  Measured: max 3.4e-3, mean 2.6e-4, 99th percentile 2.0e-3
    # (the same for FP32 and FP64 handles).
    img, mk, _ = synth.ellipses(130, 147, 6, (20, 70), 5, 0.05, 33)
    th = _theta(7)
    prec = segmg.MG_F64 if precision == "f64" else segmg.MG_F32
    s, p = gpu_solver(segmg, img, mk, precision=prec, levels=4)
    s.set_learned(th.astype(np.float32), mode=2, refresh=1)
    o = O.Solver(img, mk, oracle_params(130, 147, p))
    o.begin_step()
    K = O.frozen_coeffs(o.level(0, "phi"), o.level(0, "w"), o.level(0, "Fn"), None, p=o.p)
    x = NL.features(K["A"], K["B"], K["C"], K["D"])
    w_or, _ = NL.forward(th.astype(np.float32).astype(np.float64), x, bf16=True)
    s.begin_step()
    s.vcycle()
    w_gpu = s.level(0, "omega").cpu().numpy()
    d = np.abs(w_gpu.astype(np.float64) - w_or)
    assert d.max() < 1e-2 and d.mean() < 5e-4 and np.quantile(d, 0.99) < 4e-3
    assert 0 < w_gpu.min() and w_gpu.max() < 2


def _crops(count, seed):
    rng = np.random.default_rng(seed)
    recs = np.zeros((count, 7, 24, 24), dtype=np.float32)
    for k in range(count):
        c = np.exp(rng.normal(0, 1.0, (4, 24, 24)))
        recs[k, :4] = c
        recs[k, 4] = rng.normal(size=(24, 24))
        recs[k, 5] = rng.normal(size=(24, 24))
        recs[k, 6, 0, 0] = 0.5
        recs[k, 6, 0, 1] = k % 2
    return recs


@pytest.mark.parametrize("kind", ["full", "hf"])
def test_training_loss_and_gradient_match_oracle(segmg, kind):
    recs = _crops(6, 11)
    th = _theta(12).astype(np.float32)
    t = segmg.Trainer(capacity=16, batch_max=8, seed=1, theta0=th)
    t.set_loss(kind)
    t.load(recs.reshape(6, -1))
    idx = [0, 3, 5, 2]
    loss, g = t.grad(idx)
    lo, go = 0.0, np.zeros(NL.NPARAM)
    for k in idx:
        r = recs[k].astype(np.float64)
        c = r[:4]
        S = c.sum(axis=0) + r[6, 0, 0]
        l1, g1 = NL.crop_loss_grad(th.astype(np.float64), c, S, r[4], r[5], parity0=int(r[6, 0, 1]), loss=kind)
        lo += l1 / len(idx)
        go += g1 / len(idx)
    assert abs(loss - lo) <= 1e-4 * lo
    assert np.linalg.norm(g - go) <= 2e-3 * np.linalg.norm(go)
    # an Adam step lowers the loss of a fixed batch from omega = 1
    t2 = segmg.Trainer(capacity=16, batch_max=8, seed=2)
    t2.set_loss(kind)
    t2.load(recs.reshape(6, -1))
    l0, _ = t2.grad(list(range(6)))
    for _ in range(30):
        t2.train(1, 6, 1e-2)
    l1, _ = t2.grad(list(range(6)))
    assert l1 < l0
    t.close(); t2.close()


def test_learned_mode_keeps_the_solution(segmg):
    # per-V-cycle acceptance: the step still converges to the oracle's solution; learned V-cycles
    # are tried after the first (plain) one, with plain back-off after a rejection
    img, mk, _ = synth.ellipses(256, 256, 12, (10, 60), 8, 0.05, 11)   # converges plain to 1e-6
    s, p = gpu_solver(segmg, img.astype(np.float32), mk, precision=segmg.MG_F32, levels=7)
    t = segmg.Trainer(capacity=64, batch_max=16, seed=3)
    s.set_learned(t.theta(), mode=1, refresh=2)
    cyc, rho = s.solve_step(1e-6, 60)
    st = s.stats()
    assert rho <= 1e-6
    assert 1 <= st["learned_accepted"] + st["learned_rejected"] <= cyc - 1
    o = O.Solver(img.astype(np.float32).astype(np.float64), mk, oracle_params(256, 256, p))
    o.set_tau(st["tau"])
    hist = o.solve_step(1e-9, 80)
    assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-5
    # recording crops from the solver's state
    t.record(s, 10)
    assert t.count == 10
    loss = t.train(3, 8, 1e-3)
    assert np.isfinite(loss)
