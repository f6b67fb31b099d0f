"""The learned warm start end to end, at a size that runs in a minute: LB-
solved training fields, U-Net training on the GPU with the library's own
kernels, and warm-started solves on held-out structures.

What the trained network gains over the method without it: on held-out
structures its concentration field is closer to the converged one than the
cold start (the linear profile), the warm-started diffusion solves need
fewer LB steps in total to meet the same convergence test, and cold and
warm land on the same D_eff -- both within the FP32 bound (1e-5) of an FP64
solve converged 1e4 times tighter.  The LB, not the network, decides the
result.

The test is a relative change below 1e-7 over 1000 steps: at 1e-6 a solve
on these structures still stops ~1.5e-5 away from its fixed point (the
slowest mode decays over ~1e4 steps), cold or warm, so only the tighter test
can show agreement at the FP32 bound.  Measured on these structures: 4 %
fewer steps warm than cold, every structure fewer; the assertion asks for
1 % (the training's split-K weight gradients are summed by atomics, so the
network differs slightly from run to run)."""
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _cfg(seed, eps):
    return S.Recon(seed, (32, 32, 32), 1.0, 12.0, 3.0, 6.0, 20.0, eps, 0.3)


@pytest.mark.timeout(900)
def test_warm_start_saves_steps_and_keeps_results(om):
    from paper_1410_1921_gb300 import warmstart as W
    fp = om.flow_params(conv_tol=1e-6, check_every=1000, max_steps=400_000)
    dp = om.diff_params(conv_tol=1e-7, check_every=1000, max_steps=2_000_000)
    train_cfgs = [_cfg(100 + i, (0.30, 0.38, 0.45)[i % 3]) for i in range(18)]
    fields = ("c",)  # the concentration channel warm-starts the diffusion
    data = W.make_dataset(train_cfgs, fp, dp, fields=fields)
    assert len(data) >= 10
    net = om.UNet(2, 1, (16, 32, 64), seed=3)
    hist = W.train(net, data, epochs=40, lr=1e-3, lr_end=1e-4)
    assert hist[-1] < 0.5 * hist[0]
    cold_steps = warm_steps = n = 0
    err_cold = err_warm = 0.0
    for cfg in (_cfg(900, 0.35), _cfg(901, 0.42), _cfg(902, 0.38), _cfg(903, 0.33), _cfg(904, 0.45)):
        dom, mask, tr, d = W.structure(cfg)
        if int(tr.sum().item()) == 0:
            continue
        ns = om.NodeSet(tr, dom)
        df = om.Diffusion(ns, d, om.diff_params(precision=om.OM_F64, conv_tol=1e-11, check_every=1000,
                                                max_steps=5_000_000, accel=om.OM_ACCEL_EXTRAPOLATE))
        st, D_ref, _ = df.solve()
        df.close()
        ns.close()
        assert st == om.OM_OK
        pred = W.predict(net, mask, d, dom)
        cold = W.solve(dom, tr, d, fp, dp)
        warm = W.solve(dom, tr, d, fp, dp, prediction=pred, fields=fields)
        assert cold["flow_status"] in (om.OM_OK, om.OM_ENOPERC)
        assert warm["flow_status"] == cold["flow_status"]
        assert cold["diff_status"] == om.OM_OK and warm["diff_status"] == om.OM_OK
        # the same fixed point, met by the same test: within the FP32 bound
        assert cold["D_lattice"] == pytest.approx(D_ref, rel=1e-5)
        assert warm["D_lattice"] == pytest.approx(D_ref, rel=1e-5)
        assert warm["D_lattice"] == pytest.approx(cold["D_lattice"], rel=1e-5)
        assert warm["k_lattice"] == pytest.approx(cold["k_lattice"], rel=1e-5, abs=1e-12)
        # the network's field is nearer the converged one than the linear profile
        t = tr.bool()
        x = (torch.arange(dom.nx, device="cuda", dtype=torch.float32) + 0.5) / dom.nx
        clin = (dp.c_in + (dp.c_out - dp.c_in) * x)[:, None].expand(dom.nx, dom.ny * dom.nz).reshape(-1)
        err_cold += (clin - cold["C"])[t].norm().item() ** 2
        err_warm += (clin + pred - cold["C"])[t].norm().item() ** 2
        cold_steps += cold["diff_steps"]
        warm_steps += warm["diff_steps"]
        n += 1
    assert n >= 3 and err_warm < 0.9 * err_cold
    assert warm_steps <= 0.99 * cold_steps, (warm_steps, cold_steps)
