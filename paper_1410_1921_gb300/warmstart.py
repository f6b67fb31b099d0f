"""Learned warm start: LB-solved training fields, U-Net training, warm solves.

Orchestration only: every step runs in the library's kernels (reconstruction,
labelling, pore size, LB solves, U-Net forward/backward/Adam, warm-start
initialisation).  Training targets are assembled on the host from the solved
fields (data preparation, outside the solve path).

Targets per voxel, the network's output channels in the order of `fields`:
"ux" = u_x / U0 with U0 = g L0^2 / nu (L0 = 10 lattice units), "c" = C -
C_lin(x), the concentration's departure from the linear inlet-outlet profile;
the loss is taken over the node set.  Inputs: pore mask and d / 60 nm.

Refining form (coarse=True): a third input channel holds the departure of
the structure's 2x-coarsened diffusion solution (solved, then carried to the
fine voxels), and the network predicts the fine solution's difference from
it; the warm start is the coarse solution plus the prediction.
"""
import time

import numpy as np
import torch

from . import (OM_ENOPERC, OM_F32, OM_OK, OM_PORE_CHORD13, Batch, Diffusion, Flow, NodeSet, UNet, diff_params, domain,
               flow_params, om_coarsen2_dev, om_label_connectivity_dev, om_local_pore_diameter_dev,
               om_prolong2_dev, om_reconstruct_dev, om_unet_pack_structure, om_unet_pack_structure3, recon_params)

D_SCALE = 1.0 / 60.0
L0 = 10.0
FIELDS = ("ux", "c")


def velocity_scale(fp):
    nu = (fp.tau - 0.5) / 3.0
    return fp.body_force * L0 * L0 / nu


def structure(cfg, stream=None):
    """Reconstruct, label and size one structure on the device.  Returns
    (dom, mask, transport, d_nm) as flat CUDA tensors."""
    dom = domain(cfg.shape, cfg.dx_nm)
    N = dom.nx * dom.ny * dom.nz
    mask = torch.empty(N, dtype=torch.uint8, device="cuda")
    rp = recon_params(cfg.mean_nm, cfg.sd_nm, cfg.dmin_nm, cfg.dmax_nm, cfg.porosity, cfg.xi, cfg.p0, cfg.dist,
                      cfg.max_trials)
    om_reconstruct_dev(cfg.seed, dom, rp, mask, stream=stream)
    tr = torch.empty(N, dtype=torch.uint8, device="cuda")
    om_label_connectivity_dev(mask, dom, None, tr, stream=stream)
    d = torch.empty(N, dtype=torch.float32, device="cuda")
    om_local_pore_diameter_dev(mask, dom, OM_PORE_CHORD13, d, stream=stream)
    return dom, mask, tr, d


def net_input(mask, d, dom, extra=None):
    if extra is None:
        x = torch.empty(mask.numel() * 2, dtype=torch.float32, device="cuda")
        om_unet_pack_structure(mask, d, D_SCALE, x)
        return x.view(1, dom.nx, dom.ny, dom.nz, 2)
    x = torch.empty(mask.numel() * 3, dtype=torch.float32, device="cuda")
    om_unet_pack_structure3(mask, d, D_SCALE, extra, x)
    return x.view(1, dom.nx, dom.ny, dom.nz, 3)


def coarse_level(dom, tr, d):
    """The structure coarsened 2x per axis: (coarse domain, coarse transport
    set, coarse pore sizes); the transport set is None when nothing of the
    coarse structure spans x."""
    dc, mc, d_c = om_coarsen2_dev(tr, dom, d)
    tr_c = torch.empty_like(mc)
    om_label_connectivity_dev(mc, dc, None, tr_c)
    return dc, (tr_c if bool(tr_c.any()) else None), d_c


def prolonged(g_c, tr_c, dom, dp, departure=False, corr=None):
    """Fine float [N] field from the coarse dense populations g_c: the coarse
    concentration (or its departure from C_lin), plus corr if given."""
    c = torch.empty(dom.nx * dom.ny * dom.nz, dtype=torch.float32, device="cuda")
    om_prolong2_dev(g_c, 7, tr_c, dom, dp.c_in, dp.c_out, c, corr_dev=corr, departure=departure)
    return c


def coarse_departure(dom, tr, d, dp):
    """Departure from C_lin of the coarse-level diffusion solution carried to
    the fine voxels (zeros where the coarse structure does not span x)."""
    dc, tr_c, d_c = coarse_level(dom, tr, d)
    if tr_c is None:
        return torch.zeros(dom.nx * dom.ny * dom.nz, dtype=torch.float32, device="cuda")
    ns = NodeSet(tr_c, dc)
    df = Diffusion(ns, d_c, dp)
    df.solve()
    g = torch.empty(7 * dc.nx * dc.ny * dc.nz, dtype=torch.float64, device="cuda")
    df.get_populations(g)
    df.close()
    ns.close()
    return prolonged(g, tr_c, dom, dp, departure=True)


def solve(dom, tr, d, fp, dp, prediction=None, warm_flow=False, fields=FIELDS, flow=True):
    """Flow and diffusion solves on the transport set, cold or warm-started
    from a network output (float [N][len(fields)]): the diffusion from its
    "c" channel, the flow from its "ux" channel only with warm_flow (velocity
    warm starts were measured to slow the flow's convergence: the predicted
    field is not divergence-free and excites slow pressure modes).  flow=False
    skips the flow solve.  Returns a dict of results, step counts, wall times
    and the solved fields (ux, C)."""
    ns = NodeSet(tr, dom)
    out = {"nodes": ns.n_nodes}
    N = tr.numel()
    nch = len(fields)
    if flow:
        t0 = time.perf_counter()
        fl = Flow(ns, fp)
        if prediction is not None and warm_flow and "ux" in fields:
            fl.init_velocity(prediction[fields.index("ux"):], stride=nch, scale=velocity_scale(fp))
        st, kl, info = fl.solve()
        torch.cuda.synchronize()
        out.update(flow_status=st, k_lattice=kl, flow_steps=info.steps, flow_s=time.perf_counter() - t0)
        u = torch.empty(3 * N, dtype=torch.float32, device="cuda")
        fl.get_velocity(u)
        out["ux"] = u[:N].clone()
        fl.close()
    t0 = time.perf_counter()
    df = Diffusion(ns, d, dp)
    if prediction is not None and "c" in fields:
        df.init_concentration(prediction[fields.index("c"):], stride=nch, from_linear=True)
    st, Dl, info = df.solve()
    torch.cuda.synchronize()
    out.update(diff_status=st, D_lattice=Dl, diff_steps=info.steps, diff_s=time.perf_counter() - t0)
    c = torch.empty(N, dtype=torch.float32, device="cuda")
    df.get_fields(c, None)
    out["C"] = c
    df.close()
    ns.close()
    return out


def targets(res, dom, fp, dp, fields=FIELDS):
    """Training target [1, nx, ny, nz, len(fields)] from solved fields (host
    assembly)."""
    ch = []
    for f in fields:
        if f == "ux":
            ch.append(res["ux"].cpu().numpy().reshape(dom.nx, dom.ny, dom.nz) / velocity_scale(fp))
        elif f == "c":
            x = (np.arange(dom.nx) + 0.5)[:, None, None]
            clin = dp.c_in + (dp.c_out - dp.c_in) * x / dom.nx
            ch.append(res["C"].cpu().numpy().reshape(dom.nx, dom.ny, dom.nz) - clin)
        else:
            raise ValueError(f"unknown field {f!r}")
    t = np.stack(ch, -1)[None].astype(np.float32)
    return torch.from_numpy(t).cuda()


def make_dataset(cfgs, fp=None, dp=None, log=None, fields=FIELDS, coarse=False, dp_coarse=None):
    """Solve every structure (cold, FP32) and keep (input, target, mask) of
    those whose solves reached the convergence test (a flow with no link
    across the periodic x boundary counts: its field is exactly u = 0).  The
    flow is solved only when "ux" is among the fields.  coarse: the refining
    form (fields must be ("c",)): the input carries the coarse-level
    departure (solved with dp_coarse) and the target is the fine departure
    minus it."""
    fp = fp or flow_params(precision=OM_F32)
    dp = dp or diff_params(precision=OM_F32)
    flow = "ux" in fields
    if coarse and tuple(fields) != ("c",):
        raise ValueError("the refining form predicts the concentration only")
    data = []
    for cfg in cfgs:
        dom, mask, tr, d = structure(cfg)
        if int(tr.sum().item()) == 0:
            continue
        res = solve(dom, tr, d, fp, dp, flow=flow)
        if (flow and res["flow_status"] not in (OM_OK, OM_ENOPERC)) or res["diff_status"] != OM_OK:
            continue
        t = targets(res, dom, fp, dp, fields)
        extra = None
        if coarse:
            extra = coarse_departure(dom, tr, d, dp_coarse or dp)
            # host-side target assembly: the fine departure minus the coarse one
            t = torch.from_numpy(t.cpu().numpy() - extra.cpu().numpy().reshape(t.shape)).cuda()
        data.append((net_input(mask, d, dom, extra), t, tr.view(1, dom.nx, dom.ny, dom.nz)))
        if log:
            log(f"sample {len(data)}: {cfg.shape} eps={cfg.porosity:.2f} nodes={res['nodes']} "
                f"flow {res.get('flow_steps', 0)} diff {res['diff_steps']} steps")
    return data


def make_dataset_batched(cfgs, fp=None, dp=None, log=None, fields=FIELDS, chunk=64):
    """make_dataset on the batched path: the structures are solved `chunk` at
    a time in one om_batch (diffusion first, then the flow when "ux" is among
    the fields), each to the same convergence test as a single solve, and
    their fields taken with om_batch_get_field.  Returns the samples and the
    count of structures reconstructed."""
    fp = fp or flow_params(precision=OM_F32)
    dp = dp or diff_params(precision=OM_F32)
    flow = "ux" in fields
    data, tried = [], 0
    for c0 in range(0, len(cfgs), chunk):
        group = []
        for cfg in cfgs[c0:c0 + chunk]:
            dom, mask, tr, d = structure(cfg)
            tried += 1
            if int(tr.sum().item()) > 0:
                group.append((cfg, dom, mask, tr, d))
        if not group:
            continue
        b = Batch([g[1] for g in group], [g[3] for g in group], [g[4] for g in group],
                  flow=fp if flow else None, diff=dp)
        _, _, info_d, st_d = b.solve(1)
        st_f = info_f = None
        if flow:
            _, _, info_f, st_f = b.solve(0)
        for j, (cfg, dom, mask, tr, d) in enumerate(group):
            if st_d[j] != OM_OK or (flow and st_f[j] not in (OM_OK, OM_ENOPERC)):
                continue
            N = tr.numel()
            res = {}
            if flow:
                res["ux"] = torch.empty(N, dtype=torch.float32, device="cuda")
                b.get_field(0, j, res["ux"])
            res["C"] = torch.empty(N, dtype=torch.float32, device="cuda")
            b.get_field(1, j, res["C"])
            data.append((net_input(mask, d, dom), targets(res, dom, fp, dp, fields), tr.view(1, dom.nx, dom.ny, dom.nz)))
            if log:
                log(f"sample {len(data)}: {cfg.shape} eps={cfg.porosity:.2f} nodes={int(tr.sum().item())} "
                    f"flow {info_f[j].steps if flow else 0} diff {info_d[j].steps} steps")
        b.close()
    return data, tried


def train(net, data, epochs, lr=1e-3, lr_end=1e-4, seed=0, log=None):
    """Adam over the samples in shuffled order; learning rate decays
    geometrically from lr to lr_end.  Returns the loss history (per epoch)."""
    rng = np.random.default_rng(seed)
    hist = []
    total = max(1, epochs * len(data))
    k = 0
    for ep in range(epochs):
        acc = 0.0
        for i in rng.permutation(len(data)):
            x, t, m = data[i]
            rate = lr * (lr_end / lr) ** (k / total)
            acc += net.train_step(x, t, m, rate)
            k += 1
        hist.append(acc / len(data))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def predict(net, mask, d, dom, extra=None):
    """Network output, flat float [N][net.out_ch] on the device (extra: the
    coarse departure input of the refining form)."""
    x = net_input(mask, d, dom, extra)
    y = torch.empty(mask.numel() * net.out_ch, dtype=torch.float32, device="cuda")
    net.forward(x, y)
    return y
