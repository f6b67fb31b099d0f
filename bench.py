"""Benchmark of the LB hot path on GB300: fluid lattice updates per second.

Workload (default): the porosity sweep -- four 256^3 structures at 1 nm
(pore spheres d ~ Normal(30, 8) nm, overlap tolerance 0.3, porosity 0.15,
0.25, 0.35, 0.45), reconstructed, labelled and sized (13-direction pore
size) before the timed region.  One step = for every structure one
convergence window of the D3Q19 flow sweep (100 LB steps) and its
convergence check, then one window of the D3Q7 Knudsen diffusion sweep and
its check, with FP32 populations -- every row of the hot path once.

value: fluid MLUPS over both models, whole job (all ranks).
e2e:   the same metric through the host-buffer C ABI (om_solve_permeability
       + om_solve_knudsen with a one-window step cap), host mask and pore
       sizes copied in and the results copied out inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as S  # noqa: E402

WINDOW = 100  # LB steps per convergence check
BYTES_FLOW_F32 = 152  # 19 populations read + written, 4 B each
BYTES_DIFF_F32 = 60  # 7 populations read + written + omega
METRIC = "fluid MLUPS & %HBM roofline"
UNIT = "MLUPS"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--edge", type=int, default=256, help="structure edge (default: the 256^3 sweep)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-converge", action="store_true", help="skip the time-to-converged-results leg")
    ap.add_argument("--mode", default="throughput",
                    choices=["throughput", "converge", "batch", "precision", "warmstart", "layout", "unet"],
                    help="converge: time to converged k and D_eff, plain vs batched + FP16 + warm start; "
                         "batch: the 150-structure set in one batch; precision: a 512^3 structure with "
                         "FP32, FP16 and BF16 population storage; warmstart: the learned warm start "
                         "trained on --n-train 96^3 structures, held-out 128^3 and 256^3 structures; layout: "
                         "the sparse and the dense population layouts on 128^3 structures of rising porosity")
    ap.add_argument("--train-edge", type=int, default=96, help="warmstart mode: training box edge")
    ap.add_argument("--eval-edges", default="128,256", help="warmstart mode: held-out box edges")
    ap.add_argument("--unet-shape", default="4,64,32-64-128",
                    help="unet mode: batch, box edge and channels per level")
    ap.add_argument("--n-struct", type=int, default=150, help="batch mode: structures")
    ap.add_argument("--batch-set", default="150", choices=["150", "small"],
                    help="batch mode: the 150-structure set, or 20 structures of 64^3 drawn like it")
    ap.add_argument("--batch-split", action="store_true",
                    help="batch mode: also time the structures of >= 2^19 nodes and the rest apart")
    ap.add_argument("--n-eval", type=int, default=24, help="converge mode: structures solved")
    ap.add_argument("--n-train", type=int, default=96, help="converge mode: training structures")
    ap.add_argument("--epochs", type=int, default=60, help="converge mode: U-Net epochs")
    ap.add_argument("--max-steps", type=int, default=500_000, help="converge mode: step cap per solve")
    ap.add_argument("--warm", default="diffusion",
                    choices=["both", "diffusion", "none", "coarse", "coarse-both", "coarse+net"],
                    help="converge mode: which models the network warm-starts (velocity warm starts "
                         "measured to slow the flow's convergence); 'coarse': the diffusion starts from a "
                         "batched solve of the structures coarsened 2x per axis instead of the network; "
                         "'coarse-both': the flow too, from a coarse flow solve; "
                         "'coarse+net': from that solve refined by the network")
    return ap.parse_args()


def _workload(edge, rank):
    """Weak scaling: every rank solves its own four sweep structures (seeds
    offset by rank); no data crosses ranks."""
    return [S.sweep_structure(e, seed=1 + 1000 * rank, edge=edge) for e in S.SWEEP_POROSITIES]


def job_totals(updates, ms, world, device):
    """Whole-job figures: lattice updates summed over ranks, time the
    slowest rank's.  The only collective of the benchmark."""
    if world == 1:
        return float(updates), float(ms)
    import torch
    import torch.distributed as dist
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def _workload_name(edge):
    return (f"porosity sweep: 4 structures {edge}^3 @ 1 nm, d~N(30,8) nm, xi=0.3, "
            f"eps in {{0.15,0.25,0.35,0.45}}; D3Q19 flow (tau=1, g=1e-6) + D3Q7 Knudsen diffusion, "
            f"FP32, {WINDOW}-step windows with convergence checks")


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.lines, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for n, v in zip(names, p[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peak_hbm():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic_record():
    """DRAM bytes per launch of the D3Q19 sweep from a committed ncu summary,
    valid only while the kernel's sources are unchanged."""
    path = os.path.join(ROOT, "profiles", "d3q19_sweep_traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    h = hashlib.sha256()
    for f in ("flow.cu", "flow_core.cuh", "lattice.cuh", "common.cuh", "nodeset.cu"):
        h.update(open(os.path.join(ROOT, "paper_1410_1921_gb300", "csrc", f), "rb").read())
    if rec.get("source_sha256") != h.hexdigest():
        return None
    return rec


# ------------------------------------------------------------------ reference arm: the oracle
def _oracle_sample(edge):
    """One flow and one diffusion step of the oracle on the porosity-0.35
    structure (the oracle's own reconstruction), cropped to 64 x-layers."""
    import oracle
    cfg = S.sweep_structure(0.35, seed=1, edge=edge)
    rc, mask, *_ = oracle.reconstruct(cfg.seed, cfg.shape, cfg.dx_nm, cfg.mean_nm, cfg.sd_nm, cfg.dmin_nm,
                                      cfg.dmax_nm, cfg.porosity, cfg.xi, cfg.p0, cfg.dist)
    _, tr, _ = oracle.label18(mask)
    tr = np.ascontiguousarray(tr[: min(64, edge)])
    om_ = np.where(tr == 1, 1.0 / oracle.tau_knudsen(30.0), 0.0)  # uniform 30 nm pores (Eq. 12)
    f = oracle.flow_init(tr)
    g = oracle.diff_init(tr)
    nf = int(tr.sum())

    def step():
        nonlocal f, g
        f = oracle.flow_step(tr, f, 1.0, 1e-6, 1)
        g = oracle.diff_step(tr, g, om_, 1.0, 0.0, 1)
        return 2 * nf

    desc = (f"oracle (FP64 C, 1 thread): 1 D3Q19 MRT + 1 D3Q7 step on the eps=0.35 {edge}^3 structure "
            f"cropped to {tr.shape[0]} x-layers ({nf} nodes)")
    return step, desc


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    step, desc = _oracle_sample(a.edge)
    for _ in range(a.warmup):
        step()
    t0 = time.perf_counter()
    ups = sum(step() for _ in range(a.steps))
    dt = time.perf_counter() - t0
    v = ups / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_name(a.edge), "sample": desc},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def run_gpu(a):
    import torch
    import torch.distributed as dist

    from paper_1410_1921_gb300 import build as B
    B.build()
    import paper_1410_1921_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    sp = P._stream(stream)

    # ---------------- setup (untimed): reconstruct, label, pore size, solvers
    cfgs = _workload(a.edge, rank)
    solvers, host_inputs = [], []
    t_setup = time.perf_counter()
    with torch.cuda.stream(stream):
        for cfg in cfgs:
            dom = P.domain(cfg.shape, cfg.dx_nm)
            N = dom.nx * dom.ny * dom.nz
            mask = torch.empty(N, dtype=torch.uint8, device="cuda")
            rp = P.recon_params(cfg.mean_nm, cfg.sd_nm, cfg.dmin_nm, cfg.dmax_nm, cfg.porosity, cfg.xi, cfg.p0)
            P.om_reconstruct_dev(cfg.seed, dom, rp, mask, stream=sp)
            tr = torch.empty(N, dtype=torch.uint8, device="cuda")
            P.om_label_connectivity_dev(mask, dom, None, tr, stream=sp)
            d = torch.empty(N, dtype=torch.float32, device="cuda")
            P.om_local_pore_diameter_dev(mask, dom, P.OM_PORE_CHORD13, d, stream=sp)
            ns = P.NodeSet(tr, dom, stream=sp)
            if ns.n_nodes == 0:
                continue
            fl = P.Flow(ns, P.flow_params(precision=P.OM_F32, check_every=WINDOW), stream=sp)
            df = P.Diffusion(ns, d, P.diff_params(precision=P.OM_F32, check_every=WINDOW), stream=sp)
            solvers.append((cfg, ns, fl, df))
            # the e2e inputs live in pinned host memory (numpy views of pinned tensors)
            hm = torch.empty(mask.shape, dtype=mask.dtype, pin_memory=True)
            hd = torch.empty(d.shape, dtype=d.dtype, pin_memory=True)
            hm.copy_(mask)
            hd.copy_(d)
            host_inputs.append((dom, hm.numpy(), hd.numpy()))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    nodes = [ns.n_nodes for _, ns, _, _ in solvers]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in solvers]

    def one_step(record):
        for k, (cfg, ns, fl, df) in enumerate(solvers):
            if record:
                ev[k][0].record(stream)
            fl.step(WINDOW, stream=sp)
            if record:
                ev[k][1].record(stream)
            fl.observe(stream=sp)
            df.step(WINDOW, stream=sp)
            df.observe(stream=sp)

    for _ in range(a.warmup):
        one_step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    flow_ms = 0.0
    torch.cuda.nvtx.range_push("timed")  # lets a profiler take the launches of the timed steps only
    t0.record(stream)
    for _ in range(a.steps):
        one_step(True)
        torch.cuda.synchronize()
        flow_ms += sum(e0.elapsed_time(e1) for e0, e1 in ev)
    t1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ms = t0.elapsed_time(t1)
    ck = clocks.stop()
    updates = 2 * WINDOW * sum(nodes) * a.steps  # both models
    total_updates, ms = job_totals(updates, ms, world, "cuda")
    flow_updates, _ = job_totals(WINDOW * sum(nodes) * a.steps, 0.0, world, "cuda")
    value = total_updates / (ms * 1e-3) / 1e6

    # dominant kernel: D3Q19 sweep, algorithmic bytes per launch / event time
    flow_launches = WINDOW * len(solvers) * a.steps
    flow_bytes = BYTES_FLOW_F32 * WINDOW * sum(nodes) * a.steps
    achieved = flow_bytes / (flow_ms * 1e-3) / 1e9
    peak, peak_kind = _peak_hbm()
    trec = _traffic_record()
    roofline = {"bound": "hbm", "kernel": "d3q19_sweep<float>", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                "avg_launch_us": flow_ms * 1e3 / flow_launches,
                "algorithmic_bytes_per_launch": BYTES_FLOW_F32 * sum(nodes) / len(solvers),
                "traffic": trec["dram_bytes_per_launch"] if trec else None}

    # ---------------- e2e through the host-buffer C ABI
    fp = P.flow_params(precision=P.OM_F32, conv_tol=0.0, check_every=WINDOW, max_steps=WINDOW)
    dp = P.diff_params(precision=P.OM_F32, conv_tol=0.0, check_every=WINDOW, max_steps=WINDOW)
    e2e_steps = max(1, min(2, a.steps))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    te = time.perf_counter()
    e2e_updates = 0
    for _ in range(e2e_steps):
        for dom, m, d in host_inputs:
            try:
                st, k, kl, info, _ = P.om_solve_permeability(m, dom, fp)
                e2e_updates += info.n_nodes * info.steps
            except P.OmError as e:  # no link across the periodic x boundary: k = 0, no flow steps
                if e.status != P.OM_ENOPERC:
                    raise
            st, D, tau, info, _ = P.om_solve_knudsen(m, d, dom, dp)
            e2e_updates += info.n_nodes * info.steps
    te = time.perf_counter() - te
    e2e_updates, te = job_totals(e2e_updates, te, world, "cuda")
    e2e = {"value": e2e_updates / te / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": int(sum(2 * m.nbytes + d.nbytes for _, m, d in host_inputs)),
           "d2h_bytes_per_step": int(len(host_inputs) * 2 * (2 * 8 + 48))}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": _workload_name(a.edge), "structures_per_gpu": len(solvers),
                       "nodes_per_structure": nodes, "window": WINDOW, "precision": "f32",
                       "layout": "fluid-node SoA, AA pattern, rank-indexed neighbours",
                       "l2": f"no flush: populations {sum(nodes) * 4 * 26 / 1e9:.2f} GB per step > 129 MB L2",
                       "setup_s": t_setup},
            "flow_mlups": flow_updates / (flow_ms * 1e-3) / 1e6,
            "roofline": roofline, "clocks": ck, "e2e": e2e,
            # per structure and step: two windows, each model's observe and
            # fixed-order reduction, the diffusion's reference move
            "gpu_launches": a.steps * len(solvers) * (2 * (WINDOW + 2) + 1)}
    if rank == 0 and not a.no_converge:
        from paper_1410_1921_gb300 import warmstart as W
        try:
            line["converge"] = converge_leg(P, W)
        except Exception as exc:  # reported, never a reason to lose the line
            line["converge"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        try:
            step, desc = _oracle_sample(a.edge)
            tc = time.perf_counter()
            ups = sum(step() for _ in range(5))
            tc = time.perf_counter() - tc
            desc = "5 x " + desc
            line["cpu_baseline"] = {"value": ups / tc / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": desc}
        except Exception as exc:  # the baseline is a report, never a reason to lose the line
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {exc}"}
    if rank == 0:
        print(json.dumps(line))
    for _, ns, fl, df in solvers:
        fl.close()
        df.close()
        ns.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ time to converged results
CONV_TOL, CONV_K, CONV_CAP = 1e-6, 1000, 3_000_000  # test: relative change < 1e-6 over 1000 steps
CONV_BOUND = 1e-3  # stated bound on k and D_eff against the tight FP64 reference, both forms


def converge_leg(P, W, n_struct=6, warm="none", fast_diff_prec=None):
    """Wall time to converged k and D_eff on n_struct 64^3 structures drawn
    like the 150-structure set: the plain form (one cold FP32 solve per
    structure and model) against the fast form (all structures in one batch,
    extrapolated restarts of the diffusion, and -- warm="coarse" -- the
    diffusion started from a solve of the structures coarsened 2x per axis).
    Both stop on the same tests: the flow on the relative change of its
    velocity field, the diffusion on that of both its concentration field
    and its net flux, each below 1e-6 over 1000 steps.
    Every result is compared with an FP64 reference converged 1e4-1e5 times
    tighter.  Setup (reconstruction, labelling, pore size) is outside both
    timings; the fast form's batch creation (and coarse solve) is inside.
    The diffusion stays FP32 in both forms: 16-bit storage cannot meet the
    field test at 1e-6 (its rounding floor is ~1e-5)."""
    import torch
    fdp = P.OM_F32 if fast_diff_prec is None else fast_diff_prec
    fp = P.flow_params(precision=P.OM_F32, conv_tol=CONV_TOL, check_every=CONV_K, max_steps=CONV_CAP)
    dp = P.diff_params(precision=P.OM_F32, conv_tol=CONV_TOL, check_every=CONV_K, max_steps=CONV_CAP)
    dpx = P.diff_params(precision=fdp, conv_tol=CONV_TOL, check_every=CONV_K, max_steps=CONV_CAP,
                        accel=P.OM_ACCEL_EXTRAPOLATE)
    structs = []
    for cfg in _converge_set(3 * n_struct, 23, (64,)):
        dom, mask, tr, d = W.structure(cfg)
        if int(tr.sum().item()) > 0:
            structs.append((cfg, dom, tr, d))
        if len(structs) == n_struct:
            break
    # reference: FP64, 1e-11 over 1000 steps (the diffusion with restarts)
    ref = []
    t_ref = time.perf_counter()
    for _, dom, tr, d in structs:
        r = W.solve(dom, tr, d, P.flow_params(precision=P.OM_F64, conv_tol=1e-10, check_every=CONV_K,
                                              max_steps=CONV_CAP),
                    P.diff_params(precision=P.OM_F64, conv_tol=1e-11, check_every=CONV_K, max_steps=CONV_CAP,
                                  accel=P.OM_ACCEL_EXTRAPOLATE))
        ref.append(r)
    t_ref = time.perf_counter() - t_ref
    # plain: one cold FP32 solve per structure and model
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [W.solve(dom, tr, d, fp, dp) for _, dom, tr, d in structs]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    # fast: one batch, extrapolated restarts, two-level warm start
    t0 = time.perf_counter()
    b = P.Batch([s[1] for s in structs], [s[2] for s in structs], [s[3] for s in structs], flow=fp, diff=dpx)
    coarse_steps = 0
    if warm == "coarse":
        cs = [W.coarse_level(dom, tr, d) for _, dom, tr, d in structs]
        keep = [k for k, c in enumerate(cs) if c[1] is not None]
        if keep:
            dpc = P.diff_params(precision=fdp, conv_tol=10 * CONV_TOL, check_every=CONV_K, max_steps=CONV_CAP,
                                accel=P.OM_ACCEL_EXTRAPOLATE)
            bc = P.Batch([cs[k][0] for k in keep], [cs[k][1] for k in keep], [cs[k][2] for k in keep], diff=dpc)
            _, _, info_c, _ = bc.solve(1)
            coarse_steps = int(sum(i.steps for i in info_c))
            for j, k in enumerate(keep):
                dc, tr_c, _ = cs[k]
                g = torch.empty(7 * dc.nx * dc.ny * dc.nz, dtype=torch.float64, device="cuda")
                bc.get_populations(1, j, g)
                b.init_fields(1, k, W.prolonged(g, tr_c, structs[k][1], dpc), stride=1, from_linear=False)
            bc.close()
    kl, _, info_f, st_f = b.solve(0)
    dl, _, info_d, st_d = b.solve(1)
    torch.cuda.synchronize()
    t_fast = time.perf_counter() - t0
    b.close()

    def rel(x, y):
        return abs(x - y) / abs(y) if y != 0 else abs(x)

    per = []
    for i, (cfg, dom, tr, d) in enumerate(structs):
        p, r = plain[i], ref[i]
        per.append({"nodes": p["nodes"], "porosity": round(cfg.porosity, 3), "mean_d_nm": round(cfg.mean_nm, 1),
                    "plain": {"k": rel(p["k_lattice"], r["k_lattice"]), "D_eff": rel(p["D_lattice"], r["D_lattice"]),
                              "steps": [p["flow_steps"], p["diff_steps"]]},
                    "fast": {"k": rel(kl[i], r["k_lattice"]), "D_eff": rel(dl[i], r["D_lattice"]),
                             "steps": [info_f[i].steps, info_d[i].steps]}})
    resolved = (P.OM_OK, P.OM_ENOPERC)
    ok = (all(p["flow_status"] in resolved and p["diff_status"] == P.OM_OK for p in plain)
          and all(r["flow_status"] in resolved and r["diff_status"] == P.OM_OK for r in ref)
          and all(s in resolved for s in st_f) and all(s == P.OM_OK for s in st_d))
    worst = {form: max(max(x[form]["k"], x[form]["D_eff"]) for x in per) for form in ("plain", "fast")}
    return {"plain_s": t_plain, "fast_s": t_fast, "ratio": t_plain / t_fast,
            "fast_form": f"one batch (FP32 flow, {_prec_name(P, fdp)} diffusion), extrapolated diffusion restarts" +
                         (", two-level (2x coarsened solve) diffusion warm start" if warm == "coarse" else ""),
            "plain_form": "one cold FP32 solve per structure and model",
            "steps": {"plain": {"flow": sum(p["flow_steps"] for p in plain),
                                "diffusion": sum(p["diff_steps"] for p in plain)},
                      "fast": {"flow": sum(i.steps for i in info_f), "diffusion": sum(i.steps for i in info_d),
                               "coarse_diffusion": coarse_steps}},
            "test": f"flow: relative change of the velocity field, diffusion: of the concentration field and the "
                    f"net flux, < {CONV_TOL:g} over {CONV_K} steps (both forms)",
            "reference": "FP64; flow: sum|du_x|/sum|u_x| < 1e-10, diffusion: field and flux < 1e-11, over 1000 steps",
            "reference_s": t_ref,
            "bound": CONV_BOUND, "max_rel_err": worst,
            "within_bound": bool(worst["plain"] <= CONV_BOUND and worst["fast"] <= CONV_BOUND),
            "status_ok": bool(ok), "structures": per,
            "workload": f"{len(structs)} structures 64^3 at 1.5 nm drawn like the 150-structure set "
                        "(porosity U[0.25,0.5], <d> U[10,60] nm, sd <d>/4, tolerance U[0,0.8])"}


def _prec_name(P, prec):
    return {P.OM_F64: "FP64", P.OM_F32: "FP32", P.OM_F16DEV: "FP16", P.OM_BF16DEV: "BF16"}[prec]


def _converge_set(n, seed, edges):
    """Structures drawn like the 150-structure set (porosity, <d>, tolerance,
    1.5 nm voxels), with box edges restricted to `edges`."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        mean = float(rng.uniform(10.0, 60.0))
        sd = 0.25 * mean
        out.append(S.Recon(seed * 1000 + i, (int(rng.choice(edges)),) * 3, 1.5, mean, sd, max(3.0, mean - 3 * sd),
                           mean + 3 * sd, float(rng.uniform(0.25, 0.50)), float(rng.uniform(0.0, 0.8))))
    return out


def run_converge(a):
    """Wall time to converged k and D_eff for a set of structures: plain
    (one FP32 cold solve per structure and model) against the batched path
    with 16-bit diffusion storage and a U-Net warm start (network inference
    included).  Both stop on the same test: relative change below 1e-5 over
    1000 steps, capped at --max-steps.  Structures whose flow has no lattice
    link across the periodic x boundary have k = 0 exactly and take no flow
    steps on either side.  Training data are cold FP32 solves of other
    structures.  Per-structure lines go to stderr."""
    import torch

    from paper_1410_1921_gb300 import build as B
    B.build()
    import paper_1410_1921_gb300 as P
    from paper_1410_1921_gb300 import warmstart as W

    torch.cuda.set_device(0)
    K, tol, cap = 1000, 1e-5, a.max_steps
    fp = P.flow_params(precision=P.OM_F32, conv_tol=tol, check_every=K, max_steps=cap)
    dp = P.diff_params(precision=P.OM_F32, conv_tol=tol, check_every=K, max_steps=cap)
    fields = ("ux", "c") if a.warm == "both" else ("c",)
    learned = a.warm in ("both", "diffusion", "coarse+net")
    refine = a.warm == "coarse+net"
    # the coarse level: FP16 storage and a 10x looser test (the coarse field
    # only has to carry the structure-scale modes)
    dpc = P.diff_params(precision=P.OM_F16DEV, conv_tol=10 * tol, check_every=K, max_steps=cap)
    data, hist, t_data, t_train = [], [None], 0.0, 0.0
    if learned:
        t0 = time.perf_counter()
        data = W.make_dataset(_converge_set(a.n_train, 11, (64,)), fp, dp, fields=fields, coarse=refine,
                              dp_coarse=dpc)
        t_data = time.perf_counter() - t0
        net = P.UNet(3 if refine else 2, len(fields), (16, 32, 64, 128), seed=5)
        t0 = time.perf_counter()
        hist = W.train(net, data, epochs=a.epochs, lr=1e-3, lr_end=5e-5)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
    structs = []
    for cfg in _converge_set(a.n_eval, 23, (64, 96)):
        dom, mask, tr, d = W.structure(cfg)
        if int(tr.sum().item()) > 0:
            structs.append((cfg, dom, mask, tr, d))
    # plain: each structure and model solved on its own, cold, FP32
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [W.solve(dom, tr, d, fp, dp) for _, dom, mask, tr, d in structs]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    # fast: batch (FP32 flow, FP16 diffusion) warm-started from the network
    fp16 = P.diff_params(precision=P.OM_F16DEV, conv_tol=tol, check_every=K, max_steps=cap)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = P.Batch([s[1] for s in structs], [s[3] for s in structs], [s[4] for s in structs], flow=fp, diff=fp16)
    coarse_steps = 0
    if a.warm in ("coarse", "coarse-both", "coarse+net"):
        # the structures coarsened 2x per axis, solved together, their
        # concentration carried to the fine nodes (refined by the network)
        cs = [W.coarse_level(dom, tr, d) for _, dom, mask, tr, d in structs]
        keep = [k for k, c in enumerate(cs) if c[1] is not None]
        bc = None
        if keep:
            fpc = None
            if a.warm == "coarse-both":  # 4x the force: about the fine lattice's velocities (k ~ spacing^2)
                fpc = P.flow_params(precision=P.OM_F32, body_force=4 * fp.body_force, conv_tol=10 * tol,
                                    check_every=K, max_steps=cap)
            bc = P.Batch([cs[k][0] for k in keep], [cs[k][1] for k in keep], [cs[k][2] for k in keep], flow=fpc,
                         diff=dpc)
            _, _, info_c, _ = bc.solve(1)
            coarse_steps = int(sum(i.steps for i in info_c))
            if fpc is not None:
                _, _, _, stc = bc.solve(0)
                for j, k in enumerate(keep):
                    if stc[j] != P.OM_OK:
                        continue
                    dc, tr_c = cs[k][0], cs[k][1]
                    fcd = torch.empty(19 * dc.nx * dc.ny * dc.nz, dtype=torch.float64, device="cuda")
                    bc.get_populations(0, j, fcd)
                    dom = structs[k][1]
                    u = torch.empty(dom.nx * dom.ny * dom.nz, dtype=torch.float32, device="cuda")
                    P.om_prolong2_ux_dev(fcd, tr_c, dom, fpc.body_force, 1.0, u)
                    b.init_fields(0, k, u, stride=1, scale=1.0)
        for k, (_, dom, mask, tr, d) in enumerate(structs):
            if k not in keep:
                if refine:  # no coarse level: the network on a zero coarse departure
                    zero = torch.zeros(dom.nx * dom.ny * dom.nz, dtype=torch.float32, device="cuda")
                    b.init_fields(1, k, W.predict(net, mask, d, dom, zero), stride=1, from_linear=True)
                continue
            dc, tr_c, _ = cs[k]
            g = torch.empty(7 * dc.nx * dc.ny * dc.nz, dtype=torch.float64, device="cuda")
            bc.get_populations(1, keep.index(k), g)
            y = W.predict(net, mask, d, dom, W.prolonged(g, tr_c, dom, dpc, departure=True)) if refine else None
            b.init_fields(1, k, W.prolonged(g, tr_c, dom, dpc, corr=y), stride=1, from_linear=False)
        if bc is not None:
            bc.close()
    elif a.warm != "none":
        nch, ci = len(fields), fields.index("c")
        for k, (_, dom, mask, tr, d) in enumerate(structs):
            y = W.predict(net, mask, d, dom)
            if a.warm == "both":
                b.init_fields(0, k, y[fields.index("ux"):], stride=nch, scale=W.velocity_scale(fp))
            b.init_fields(1, k, y[ci:], stride=nch, from_linear=True)
    torch.cuda.synchronize()
    t_warm = time.perf_counter() - t0
    kl, _, info_f, st_f = b.solve(0)
    torch.cuda.synchronize()
    t_flow = time.perf_counter() - t0 - t_warm
    dl, _, info_d, st_d = b.solve(1)
    torch.cuda.synchronize()
    t_fast = time.perf_counter() - t0
    b.close()
    for i, (cfg, dom, *_r) in enumerate(structs):
        p = plain[i]
        print(f"[{i}] edge {dom.nx} <d> {cfg.mean_nm:.1f} eps {cfg.porosity:.3f} xi {cfg.xi:.2f} "
              f"nodes {p['nodes']}: flow {P.STATUS_NAMES[p['flow_status']]} {p['flow_steps']} -> "
              f"{P.STATUS_NAMES[st_f[i]]} {info_f[i].steps} k {p['k_lattice']:.5e} {kl[i]:.5e}; "
              f"diffusion {P.STATUS_NAMES[p['diff_status']]} {p['diff_steps']} -> {P.STATUS_NAMES[st_d[i]]} "
              f"{info_d[i].steps} D {p['D_lattice']:.5e} {dl[i]:.5e}", file=sys.stderr, flush=True)

    def rel(x, y):
        return abs(x - y) / abs(y) if y != 0 else abs(x)

    resolved = (P.OM_OK, P.OM_ENOPERC)  # ENOPERC: k = 0 exactly, on both sides
    dk = max(rel(kl[i], p["k_lattice"]) for i, p in enumerate(plain))
    dD = max(rel(dl[i], p["D_lattice"]) for i, p in enumerate(plain))
    warm_name = {"coarse": "two-level (2x coarsened solve) warm start", "none": "no warm start",
                 "coarse-both": "two-level warm start of both models",
                 "coarse+net": "two-level warm start refined by the U-Net"}.get(a.warm, "U-Net warm start")
    line = {"metric": f"time to converged k, D_eff: plain / (batched + FP16 diffusion + {warm_name})",
            "value": t_plain / t_fast, "unit": "x", "higher_is_better": True, "n_gpus": 1,
            "plain_s": t_plain, "fast_s": t_fast,
            "fast_split_s": {"batch_and_warm_start": t_warm, "flow": t_flow, "diffusion": t_fast - t_warm - t_flow},
            "structures": len(structs),
            "max_rel_diff_k": dk, "max_rel_diff_D_eff": dD,
            "plain_steps": {"flow": int(sum(p["flow_steps"] for p in plain)),
                            "diffusion": int(sum(p["diff_steps"] for p in plain))},
            "fast_steps": {"flow": int(sum(i.steps for i in info_f)), "diffusion": int(sum(i.steps for i in info_d)),
                           "coarse_diffusion": coarse_steps},
            "zero_flux_structures": int(sum(p["flow_status"] == P.OM_ENOPERC for p in plain)),
            "status_ok": bool(all(s in resolved for s in st_f) and all(s == P.OM_OK for s in st_d)
                              and all(p["flow_status"] in resolved and p["diff_status"] == P.OM_OK
                                      for p in plain)),
            "warm_start": a.warm, "step_cap": cap,
            "training": {"samples": len(data), "epochs": a.epochs, "data_s": t_data, "train_s": t_train,
                         "loss_first": hist[0], "loss_last": hist[-1]},
            "config": {"workload": "structures drawn like the 150-structure set (1.5 nm voxels, porosity "
                                   "U[0.25,0.5], <d> U[10,60] nm, sd <d>/4, tolerance U[0,0.8]), edges {64,96}; "
                                   "test: relative change < 1e-5 over 1000 steps; U-Net 16-32-64-128 trained on "
                                   "64^3 structures of the same law",
                       "data": "synthetic"}}
    print(json.dumps(line))
    return 0


def _device_structure(P, W, cfg):
    dom, mask, tr, d = W.structure(cfg)
    return dom, tr, d


def _window_mlups(step, nodes, steps, reps, nvtx=None):
    """Device MLUPS of `reps` calls of step() (each `steps` LB steps over
    `nodes` nodes), CUDA events around the calls after one warm-up call;
    nvtx names an NVTX range around the timed calls (for a profiler)."""
    import torch
    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if nvtx:
        torch.cuda.nvtx.range_push(nvtx)
    e0.record()
    for _ in range(reps):
        step()
    e1.record()
    torch.cuda.synchronize()
    if nvtx:
        torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    return nodes * steps * reps / (ms * 1e-3) / 1e6, ms / reps


def _parity_us(model, nodes, bytes_per_node, peak, reps=20):
    """Mean CUDA-event time of single even and odd sweeps of `model` (one
    step() call each, outside any captured window) and the fraction of the
    measured HBM bandwidth that the algorithmic bytes make of it."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    if model.time & 1:
        model.step(1)
    model.step(2)
    torch.cuda.synchronize()
    te = to = 0.0
    for _ in range(reps):
        ev[0].record()
        model.step(1)
        ev[1].record()
        model.step(1)
        ev[2].record()
        torch.cuda.synchronize()
        te += ev[0].elapsed_time(ev[1])
        to += ev[1].elapsed_time(ev[2])
    out = {}
    for k, ms in (("even", te / reps), ("odd", to / reps)):
        out[k] = {"us": ms * 1e3, "frac_hbm": nodes * bytes_per_node / (ms * 1e-3) / 1e9 / peak}
    return out


def _batch_split(P, items, nodes):
    """The set split at 2^19 nodes (structures that form groups of their
    own, and the rest): each part as a batch (launch variant tuned, or forced
    to 0, 1, 2 for the flow and 0, 1 for the diffusion) against one solver per
    structure, MLUPS over 100-step windows."""
    out = {}
    for name, sub in (("large", [k for k in range(len(items)) if nodes[k] >= 1 << 19]),
                      ("small", [k for k in range(len(items)) if nodes[k] < 1 << 19])):
        total = sum(nodes[k] for k in sub)
        part = {"structures": len(sub), "nodes": total}
        for model, mname in ((0, "flow"), (1, "diffusion")):
            res = {}
            for var in ((-1, 0, 1, 2) if model == 0 else (-1, 0, 1)):
                fp = P.flow_params(precision=P.OM_F32, check_every=WINDOW, variant=var)
                dp = P.diff_params(precision=P.OM_F32, check_every=WINDOW, variant=var)
                b = P.Batch([items[k][0] for k in sub], [items[k][1] for k in sub], [items[k][2] for k in sub],
                            flow=fp if model == 0 else None, diff=dp if model == 1 else None)
                res["tuned" if var < 0 else f"variant_{var}"] = _window_mlups(lambda: b.step(model, WINDOW), total,
                                                                              WINDOW, 3)[0]
                b.close()
            solvers = []
            for k in sub:
                dom, tr, d = items[k]
                ns = P.NodeSet(tr, dom)
                solvers.append((ns, P.Flow(ns, P.flow_params(precision=P.OM_F32, check_every=WINDOW)) if model == 0
                                else P.Diffusion(ns, d, P.diff_params(precision=P.OM_F32, check_every=WINDOW))))

            def step_all():
                for _, sv in solvers:
                    sv.step(WINDOW)

            res["plain"] = _window_mlups(step_all, total, WINDOW, 3)[0]
            for ns, sv in solvers:
                sv.close()
                ns.close()
            part[mname] = res
        out[name] = part
    return out


def run_layout(a):
    """The two population layouts of the host-level solves on structures of
    rising porosity: the sweep workload's generator at 128^3 (porosity 0.35,
    0.45) and body-centred cubic sphere arrays at 128^3 (0.5, 0.7, 0.9).
    Per structure and model the fluid MLUPS of 2000 steps (20 windows with
    their checks, no convergence) in the sparse and the dense layout (FP32),
    and the layout OM_LAYOUT_AUTO picks."""
    from paper_1410_1921_gb300 import build as B
    B.build()
    import paper_1410_1921_gb300 as P
    from paper_1410_1921_gb300 import warmstart as W

    cases = []
    for eps in (0.35, 0.45):
        dom, mask, tr, d = W.structure(S.sweep_structure(eps, seed=1, edge=128))
        cases.append((f"sweep generator, porosity {eps}", dom, mask.cpu().numpy().reshape(128, 128, 128),
                      d.cpu().numpy().reshape(128, 128, 128)))
    for eps in (0.5, 0.7, 0.9):
        m, _ = S.bcc_array(128, eps)
        dom = P.domain(m.shape, 1.0)
        d, _ = P.om_local_pore_diameter(m, dom, P.OM_PORE_CHORD13)
        cases.append((f"bcc sphere array, porosity {eps}", dom, m, d))
    rows = []
    for name, dom, mask, d in cases:
        row = {"structure": name, "pore_fraction": float(mask.mean())}
        for model in ("flow", "diffusion"):
            for lay, lname in ((P.OM_LAYOUT_SPARSE, "sparse"), (P.OM_LAYOUT_DENSE, "dense")):
                if model == "flow":
                    info = P.om_solve_permeability(mask, dom, P.flow_params(conv_tol=0.0, max_steps=2000,
                                                                            layout=lay))[3]
                else:
                    info = P.om_solve_knudsen(mask, d, dom, P.diff_params(conv_tol=0.0, max_steps=2000,
                                                                          layout=lay))[3]
                row[f"{model}_{lname}_mlups"] = info.mlups
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "fluid MLUPS by population layout", "unit": "MLUPS", "n_gpus": 1, "dtype": "f32",
                      "data": "synthetic", "structures": rows,
                      "config": {"workload": "128^3 structures, porosity 0.35-0.9; 2000 steps in 100-step windows"}}))
    return 0


def run_unet(a):
    """The warm start's U-Net alone: forward and training step (forward, backward,
    Adam) of a B x E^3 batch with 2 input and 1 output channel, random inputs,
    CUDA events around 20 forwards and 10 steps after 3 warm-up passes.  The
    convolution FLOPs of a forward are 2 x voxels x 27 x K x N per layer, K
    counted as stored (the first layer's 2 input channels are padded to 16)."""
    import torch

    from paper_1410_1921_gb300 import build as B
    B.build()
    import paper_1410_1921_gb300 as P

    nb, edge, chs = a.unet_shape.split(",")
    nb, edge = int(nb), int(edge)
    ch = tuple(int(c) for c in chs.split("-"))
    torch.cuda.set_device(0)
    net = P.UNet(2, 1, ch, seed=3)
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.rand(nb, edge, edge, edge, 2, device="cuda", generator=g)
    t = torch.rand(nb, edge, edge, edge, 1, device="cuda", generator=g)
    y = torch.empty(nb, edge, edge, edge, 1, device="cuda")
    m = torch.ones(nb, edge, edge, edge, dtype=torch.uint8, device="cuda")
    flops = 0
    for lv in range(len(ch)):
        v = nb * (edge >> lv) ** 3
        cin = 16 if lv == 0 else ch[lv - 1]
        flops += 2 * v * 27 * (cin * ch[lv] + ch[lv] * ch[lv])
        if lv + 1 < len(ch):
            flops += 2 * v * 27 * ((ch[lv + 1] + ch[lv]) * ch[lv] + ch[lv] * ch[lv])
    for _ in range(3):
        net.forward(x, y)
        net.train_step(x, t, m, 1e-4)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        net.forward(x, y)
    e1.record()
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1) / 20
    e0.record()
    for _ in range(10):
        net.train_step(x, t, m, 1e-4)
    e1.record()
    torch.cuda.synchronize()
    step = e0.elapsed_time(e1) / 10
    print(json.dumps({"metric": "U-Net training step", "value": round(step, 3), "unit": "ms", "higher_is_better": False,
                      "n_gpus": 1, "dtype": "bf16", "data": "synthetic", "forward_ms": round(fwd, 3),
                      "forward_conv_gflop": round(flops / 1e9, 2),
                      "forward_conv_tflops": round(flops / fwd / 1e9, 1),
                      "config": {"workload": f"U-Net {a.unet_shape.split(',')[2]}, {nb} x {edge}^3, 2 -> 1 channels",
                                 "l2": "activations larger than L2"}}))
    return 0


def run_batch(a):
    """The 150-structure set (edges {64..200}^3, porosity U[0.10, 0.50], <d>
    U[10, 60] nm, tolerance U[0, 0.8], 1.5 nm voxels) advanced together: one
    launch per LB step and L2-sized group over a work list of tiles, check
    windows replayed as CUDA graphs, launch shape autotuned.  Aggregate MLUPS
    of each model over 100-step windows (FP32), and the plain form for
    comparison: the same structures one solver each, the same windows.
    Also the two window modes of a batch solve (graph of per-step launches,
    one persistent grid-barrier launch per group), each over 4 windows with
    their convergence checks."""
    import torch

    from paper_1410_1921_gb300 import build as B
    B.build()
    import paper_1410_1921_gb300 as P
    from paper_1410_1921_gb300 import warmstart as W

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    items = []
    cfgs = S.batch_structures(a.n_struct) if a.batch_set == "150" else _converge_set(20, 23, (64,))
    for cfg in cfgs:
        dom, tr, d = _device_structure(P, W, cfg)
        if int(tr.sum().item()) > 0:
            items.append((dom, tr, d))
    t_setup = time.perf_counter() - t0
    fp = P.flow_params(precision=P.OM_F32, check_every=WINDOW)
    dp = P.diff_params(precision=P.OM_F32, check_every=WINDOW)
    t0 = time.perf_counter()
    b = P.Batch([i[0] for i in items], [i[1] for i in items], [i[2] for i in items], flow=fp, diff=dp)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    nodes = [int(i[1].sum().item()) for i in items]
    total = sum(nodes)
    out = {}
    for model, name in ((0, "flow"), (1, "diffusion")):
        mlups, ms = _window_mlups(lambda: b.step(model, WINDOW), total, WINDOW, 3, nvtx="timed")
        out[name] = {"mlups": mlups, "ms_per_window": ms}
    b.close()
    modes = {}
    for mode, mname in ((0, "graph"), (1, "persistent")):
        fp0 = P.flow_params(precision=P.OM_F32, conv_tol=0.0, check_every=WINDOW, max_steps=4 * WINDOW)
        dp0 = P.diff_params(precision=P.OM_F32, conv_tol=0.0, check_every=WINDOW, max_steps=4 * WINDOW)
        bm = P.Batch([i[0] for i in items], [i[1] for i in items], [i[2] for i in items], flow=fp0, diff=dp0)
        modes[mname] = {}
        for model, name in ((0, "flow"), (1, "diffusion")):
            bm.set_window_mode(model, mode)
            res, _, info, st = bm.solve(model)
            moved = sum(nodes[k] * info[k].steps for k in range(len(nodes)) if st[k] != P.OM_ENOPERC)
            modes[mname][name] = {"mlups": moved / info[0].seconds / 1e6, "s": info[0].seconds}
        bm.close()
    # plain: one solver per structure, the same windows one after the other
    plain = {}
    for name in ("flow", "diffusion"):
        solvers = []
        for dom, tr, d in items:
            ns = P.NodeSet(tr, dom)
            sv = P.Flow(ns, fp) if name == "flow" else P.Diffusion(ns, d, dp)
            solvers.append((ns, sv))

        def step_all():
            for _, sv in solvers:
                sv.step(WINDOW)

        mlups, ms = _window_mlups(step_all, total, WINDOW, 3)
        plain[name] = {"mlups": mlups, "ms_per_window": ms}
        for ns, sv in solvers:
            sv.close()
            ns.close()
    split = _batch_split(P, items, nodes) if a.batch_split else None
    line = {"metric": "aggregate fluid MLUPS, batched structures", "value": out["flow"]["mlups"],
            "unit": "MLUPS", "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "batched": out, "plain": plain, "window_modes": modes, "structures": len(items), "nodes": total,
            "setup_s": t_setup, "batch_create_s": t_create, **({"split": split} if split else {}),
            "config": {"workload": ("150 structures, edges {64,96,128,160,200}^3 at 1.5 nm, porosity U[0.10,0.50]"
                                    if a.batch_set == "150" else
                                    "20 structures of 64^3 at 1.5 nm, porosity U[0.25,0.50]") +
                                   ", <d> U[10,60] nm (sd <d>/4), tolerance U[0,0.8]; 100-step windows",
                       "l2": "no flush: the set's populations exceed L2; a group's stay in L2 across its window"}}
    print(json.dumps(line))
    return 0


def run_precision(a):
    """A 512^3 structure (porosity 0.30, <d> 40 nm, sd 10, tolerance 0.5, 1 nm
    voxels): device MLUPS of both sweeps with FP32, FP16 and BF16 population
    storage over 100-step windows, and the time of single even and odd sweeps
    against the HBM roofline of their algorithmic bytes (the errors of each
    format against FP64 are the subject of tests/test_gpu_precision.py)."""
    import torch

    from paper_1410_1921_gb300 import build as B
    B.build()
    import paper_1410_1921_gb300 as P
    from paper_1410_1921_gb300 import warmstart as W

    torch.cuda.set_device(0)
    dom, tr, d = _device_structure(P, W, S.large_structure())
    ns = P.NodeSet(tr, dom)
    out = {}
    peak, _ = _peak_hbm()
    for name, prec in (("f32", P.OM_F32), ("f16", P.OM_F16DEV), ("bf16", P.OM_BF16DEV)):
        bf, bd = (BYTES_FLOW_F32, BYTES_DIFF_F32) if prec == P.OM_F32 else (BYTES_FLOW_F32 // 2, 32)
        fl = P.Flow(ns, P.flow_params(precision=prec, check_every=WINDOW))
        fm, fms = _window_mlups(lambda: fl.step(WINDOW), ns.n_nodes, WINDOW, 3)
        fpar = _parity_us(fl, ns.n_nodes, bf, peak)
        fl.close()
        df = P.Diffusion(ns, d, P.diff_params(precision=prec, check_every=WINDOW))
        dm, dms = _window_mlups(lambda: df.step(WINDOW), ns.n_nodes, WINDOW, 3)
        dpar = _parity_us(df, ns.n_nodes, bd, peak)
        df.close()
        out[name] = {"flow_mlups": fm, "diffusion_mlups": dm, "flow_sweeps": fpar, "diffusion_sweeps": dpar}
        if prec == P.OM_F32:  # the paper's diffusion lattice, for comparison (not a bench line)
            d19 = P.Diffusion(ns, d, P.diff_params(precision=prec, check_every=WINDOW, lattice=19))
            m19, _ = _window_mlups(lambda: d19.step(WINDOW), ns.n_nodes, WINDOW, 3)
            out[name]["diffusion_d3q19_mlups"] = m19
            out[name]["diffusion_d3q19_sweeps"] = _parity_us(d19, ns.n_nodes, 19 * 4 * 2 + 4, peak)
            d19.close()
    line = {"metric": "fluid MLUPS by population storage, 512^3", "value": out["f16"]["flow_mlups"], "unit": "MLUPS",
            "higher_is_better": True, "n_gpus": 1, "data": "synthetic", "nodes": ns.n_nodes, "by_storage": out,
            "gain_over_f32": {k: {"flow": v["flow_mlups"] / out["f32"]["flow_mlups"],
                                  "diffusion": v["diffusion_mlups"] / out["f32"]["diffusion_mlups"]}
                              for k, v in out.items()},
            "config": {"workload": "512^3 at 1 nm, porosity 0.30, <d> 40 nm (sd 10), tolerance 0.5; 100-step windows"}}
    ns.close()
    print(json.dumps(line))
    return 0


def _diff_solve(P, dom, tr, d, dp, init=None, from_linear=True):
    """One diffusion solve on the transport set, optionally warm-started from
    a device field; (status, D_lattice, steps, seconds)."""
    import torch
    ns = P.NodeSet(tr, dom)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    df = P.Diffusion(ns, d, dp)
    if init is not None:
        df.init_concentration(init, stride=1, from_linear=from_linear)
    st, D, info = df.solve()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    df.close()
    ns.close()
    return st, D, info.steps, sec


def run_warmstart(a):
    """The learned warm start at the scale of its configuration: a 3-D U-Net
    (4 levels, 16-32-64-128) trained on `--n-train` LB-solved 96^3
    structures from the 256^3 sweep's generator (1 nm voxels, <d> 30 nm, sd
    8, tolerance 0.3, porosity U[0.15, 0.45]; structures without transport
    pores are redrawn), targets u_x and C from batched solves; then held-out
    128^3 and 256^3 structures solved cold, warm-started by the network and
    warm-started by a 2x-coarsened diffusion solve, every form with the same
    solver and test (FP32, extrapolated restarts, relative change < 1e-6 over
    1000 steps).  Per structure: diffusion steps and wall time of each form
    (the network's inference and the coarse solve included in theirs), and
    the D_eff of each against the cold one; at 128^3 against an FP64 solve
    converged to 1e-11 too.  The flow is not warm-started (a predicted
    velocity field excites slow pressure modes): its cold solve is reported
    once per structure."""
    import torch

    from paper_1410_1921_gb300 import build as B
    B.build()
    import paper_1410_1921_gb300 as P
    from paper_1410_1921_gb300 import warmstart as W

    torch.cuda.set_device(0)
    log = lambda m: print(m, file=sys.stderr, flush=True)
    rng = np.random.default_rng(5)
    fp = P.flow_params(precision=P.OM_F32, conv_tol=1e-6, check_every=1000, max_steps=3_000_000)
    dp = P.diff_params(precision=P.OM_F32, conv_tol=1e-6, check_every=1000, max_steps=6_000_000,
                       accel=P.OM_ACCEL_EXTRAPOLATE)
    # training set: draw until n_train structures are solved
    t0 = time.perf_counter()
    data, tried, seed = [], 0, 500_000
    while len(data) < a.n_train and tried < 4 * a.n_train:
        want = a.n_train - len(data)
        cfgs = []
        for _ in range(min(64, int(want * 1.4) + 4)):
            cfgs.append(S.sweep_structure(float(rng.uniform(0.15, 0.45)), seed=seed, edge=a.train_edge))
            seed += 1
        got, n = W.make_dataset_batched(cfgs, fp, dp, fields=("ux", "c"))
        data += got[:want]
        tried += n
        log(f"training set: {len(data)} solved of {tried} drawn, {time.perf_counter() - t0:.0f} s")
    t_data = time.perf_counter() - t0
    net = P.UNet(2, 2, (16, 32, 64, 128), seed=3)
    t0 = time.perf_counter()
    hist = W.train(net, data, epochs=a.epochs, lr=1e-3, lr_end=1e-4, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    n_train = len(data)
    del data
    torch.cuda.empty_cache()
    # held-out structures
    rows = []
    dp64 = P.diff_params(precision=P.OM_F64, conv_tol=1e-11, check_every=1000, max_steps=20_000_000,
                         accel=P.OM_ACCEL_EXTRAPOLATE)
    edges = [int(e) for e in a.eval_edges.split(",")]
    evals = [(e, p, 700_000 + 1000 * e + i) for e in edges
             for i, p in enumerate((0.25, 0.35, 0.45) if e <= 128 else (0.30, 0.40))]
    for edge, eps, sd in evals:
        dom, mask, tr, d = W.structure(S.sweep_structure(eps, seed=sd, edge=edge))
        if int(tr.sum().item()) == 0:
            continue
        row = {"edge": edge, "porosity_target": eps, "nodes": int(tr.sum().item())}
        ns = P.NodeSet(tr, dom)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        fl = P.Flow(ns, fp)
        st, kl, info = fl.solve()
        torch.cuda.synchronize()
        row["flow"] = {"status": int(st), "k_lattice": kl, "steps": info.steps, "s": time.perf_counter() - t1}
        fl.close()
        ns.close()
        st, Dc, sc, tc = _diff_solve(P, dom, tr, d, dp)
        row["cold"] = {"status": int(st), "D_lattice": Dc, "steps": sc, "s": tc}
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        pred = W.predict(net, mask, d, dom)
        c = pred.view(-1, 2)[:, 1].contiguous()
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t1
        st, Dl, sl, tl = _diff_solve(P, dom, tr, d, dp, init=c)
        row["learned"] = {"status": int(st), "D_lattice": Dl, "steps": sl, "s": tl + t_inf, "inference_s": t_inf,
                          "rel_diff_D": abs(Dl - Dc) / abs(Dc)}
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        dep = W.coarse_departure(dom, tr, d, dp)
        torch.cuda.synchronize()
        t_c = time.perf_counter() - t1
        st, D2, s2, t2 = _diff_solve(P, dom, tr, d, dp, init=dep)
        row["two_level"] = {"status": int(st), "D_lattice": D2, "steps": s2, "s": t2 + t_c, "coarse_s": t_c,
                            "rel_diff_D": abs(D2 - Dc) / abs(Dc)}
        if edge <= 128:
            st, D64, s64, t64 = _diff_solve(P, dom, tr, d, dp64)
            row["fp64_reference"] = {"status": int(st), "D_lattice": D64, "steps": s64}
            for k in ("cold", "learned", "two_level"):
                row[k]["rel_err_D_vs_fp64"] = abs(row[k]["D_lattice"] - D64) / abs(D64)
        rows.append(row)
        log(json.dumps(row))
    sums = {k: {"steps": sum(r[k]["steps"] for r in rows), "s": sum(r[k]["s"] for r in rows)}
            for k in ("cold", "learned", "two_level")}
    line = {"metric": "diffusion steps and wall time to the 1e-6 test, learned warm start vs cold start",
            "value": sums["cold"]["s"] / sums["learned"]["s"] if sums["learned"]["s"] > 0 else None,
            "unit": "x (cold wall time / learned wall time)", "higher_is_better": True, "n_gpus": 1,
            "data": "synthetic", "dtype": "f32",
            "training": {"structures": n_train, "edge": a.train_edge, "epochs": a.epochs,
                         "loss_first": hist[0], "loss_last": hist[-1], "data_s": t_data, "train_s": t_train},
            "totals": sums, "structures": rows,
            "config": {"workload": f"U-Net 16-32-64-128 trained on {n_train} LB-solved {a.train_edge}^3 structures "
                                   "(1 nm, <d> 30 nm sd 8, tolerance 0.3, porosity U[0.15,0.45]); held out "
                                   "128^3 (porosity 0.25/0.35/0.45) and 256^3 (0.30/0.40)",
                       "test": "relative change of the concentration field and the net flux < 1e-6 over 1000 "
                               "steps, extrapolated restarts, FP32, in every form"}}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    args = _args()
    if args.mode == "warmstart":
        sys.exit(run_warmstart(args))
    if args.mode == "layout":
        sys.exit(run_layout(args))
    if args.mode == "unet":
        sys.exit(run_unet(args))
    if args.mode == "batch":
        sys.exit(run_batch(args))
    if args.mode == "precision":
        sys.exit(run_precision(args))
    if args.mode == "converge":
        sys.exit(run_converge(args))
    sys.exit(run_reference(args) if args.impl == "reference" else run_gpu(args))
