#!/usr/bin/env python
"""Benchmark of the P-hat-preconditioned CG solve of the space-time least-squares system.

One step = one solve as timed in the paper's Table 1: preconditioner setup
(generalized eigendecompositions and the banded factors of every H_i,
stst_build_fd) plus PCG from the zero initial guess to relative residual tol
(stst_pcg_solve), on the 2D+t workload with p=3, 64^2 x 64 elements, the
harmonic potential scaled to [0,10] and a windowed Gaussian wavepacket as
initial datum (278,850 complex unknowns). Inputs are resident in HBM when
the timed region starts; the L2 cache is flushed before every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config c2] [--prec fp64|fp32|bf16]

--config c4 times the batched workload (128 problems, one graph launch per step); --config c5
trains the learned warm start on method-generated solutions, then times solves of new problems
from the network's iterate against cold-start PCG.

One JSON line on rank 0. It also carries: the accurate solve (the same step
to relative residual 1e-10) and both solutions' errors against the FP64
oracle's solution of the same system; the FP64 and BF16x3 preconditioners and
the 3D+t workloads c3p2 / c3p4 timed the same way (`variants`); the oracle
timed on the host cores (`cpu_baseline`: medians of full solves, all cores
and one thread, with the CPU model). With --impl reference the oracle is the
timed arm: one step is one full oracle solve of the workload (no
extrapolation; 3D+t workloads use the stated half-size mesh).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG solve time to rel. residual 1e-8 and apply_prec DOF/s; fraction of roofline"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
N_SM = 152
FP64_FMA_PER_CLK_SM = 2      # 1.25 TFLOP/s nominal FP64 at 2.07 GHz over 152 SMs
FP32_FMA_PER_CLK_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--prec", default="fp32", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--solver", default="pcg", choices=["pcg", "ir"])
    ap.add_argument("--prec-op", default="phat", choices=["phat", "potential"],
                    help="preconditioner operator: the paper's P-hat, or P_V built from the potential's "
                         "one-direction operators (sums of one-direction factors only)")
    ap.add_argument("--autotune", type=int, default=1,
                    help="mode-product tiles: 1 measured per shape, 0 default, 10 rpt + cpt forced (stst_set_autotune)")
    ap.add_argument("--tw-p", type=int, default=3, help="degree of the travelling-wave workload (--config tw)")
    ap.add_argument("--tw-nel", type=int, default=64, help="elements per direction of --config tw")
    ap.add_argument("--fused-transforms", type=int, default=0,
                    help="d = 2, FP32 preconditioner: 0 chosen per shape, 1 separate mode products, 2 fused, "
                         "11..14 fused with 1..4 CTAs per time index (stst_set_fused_transforms)")
    ap.add_argument("--time-solver", type=int, default=0,
                    help="0 chosen per shape, 1 sequential, 2 segmented (stst_set_time_solver)")
    ap.add_argument("--pencil", type=int, default=0,
                    help="FP32 preconditioner, last direction and time solves in one kernel: 0 chosen per shape, "
                         "1 off, 2 one CTA per pencil, 3 a cluster of two (stst_set_pencil)")
    ap.add_argument("--fused-matvec", type=int, default=0,
                    help="FP64 mat-vec levels in one launch with grid barriers: 0 one launch per level (default), "
                         "1 one launch for all levels (stst_set_fused_matvec)")
    ap.add_argument("--tensor-products", type=int, default=0,
                    help="FP32 preconditioner, TF32 tensor-core mode products: 0 an autotuner candidate, 1 off, "
                         "2 wherever they apply (stst_set_tensor_products)")
    ap.add_argument("--cpu-baseline", default="on", choices=["on", "off"],
                    help="time the oracle on the host cores (off: skip it, e.g. for the 3D workloads)")
    ap.add_argument("--variants", default="on", choices=["on", "off"],
                    help="c2 only: also time the FP64 and BF16x3 preconditioners, the accurate solve (tolerance "
                         "1e-10) and the 3D+t workloads c3p2 / c3p4, as extra keys of the one JSON line")
    ap.add_argument("--formulation", default="ls", choices=["ls", "uw"],
                    help="least squares (Sec. 4.3) or ultraweak (Sec. 4.4)")
    ap.add_argument("--inner-tol", type=float, default=1e-4)
    ap.add_argument("--batch", type=int, default=128, help="number of problems of the c4 workload")
    ap.add_argument("--train", type=int, default=10000, help="training solves of the c5 workload")
    ap.add_argument("--stages", type=int, default=3, help="network stages of the c5 warm start")
    ap.add_argument("--train-steps", type=int, default=6000, help="Adam steps per stage (c5)")
    ap.add_argument("--basis", type=int, default=1024, help="basis size K of the c5 warm start")
    ap.add_argument("--hidden", default="", help="c5: comma-separated widths of tanh hidden layers (empty: linear "
                                                 "stages)")
    return ap.parse_args()


def max_over_ranks(value, dist=None, device="cpu"):
    """Largest value over the ranks (the slowest replica sets the step time); the value itself when
    running alone. Replicas exchange nothing else: every rank solves its own copy of the workload."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_hash(span):
    """Hash of a kernel's own source text (from `begin` up to `end` in `file`): traffic figures taken
    with ncu are void once the kernel they describe has changed."""
    path = os.path.join(ROOT, "paper_2311_18461_gb300", "csrc", span["file"])
    text = open(path).read()
    i = text.index(span["begin"])
    j = text.index(span["end"], i)
    return hashlib.sha256(text[i:j].encode()).hexdigest()[:16]


def traffic_for(kernel, shape):
    """DRAM bytes per launch from the committed ncu summary, if taken on the kernel's current source and
    on this workload's shape (`shape`: the number of unknowns and the plan's band applications per one)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get("kernels", {}).get(kernel)
        if not rec or rec.get("source_hash") != source_hash(rec["span"]):
            return None
        if rec.get("shape") != shape:
            return None
        return rec.get("dram_bytes_per_launch")
    except Exception:
        return None


# Table 1 of the paper (P-hat-CG on the travelling wave, 1e-8 from x0 = 0, one CPU thread at 1 GHz):
# (p, n_el) -> (iterations, seconds including the preconditioner setup)
TABLE1 = {(2, 8): (7, 0.0426), (2, 16): (7, 0.0659), (2, 32): (7, 0.2992), (2, 64): (7, 2.7304),
          (3, 8): (8, 0.0302), (3, 16): (9, 0.0982), (3, 32): (8, 0.4703), (3, 64): (8, 4.7142),
          (4, 8): (10, 0.0427), (4, 16): (10, 0.2289), (4, 32): (10, 1.2329), (4, 64): (10, 9.0219)}
TW = {"p": 3, "n_el": 64}  # set from --tw-p / --tw-nel


def workload(cfg_name):
    from inputs import CONFIGS, potential, initial_factors
    cfg = dict(CONFIGS[cfg_name])
    if cfg_name == "tw":
        cfg["p"] = TW["p"]
        cfg["n_el"] = [TW["n_el"]] * 3
    return cfg, potential(cfg), initial_factors(cfg)


def tw_rhs(prob):
    """Right-hand side of the travelling wave: its forcing and its Dirichlet and initial values (from u
    on the whole space-time grid) through stst_rhs_lift; the grids are built on the device."""
    import torch
    from inputs import travelling_wave
    u_fn, f_fn = travelling_wave(xp=torch)
    g = [prob.quad_points(l) for l in range(3)]
    t, x1, x2 = g[0].view(1, 1, -1), g[1].view(1, -1, 1), g[2].view(-1, 1, 1)
    u_qp = u_fn(t, x1, x2).to(torch.complex128).contiguous().view(-1)
    f_qp = f_fn(t, x1, x2).to(torch.complex128).contiguous().view(-1)
    b = prob.rhs_lift(f_qp, u_qp)
    torch.cuda.synchronize()
    del u_qp, f_qp
    return b


def sample_1d(prob, fn, l):
    import numpy as np
    x = prob.quad_points(l).cpu().numpy()
    return np.asarray(fn(x)) * np.ones_like(x)


def build_problem(cfg, V, u0, prec, stream, formulation="ls", prec_op="phat"):
    import numpy as np
    import torch
    import paper_2311_18461_gb300 as S
    d = cfg["d"]
    prob = S.Problem(d, cfg["n_el"], [cfg["p"]] * (d + 1), T=cfg["T"], nu=cfg["nu"],
                     prec_mode={"fp64": S.STST_PREC_FP64, "fp32": S.STST_PREC_FP32, "bf16": S.STST_PREC_BF16}[prec],
                     stream=stream, formulation={"ls": S.STST_FORM_LS, "uw": S.STST_FORM_UW}[formulation])
    if V:
        cols = [sample_1d(prob, term[l - 1], l) for term in V for l in range(1, d + 1)]
        prob.set_potential(torch.tensor(np.concatenate(cols), dtype=torch.float64, device="cuda"), len(V))
    if prec_op == "potential":
        S.stst_set_prec_operator(prob.h, 1)
    if u0 is None:  # the travelling wave
        return prob, tw_rhs(prob)
    grids = [prob.quad_points(l).cpu().numpy() for l in range(1, d + 1)]
    U = np.ones([1] * d, dtype=complex)
    for l, g in enumerate(u0):
        shp = [1] * d
        shp[d - 1 - l] = len(grids[l])
        U = U * np.asarray(g(grids[l])).reshape(shp)
    u0_qp = torch.tensor(np.ascontiguousarray(U).ravel(), dtype=torch.complex128, device="cuda")
    b = prob.rhs(None, u0_qp)
    torch.cuda.synchronize()
    return prob, b


def workload_name(name, cfg, tol):
    d = cfg["d"]
    space = "x".join(str(v) for v in cfg["n_el"][1:])
    pot = {None: "V=0", "harmonic": "harmonic V in [0,10]", "bump": "Gaussian bump V"}[cfg["potential"]]
    u0 = {"sine": "sin(pi x) initial datum", "travelling_wave":
          "travelling wave of Sec. 6.2 with its forcing, Dirichlet and initial values"}.get(cfg["u0"],
                                                                                         "windowed Gaussian wavepacket u0")
    return (f"{name}: {d}D+t p={cfg['p']} {space} x {cfg['n_el'][0]} elements, {pot}, {u0}, complex128, "
            f"tol {tol:g}")


def run_batch(args):
    """Batched workload: 128 heterogeneous 2D+t problems solved by one graph launch per step."""
    import numpy as np
    import torch
    import paper_2311_18461_gb300 as S
    from inputs import c4_instances

    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:  # replicas: every rank solves the whole batch; only the step time is reduced
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n_inst = args.batch
    specs = c4_instances(n_inst)
    prec = {"fp64": S.STST_PREC_FP64, "fp32": S.STST_PREC_FP32, "bf16": S.STST_PREC_BF16}[args.prec]
    probs, rhs, xs = [], [], []
    for sp in specs:
        prob = S.Problem(2, sp["n_el"], [sp["p"]] * 3, prec_mode=prec)
        cols = [sample_1d(prob, term[l - 1], l) for term in sp["potential_terms"] for l in (1, 2)]
        prob.set_potential(torch.tensor(np.concatenate(cols), dtype=torch.float64, device="cuda"),
                           len(sp["potential_terms"]))
        g1, g2 = (prob.quad_points(l).cpu().numpy() for l in (1, 2))
        U = np.asarray(sp["u0_factors"][1](g2)).reshape(-1, 1) * np.asarray(sp["u0_factors"][0](g1)).reshape(1, -1)
        b = prob.rhs(None, torch.tensor(np.ascontiguousarray(U).ravel(), dtype=torch.complex128, device="cuda"))
        probs.append(prob)
        rhs.append(b)
        xs.append(prob.vec())
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    batch = S.stst_batch_create([p.h for p in probs], rhs, xs, stream)
    tol = 1e-8
    n_dof = sum(p.n_dof for p in probs)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def step():
        with torch.cuda.stream(stream):  # ordered before the batch graph on the same stream
            for x in xs:
                x.zero_()
        return S.stst_batch_solve(batch, n_inst, tol, 200)

    for _ in range(max(args.warmup, 3)):
        status, iters, relres, sts = step()
    assert status == 0, f"batch failed: {sts}"
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    times = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        status, iters, relres, sts = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    # end to end: right-hand sides from pinned host memory in, solutions out, every step
    b_host = [b.cpu().pin_memory() for b in rhs]
    x_host = [torch.empty_like(h).pin_memory() for h in b_host]
    e2e = []
    for k in range(args.steps + 1):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            for bd, bh in zip(rhs, b_host):
                bd.copy_(bh, non_blocking=True)
        step()
        with torch.cuda.stream(stream):
            for xd, xh in zip(xs, x_host):
                xh.copy_(xd, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if k > 0:
            e2e.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = max_over_ranks(statistics.mean(times), dist, "cuda")
    out = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f64+f32", "bf16": "f64+f32+bf16"}[args.prec],
        "data": "synthetic",
        "config": {"workload": f"c4: {n_inst} 2D+t problems, n_el in {{16..96}}^2 x {{16..96}}, p in {{2,3,4}}, "
                               f"random separable potentials (rank <= 3), wavepackets, seeds 4+i, tol {tol:g}",
                   "n_dof_total": n_dof, "step": "one graph launch: setup + PCG of every problem",
                   "pcg_iterations": {"min": min(iters), "median": statistics.median(iters), "max": max(iters)},
                   "l2": "flushed (512 MB write) before each step", "parallelism": f"replicas x{world}"},
        "dofs_per_s": n_dof / (ms / 1e3),
        "clocks": clocks,
        "e2e": {"value": statistics.mean(e2e) / 1e3, "unit": "s", "h2d_bytes_per_step": 16 * n_dof,
                "d2h_bytes_per_step": 16 * n_dof},
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    S.stst_batch_destroy(batch)
    for p in probs:
        p.close()
    if dist:
        dist.destroy_process_group()


def run_warmstart(args):
    """Learned warm start (c5): train on method-generated solutions, then time solves of new problems
    from the network's iterate (guarded PCG) against cold-start PCG on the same problems."""
    import numpy as np
    import torch
    import paper_2311_18461_gb300 as S
    from paper_2311_18461_gb300.warmstart import WarmStart
    from inputs import CONFIGS, potential, wavepacket_factors, wavepacket_params

    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    cfg = CONFIGS["c5"]
    tol = cfg["tol"]
    prec = {"fp64": S.STST_PREC_FP64, "fp32": S.STST_PREC_FP32, "bf16": S.STST_PREC_BF16}[args.prec]
    prob = S.Problem(2, cfg["n_el"], [cfg["p"]] * 3, T=cfg["T"], nu=cfg["nu"], prec_mode=prec)
    V = potential(cfg)
    cols = [sample_1d(prob, term[l - 1], l) for term in V for l in (1, 2)]
    prob.set_potential(torch.tensor(np.concatenate(cols), dtype=torch.float64, device="cuda"), len(V))
    prob.build_fd()
    g1, g2 = (prob.quad_points(l).cpu().numpy() for l in (1, 2))

    def u0_qp(par):
        f = wavepacket_factors(par)
        U = np.asarray(f[1](g2)).reshape(-1, 1) * np.asarray(f[0](g1)).reshape(1, -1)
        return torch.tensor(np.ascontiguousarray(U).ravel(), dtype=torch.complex128, device="cuda")

    seed = cfg["u0"][1]
    rng = np.random.default_rng(seed)
    train = [wavepacket_params(rng, 2) for _ in range(args.train)]
    K = args.basis
    hidden = tuple(int(v) for v in args.hidden.split(",") if v.strip())
    ws = WarmStart(prob, K, K, hidden=hidden, stages=args.stages, max_batch=256, seed=seed)
    t0 = time.time()
    its_train = ws.collect([lambda par=par: u0_qp(par) for par in train], tol=tol)
    torch.cuda.synchronize()
    t1 = time.time()
    ws.fit(power_its=1, seed=seed + 1)
    torch.cuda.synchronize()
    t2 = time.time()
    ws.train(args.train_steps, batch=256, lr0=3e-3, lr1=3e-6, seed=seed + 2)
    t3 = time.time()
    # new problems (a different seed), inputs resident in HBM
    trng = np.random.default_rng(seed + 1000)
    n_test = max(args.steps, 1) + max(args.warmup, 3)
    tests = []
    for _ in range(n_test):
        f, c0 = prob.rhs(u0_qp=u0_qp(wavepacket_params(trng, 2)), want_c0=True)
        tests.append((f, c0))
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn):
        flush.fill_(1)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record()
        r = fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b), r

    warm_ms, cold_ms, it_w, it_c, e0s, diffs, used = [], [], [], [], [], [], []
    sampler = ClockSampler(local)
    for i, (f, c0) in enumerate(tests):
        if i == max(args.warmup, 3):
            sampler.start()

        def cold():
            x, s, it, rr = prob.pcg(f, tol=tol)
            return x, s, it

        def warm():
            x0 = ws.predict(c0)[0]
            x, s, it, rr, u = ws.solve(f, x0, tol=tol)
            return x, s, it, u

        tc, (xc, sc, itc) = timed(cold)
        x0 = ws.predict(c0)[0].clone()
        e0 = (torch.linalg.vector_norm(x0 - xc) / torch.linalg.vector_norm(xc)).item()
        tw, (xw, sw, itw, u) = timed(warm)
        if sc != 0 or sw != 0:
            raise RuntimeError(f"solve failed: cold {sc}, warm {sw}")
        if i >= max(args.warmup, 3):
            warm_ms.append(tw)
            cold_ms.append(tc)
            it_w.append(itw)
            it_c.append(itc)
            e0s.append(e0)
            diffs.append((torch.linalg.vector_norm(xw - xc) / torch.linalg.vector_norm(xc)).item())
            used.append(u)
    clocks = sampler.stop()
    # end to end through the public calls: rhs and c0 from pinned host memory, solution back, every step
    f_h = [f.cpu().pin_memory() for f, _ in tests[:args.steps]]
    c_h = [c.cpu().pin_memory() for _, c in tests[:args.steps]]
    x_h = torch.empty_like(f_h[0]).pin_memory()
    fd, cd = prob.vec(), torch.empty_like(tests[0][1])
    e2e = []
    for fh, ch in zip(f_h, c_h):
        def e2e_step():
            fd.copy_(fh, non_blocking=True)
            cd.copy_(ch, non_blocking=True)
            x0 = ws.predict(cd)[0]
            x, s, it, rr, u = ws.solve(fd, x0, tol=tol)
            x_h.copy_(x, non_blocking=True)
            return s
        e2e.append(timed(e2e_step)[0])
    # the expansion kernel alone (reads the basis once: HBM-bound)
    Cq = torch.zeros((1, K), dtype=torch.float32, device="cuda")
    Xq = torch.empty((1, ws.m), dtype=torch.float64, device="cuda")
    exp_ms = []
    for _ in range(5):
        exp_ms.append(timed(lambda: S.stst_pod_expand(ws.Q_out, K, ws.m, Cq, 1, 1.0, 0.0, None, Xq))[0])
    exp_ms = statistics.median(exp_ms)
    peaks, src = load_peaks()
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    bytes_exp = 4.0 * K * ws.m + 8.0 * ws.m
    ms = statistics.mean(warm_ms)
    out = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": len(warm_ms),
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f64+f32", "bf16": "f64+f32+bf16"}[args.prec] + "+bf16 net",
        "data": "synthetic",
        "config": {"workload": f"c5: 2D+t p=3 48^2 x 48 elements ({prob.n_dof} unknowns), harmonic V in [0,10], "
                               f"wavepacket u0 (centre, width, momentum, phase drawn), tol {tol:g}",
                   "step": "one new problem: network inference (project c0, forward of every stage, expand) + "
                           "guarded PCG from the predicted iterate",
                   "model": (f"{args.stages} stages {K}->" + "".join(f"{h}->" for h in hidden) + f"{K}"
                             + (" (tanh between layers)" if hidden else " (linear)")
                             + f", {ws.n_params} parameters, BF16 weights, FP32 accumulation"),
                   "training_solves": args.train,
                   "l2": "flushed (512 MB write) before each step", "parallelism": f"replicas x{world}"},
        "warm": {"ms": ms, "pcg_iterations_mean": statistics.mean(it_w), "x0_rel_err_median": statistics.median(e0s),
                 "final_rel_diff_vs_cold_max": max(diffs), "warm_start_kept": int(sum(used))},
        "cold": {"ms": statistics.mean(cold_ms), "pcg_iterations_mean": statistics.mean(it_c)},
        "training": {"collect_s": t1 - t0, "pcg_iterations_mean": statistics.mean(its_train), "basis_s": t2 - t1,
                     "train_s": t3 - t2, "adam_steps_per_stage": args.train_steps},
        "roofline": {"kernel": "k_pod_expand_rows", "bound": "hbm", "achieved": bytes_exp / (exp_ms * 1e-3) / 1e9,
                     "peak": hbm, "unit": "GB/s", "frac": bytes_exp / (exp_ms * 1e-3) / 1e9 / hbm,
                     "peak_source": src, "traffic": None},
        "clocks": clocks,
        "e2e": {"value": statistics.mean(e2e) / 1e3, "unit": "s", "h2d_bytes_per_step": 16 * (prob.n_dof + prob.N_s),
                "d2h_bytes_per_step": 16 * prob.n_dof},
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    ws.close()
    prob.close()


def roofline_steps(n_dof, n_l, flops_dof, t_prec_ms, t_sys_ms, prec, peaks, fp64_peak, fp32_peak):
    """t_bound / t_measured per operator, t_bound = max(flops / pipe peak, algorithmic bytes / HBM peak).

    apply_prec (Algorithm 1 steps 2-4): 8 N sum_l n_l flops for the mode products (4 n_l per complex
    unknown per mode, forward and backward) on the FP32 or FP64 pipe; apply_sys (Eq. syst_mat): the
    planner's flops per unknown on the FP64 pipe. Bytes: r in and s out in FP64, 32 B per unknown."""
    hbm = peaks["hbm_gbs"] * 1e9
    out = {}
    fl = 8.0 * n_dof * sum(n_l)
    pk = (fp64_peak if prec == "fp64" else fp32_peak) * 1e12
    tb = max(fl / pk, 32.0 * n_dof / hbm)
    out["apply_prec"] = {"flops": fl, "bytes": 32.0 * n_dof, "pipe": "fp64" if prec == "fp64" else "fp32",
                         "t_bound_ms": tb * 1e3, "t_ms": t_prec_ms, "frac": tb * 1e3 / t_prec_ms}
    if prec == "bf16":
        out["apply_prec"]["pipe"] = "fp32 bound used (BF16x3 on tensor cores, time solves FP32)"
    fl = flops_dof * n_dof
    tb = max(fl / (fp64_peak * 1e12), 32.0 * n_dof / hbm)
    out["apply_sys"] = {"flops": fl, "bytes": 32.0 * n_dof, "pipe": "fp64", "t_bound_ms": tb * 1e3, "t_ms": t_sys_ms,
                        "frac": tb * 1e3 / t_sys_ms}
    return out


def run_ours(args):
    import numpy as np
    import torch
    import paper_2311_18461_gb300 as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cfg, V, u0 = workload(args.config)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        prob, b = build_problem(cfg, V, u0, args.prec, stream, args.formulation, args.prec_op)
    tol = cfg.get("tol", 1e-8)
    x = prob.vec()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    def solve(xv, rhs=None):
        rhs = b if rhs is None else rhs
        xv.zero_()
        prob.build_fd()
        if args.solver == "ir":
            st, inner, outer, rr = S.stst_ir_solve(prob.h, rhs, xv, tol, 30, args.inner_tol, 200)
            return st, inner, rr
        return S.stst_pcg_solve(prob.h, rhs, xv, tol, 200)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            st, it, rr = solve(x)
        assert st == 0, f"solve failed: status {st}"
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        times, iters = [], []
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, it, rr = solve(x)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            iters.append(it)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        if dist:
            dist.barrier()
        ms = max_over_ranks(statistics.mean(times), dist, "cuda")

        # PCG alone (preconditioner built beforehand): the paper's "solve" without its setup
        prob.build_fd()
        pcg_only = []
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            x.zero_()
            e0.record(stream)
            if args.solver == "ir":
                S.stst_ir_solve(prob.h, b, x, tol, 30, args.inner_tol, 200)
            else:
                S.stst_pcg_solve(prob.h, b, x, tol, 200)
            e1.record(stream)
            e1.synchronize()
            pcg_only.append(e0.elapsed_time(e1))
        pcg_only_ms = statistics.mean(pcg_only)
        # the accurate solve: the same solve to relative residual ACC_TOL, which brings the mixed path's
        # solution within 1e-8 of the FP64 oracle's (timed like the steps)
        x_acc = prob.vec()
        acc_ms, acc_its = [], []
        for _ in range(max(1, min(args.steps, 5))):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x_acc.zero_()
            prob.build_fd()
            if args.solver == "ir":
                st_t, it_t, _, rr_t = S.stst_ir_solve(prob.h, b, x_acc, ACC_TOL, 60, args.inner_tol, 200)
            else:
                st_t, it_t, rr_t = S.stst_pcg_solve(prob.h, b, x_acc, ACC_TOL, 400)
            e1.record(stream)
            e1.synchronize()
            acc_ms.append(e0.elapsed_time(e1))
            acc_its.append(it_t)

        # end to end through the C ABI with host buffers: pinned rhs in, solution out, every step
        b_host = b.cpu().pin_memory()
        x_host = torch.empty_like(b_host).pin_memory()
        b_dev = torch.empty_like(b)
        e2e = []
        for k in range(args.steps + 1):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b_dev.copy_(b_host, non_blocking=True)
            st, it2, rr2 = solve(x, b_dev)
            x_host.copy_(x, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if k > 0:
                e2e.append(e0.elapsed_time(e1))
        e2e_ms = statistics.mean(e2e)

        # per-kernel device times: launch durations from back-to-back profiled operator calls (the queue
        # stays ahead of the GPU, so events bracket kernels only), launch counts from one profiled solve
        r = prob.vec()
        r.real.normal_()
        s = prob.vec()
        y = prob.vec()

        def tm(fn, n=30):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n):
                fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / n

        t_prec = tm(lambda: S.stst_apply_prec(prob.h, r, s))
        t_sys = tm(lambda: S.stst_apply_sys(prob.h, r, y))
        S.stst_profile(prob.h, 1)
        for _ in range(30):
            S.stst_apply_sys(prob.h, r, y)
        for _ in range(30):
            S.stst_apply_prec(prob.h, r, s)
        prof_ops = S.stst_profile_read(prob.h)
        S.stst_profile(prob.h, 1)
        flush.fill_(1)
        torch.cuda.nvtx.range_push("profiled_solve")
        _, it_prof, _ = solve(x)
        torch.cuda.nvtx.range_pop()
        prof_solve = S.stst_profile_read(prob.h)
        S.stst_profile(prob.h, 0)
        prof = {}
        for k, (cnt, tot) in prof_solve.items():
            per = prof_ops[k][1] / prof_ops[k][0] if k in prof_ops else tot / cnt
            prof[k] = (cnt, per * cnt)
        # kernels launched in the timed steps: the profiled solve runs the loop as plain launches, the
        # timed ones as graph bodies of several iterations (the last body may run past convergence)
        plain = int(sum(v[0] for v in prof.values()))
        if args.solver == "ir":
            launches = plain * args.steps
            launch_basis = "plain-launch count of one profiled solve x steps"
        else:
            kpb, ipb = S.stst_pcg_graph_info(prob.h)
            setup = plain - it_prof * (kpb // ipb)
            launches = sum(setup + -(-int(k) // ipb) * kpb for k in iters)
            launch_basis = (f"setup and PCG start {setup} kernels + ceil(iterations / {ipb}) graph bodies of "
                            f"{kpb} kernel nodes, per timed step")

    n_dof = prob.n_dof
    d = cfg["d"]
    n_l = prob.n[1:]
    n_passes, band_apps, flops_dof = S.stst_plan_info(prob.h)
    peaks, peak_src = load_peaks()
    fp64_peak = N_SM * FP64_FMA_PER_CLK_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    fp32_peak = N_SM * FP32_FMA_PER_CLK_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    # per-kernel shares of one profiled solve (plain launches bracketed by events), scaled to the graph-timed
    # step so that they add up to it
    prof_total = sum(v[1] for v in prof.values())
    shares = {k: v[1] / prof_total for k, v in prof.items()} if prof_total > 0 else {}
    # dominant kernel of the step = largest share
    dom = max(shares.items(), key=lambda kv: kv[1])[0] if shares else None
    roof = None
    if dom:
        cnt, tot = prof[dom]
        per_launch_s = tot / cnt / 1e3
        timing = "events around back-to-back profiled launches of the kernel"
        # the fused mat-vec runs all levels of one application in a single launch
        per_apply = 1 if dom.startswith("pass_fused") else n_passes
        if dom.startswith("pass"):
            # the mat-vec's launches: events around 30 back-to-back stst_apply_sys calls, per launch
            per_launch_s = t_sys / per_apply / 1e3
            timing = (f"events around 30 back-to-back stst_apply_sys calls on the handle's stream, divided by "
                      f"the {per_apply} launch(es) of one call")
        if dom.startswith("modeprod_bf16"):
            # HBM/L2 bound on tensor cores: read FP32 tile + write FP32 result per complex unknown
            roof = {"kernel": dom, "bound": "hbm", "achieved": 16.0 * n_dof / per_launch_s / 1e9,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s"}
        elif dom.startswith("modeprod"):
            flops = 4.0 * (sum(n_l) / d) * n_dof
            peak = fp64_peak if dom.endswith("f64") else fp32_peak
            roof = {"kernel": dom, "bound": "alu", "achieved": flops / per_launch_s / 1e12,
                    "peak": peak, "unit": "TFLOP/s"}
        elif dom.startswith("pass"):
            flops = flops_dof * n_dof / per_apply
            peak = fp64_peak if dom.endswith("f64") else fp32_peak
            roof = {"kernel": dom, "bound": "alu", "achieved": flops / per_launch_s / 1e12,
                    "peak": peak, "unit": "TFLOP/s"}
        else:
            vec_bytes = 16 * n_dof
            roof = {"kernel": dom, "bound": "hbm", "achieved": 3 * vec_bytes / per_launch_s / 1e9,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["peak_source"] = ("derived: %d SMs x %d FMA/clk x 2 x %.0f MHz (nominal max clock)"
                               % (N_SM, FP64_FMA_PER_CLK_SM if dom.endswith("f64") else FP32_FMA_PER_CLK_SM,
                                  SM_MAX_MHZ_NOMINAL)) if roof["bound"] == "alu" else f"hbm_gbs of {peak_src}"
        roof["launch_ms"] = per_launch_s * 1e3
        roof["launch_timing"] = timing
        roof["traffic"] = traffic_for(dom, {"n_dof": n_dof, "band_apps_per_dof": band_apps})
        if roof["traffic"] and dom.startswith("pass"):
            # the mat-vec's algorithmic bytes: x in and y out once per application, 32 B per unknown
            roof["traffic_per_apply_sys"] = roof["traffic"] * per_apply
            roof["traffic_over_algorithmic_bytes"] = roof["traffic"] * per_apply / (32.0 * n_dof)
        roof["share_of_step"] = shares[dom]
    out = {
        "metric": METRIC,
        "value": ms / 1e3,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": ms,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": (ms / 1e3 / TABLE1[(cfg["p"], cfg["n_el"][0])][1]
                        if args.config == "tw" and (cfg["p"], cfg["n_el"][0]) in TABLE1 else None),
        "dtype": {"fp64": "f64", "fp32": "f64+f32", "bf16": "f64+f32+bf16"}[args.prec],
        "data": "synthetic",
        "config": {"workload": workload_name(args.config, cfg, tol) + (", ultraweak formulation (Sec. 4.4)"
                                                                       if args.formulation == "uw" else ""),
                   "n_dof": n_dof, "preconditioner": args.prec + (" P_V (potential-aware)" if args.prec_op == "potential"
                                                                  else " P-hat"), "solver": args.solver,
                   "pcg_iterations": statistics.median(iters),
                   "step": "build_fd (setup) + pcg_solve from x0 = 0", "l2": "flushed (512 MB write) before each step",
                   "parallelism": f"replicas x{world}"},
        "pcg_only_ms": pcg_only_ms,
        "accurate_solve": {"tol": ACC_TOL, "ms": statistics.mean(acc_ms), "pcg_iterations": statistics.median(acc_its),
                           "status": st_t, "relres": rr_t,
                           "why": "the same step to relative residual 1e-10: the residual at which the mixed path's "
                                  "solution is within 1e-8 of the FP64 oracle's (error_vs_fp64_oracle)"},
        "roofline_steps": roofline_steps(n_dof, n_l, flops_dof, t_prec, t_sys, args.prec, peaks, fp64_peak, fp32_peak),
        "apply_prec_dofs_per_s": n_dof / (t_prec / 1e3),
        "apply_prec_ms": t_prec,
        "apply_sys_ms": t_sys,
        "mat_vec_plan": {"passes": n_passes, "band_apps_per_dof": band_apps, "flops_per_dof": flops_dof},
        "mode_product_tiles": [dict(zip(("cols_per_cta", "rows_per_cta", "tuned_us"), S.stst_tile_info(prob.h, l)))
                               for l in range(1, cfg["d"] + 1)],
        "time_solver": dict(zip(("segments", "segment_len", "segmented"),
                                S.stst_time_solver_info(prob.h, 0 if args.prec == "fp64" else 1))),
        "fused_2d_transforms": S.stst_fused_transforms_info(prob.h),
        "fused_2d_backward_split": S.stst_fused_transforms_split(prob.h)[1],
        "pencil_ctas": S.stst_pencil_info(prob.h),
        "kernels_ms_per_step": {k: round(ms * v, 4) for k, v in sorted(shares.items(), key=lambda kv: -kv[1])},
        "kernels_ms_profiled_solve": {k: round(v[1], 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
        "kernel_time_basis": ("kernels_ms_per_step = each kernel's share of one profiled solve (plain launches, "
                              "each bracketed by CUDA events; operator kernels timed back to back) times the "
                              "graph-timed step; the profiled solve itself is slower (launch gaps, no graph)"),
        "kernel_launches_per_solve": {k: v[0] for k, v in prof.items()},
        "gpu_launches": launches,
        "gpu_launches_basis": launch_basis,
        "roofline": roof,
        "clocks": clocks,
        "e2e": {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": 16 * n_dof, "d2h_bytes_per_step": 16 * n_dof},
        "paper_context": ({"table": f"Table 1, p={cfg['p']}, n_el={cfg['n_el'][0]}, this travelling wave, 1 CPU "
                                    f"thread at 1 GHz (vs_baseline = value / seconds)",
                           "seconds": TABLE1[(cfg["p"], cfg["n_el"][0])][1],
                           "iterations": TABLE1[(cfg["p"], cfg["n_el"][0])][0]}
                          if args.config == "tw" and (cfg["p"], cfg["n_el"][0]) in TABLE1 else
                          {"table": "Table 1, p=3, n_el=64, V=0 travelling wave, 1 CPU thread at 1 GHz",
                           "seconds": 4.7142, "iterations": 8}),
    }
    xg, xa, bn = x.cpu().numpy(), x_acc.cpu().numpy(), b.cpu().numpy()
    prob.close()
    del flush
    if rank == 0 and world == 1 and args.variants == "on" and args.config == "c2" and args.solver == "pcg":
        out["variants"] = run_variants(args)
    if rank == 0 and world == 1 and args.cpu_baseline == "on":
        out["cpu_baseline"] = cpu_baseline(args.config, formulation=args.formulation, prec_op=args.prec_op)
        out["error_vs_fp64_oracle"] = error_vs_oracle(args, xg, xa, bn, tol)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


ACC_TOL = 1e-10
ORACLE_REF_TOL = 1e-13


def error_vs_oracle(args, x_timed, x_acc, b, tol):
    """The GPU's solutions against the FP64 oracle's solution of the same system: the oracle's PCG with the
    exact P-hat to relative residual 1e-13 on the GPU's own right-hand side (so that the comparison measures
    the solver, not the right-hand side's rounding times the condition number), errors as max-abs relative."""
    import numpy as np
    from oracle import fd, pcg
    cfg, disc, _ = oracle_problem(args.config, args.formulation)
    F = (fd.PotentialFastDiagonalization if args.prec_op == "potential" else fd.FastDiagonalization)(disc)
    x_ref, its, rr, _ = pcg.pcg(disc.apply, F.apply, b, tol=ORACLE_REF_TOL, maxit=400)
    den = np.abs(x_ref).max()
    true_res = float(np.linalg.norm(b - disc.apply(x_timed)) / np.linalg.norm(b))
    return {"timed_solve_rel_err": float(np.abs(x_timed - x_ref).max() / den),
            "timed_solve_true_residual": true_res,
            "accurate_solve_rel_err": float(np.abs(x_acc - x_ref).max() / den),
            "accurate_solve_tol": ACC_TOL,
            "reference": f"oracle PCG (numpy FP64, exact P-hat, {its} iterations) to relative residual "
                         f"{ORACLE_REF_TOL:g} on the GPU's right-hand side; max |x - x_ref| / max |x_ref|",
            "gpu": f"{args.prec} preconditioner in the FP64 flexible CG; timed solve to {tol:g}, accurate solve to "
                   f"{ACC_TOL:g}"}


VARIANTS = [("c2", "fp64"), ("c2", "bf16"), ("c3p2", "fp32"), ("c3p4", "fp32")]


def run_variants(args, steps=5, warmup=3):
    """Other precisions and the 3D+t workloads, each timed like the main step (setup + PCG from x0 = 0 to the
    workload's tolerance, L2 flushed, CUDA events on the handle's stream), so that one driver run carries
    them: the FP64-preconditioned path is the precision-matched baseline of the mixed one."""
    import torch
    import paper_2311_18461_gb300 as S
    out = {}
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for name, prec in VARIANTS:
        cfg, V, u0 = workload(name)
        tol = cfg.get("tol", 1e-8)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            prob, b = build_problem(cfg, V, u0, prec, stream)
            x = prob.vec()

            def solve():
                x.zero_()
                prob.build_fd()
                return S.stst_pcg_solve(prob.h, b, x, tol, 200)

            for _ in range(warmup):
                st, it, rr = solve()
            times, its = [], []
            for _ in range(steps):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st, it, rr = solve()
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                its.append(it)
        out[f"{name}_{prec}"] = {"workload": workload_name(name, cfg, tol), "preconditioner": prec, "n_dof": prob.n_dof,
                                 "ms_per_step": statistics.mean(times), "pcg_iterations": statistics.median(its),
                                 "status": st, "relres": rr, "steps": steps, "warmup": warmup}
        prob.close()
        torch.cuda.synchronize()
    out["c2_annulus_fp32"] = run_mapped(flush, steps, warmup)
    return out


def run_mapped(flush, steps, warmup):
    """The c2 mesh (2D+t, p=3, 64^2 x 64 elements, V = 0) on the quarter annulus 1 <= r <= 2 (Sec. 3.2 with
    F != id): setup (the mapped-domain matrices and the scaled P-hat) plus PCG to relative residual 1e-8 with
    the FP32 preconditioner, for a seeded random load vector (the library assembles no mapped-domain load
    vector)."""
    import numpy as np
    import torch
    import paper_2311_18461_gb300 as S
    from inputs import random_complex
    from inputs.geometry import QuarterAnnulus, geometry_at
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        prob = S.Problem(2, [64, 64, 64], 3, prec_mode=S.STST_PREC_FP32, stream=stream)
        grids = [prob.quad_points(l).cpu().numpy() for l in (1, 2)]
        J, H = geometry_at(QuarterAnnulus(1.0, 2.0), grids)
        jac = torch.tensor(np.ascontiguousarray(J), device="cuda")
        hess = torch.tensor(np.ascontiguousarray(H), device="cuda")
        b = torch.tensor(random_complex(prob.n_dof, 12), device="cuda")
        x = prob.vec()

        def solve():
            x.zero_()
            prob.set_geometry(jac, hess)
            prob.build_fd()
            return S.stst_pcg_solve(prob.h, b, x, 1e-8, 1000)

        for _ in range(warmup):
            st, it, rr = solve()
        times, its = [], []
        for _ in range(steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, it, rr = solve()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            its.append(it)
    scales = S.stst_geometry_info(prob.h, with_scales=True)[2][:2]
    prob.close()
    torch.cuda.synchronize()
    return {"workload": "c2 mesh (2D+t p=3 64^2 x 64) on the quarter annulus 1 <= r <= 2, V=0, seeded random "
                        "load vector, tol 1e-8", "preconditioner": "fp32 (scaled P-hat)", "n_dof": 278850,
            "prec_scales": scales, "ms_per_step": statistics.mean(times), "pcg_iterations": statistics.median(its),
            "status": st, "relres": rr, "steps": steps, "warmup": warmup,
            "timed": "geometry setup (metric, stencil assembly) + build_fd + PCG"}


def _oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        return max(i.get("num_threads", 1) for i in threadpool_info()) or os.cpu_count()
    except Exception:
        return os.cpu_count()


def cpu_model():
    """The host CPU's model name and logical core count (recorded beside every oracle timing)."""
    name = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    name = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"model": name or platform.processor() or platform.machine(), "logical_cores": os.cpu_count(),
            "machine": platform.machine()}


def oracle_problem(cfg_name, formulation="ls", n_el=None):
    """The oracle's discretisation and right-hand side of a workload (n_el: the same workload on another mesh)."""
    from inputs import potential, initial_factors, product_fn, travelling_wave
    from oracle import rhs
    from oracle.system import Discretization
    cfg, _, _ = workload(cfg_name)
    if n_el is not None:
        cfg = dict(cfg, n_el=list(n_el))
    d = cfg["d"]
    disc = Discretization(cfg["n_el"], [cfg["p"]] * (d + 1), T=cfg["T"], nu=cfg["nu"], potential=potential(cfg),
                          formulation=formulation)
    if cfg["u0"] == "travelling_wave":
        u_fn, f_fn = travelling_wave()
        b, _ = rhs.full_lifting(disc, u_fn, f_fn)
    elif formulation == "uw":
        b = rhs.rhs_ultraweak(disc, None, product_fn(initial_factors(cfg)))
    else:
        b, _ = rhs.rhs_initial(disc, None, product_fn(initial_factors(cfg)))
    return cfg, disc, b


def oracle_solve_times(disc, b, tol, runs, prec_op="phat"):
    """Full oracle solves as in the paper's Table 1: preconditioner setup (Algorithm 1 step 1 and the H_i)
    plus PCG from x0 = 0 to relative residual tol. Returns (seconds of each run, iterations)."""
    from oracle import fd, pcg
    FD = fd.PotentialFastDiagonalization if prec_op == "potential" else fd.FastDiagonalization
    times, its = [], None
    for _ in range(runs):
        t0 = time.perf_counter()
        F = FD(disc)
        _, its, _, _ = pcg.pcg(disc.apply, F.apply, b, tol=tol, maxit=400)
        times.append(time.perf_counter() - t0)
    return times, its


SINGLE_THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                     "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")


def oracle_single_thread_times(cfg_name, formulation, prec_op, n_el, runs):
    """oracle_solve_times in a child process whose BLAS and OpenMP pools have one thread (the pools are
    sized when numpy loads, so the limit has to be set before that)."""
    env = dict(os.environ)
    for k in SINGLE_THREAD_ENV:
        env[k] = "1"
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "cfg, disc, b = bench.oracle_problem(%r, %r, n_el=%r); "
            "bench.oracle_solve_times(disc, b, cfg.get('tol', 1e-8), 1, %r); "
            "t, it = bench.oracle_solve_times(disc, b, cfg.get('tol', 1e-8), %d, %r); "
            "print(json.dumps({'t': t, 'its': it, 'n_dof': disc.N_dof}))"
            % (ROOT, cfg_name, formulation, list(n_el), prec_op, runs, prec_op))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("single-thread oracle run failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def _small_mesh(cfg):
    """The same workload on half the elements per direction (the stated smaller sample)."""
    return [max(4, n // 2) for n in cfg["n_el"]]


def cpu_baseline(cfg_name, formulation="ls", prec_op="phat", runs=3, small_runs=5):
    """The oracle as it stands (numpy/scipy FP64) timed on this host's cores, no extrapolation:
      * all cores: the median of `runs` full solves of the workload itself (2D+t and smaller), or of the
        stated half-size mesh for 3D+t workloads (a full 3D+t oracle solve takes minutes);
      * one thread: the median of `small_runs` full solves of the workload on the half-size mesh.
    A full solve is the preconditioner setup plus PCG from x0 = 0 to the workload's tolerance."""
    cfg, _, _ = workload(cfg_name)
    tol = cfg.get("tol", 1e-8)
    big = cfg["d"] <= 2
    small = _small_mesh(cfg)
    _, disc_s, b_s = oracle_problem(cfg_name, formulation, n_el=small)
    oracle_solve_times(disc_s, b_s, tol, 1, prec_op)              # warm-up: libraries loaded, caches filled
    if big:
        _, disc, b = oracle_problem(cfg_name, formulation)
        t_all, its_all = oracle_solve_times(disc, b, tol, runs, prec_op)
    else:
        disc = disc_s
        t_all, its_all = oracle_solve_times(disc_s, b_s, tol, runs, prec_op)
    cores = _oracle_threads()
    one = oracle_single_thread_times(cfg_name, formulation, prec_op, small, small_runs)
    t_one, its_one = one["t"], one["its"]
    mesh = "x".join(str(n) for n in cfg["n_el"])
    smesh = "x".join(str(n) for n in small)
    out = {"value": statistics.median(t_all), "unit": "s", "cores": cores, "kind": "oracle",
           "sample": (f"median of {runs} full oracle solves (setup + PCG from x0 = 0 to {tol:g}, {its_all} "
                      f"iterations) of the {'workload' if big else 'workload on the half-size mesh ' + smesh} "
                      f"({disc.N_dof} unknowns) on {cores} threads; numpy/scipy FP64, no extrapolation"),
           "runs_s": [round(t, 4) for t in t_all],
           "single_thread": {"value": statistics.median(t_one), "unit": "s", "cores": 1, "runs": small_runs,
                             "runs_s": [round(t, 4) for t in t_one], "iterations": its_one,
                             "workload": f"{cfg_name} on the half-size mesh {smesh} ({disc_s.N_dof} unknowns)"},
           "cpu": cpu_model(),
           "workload_mesh": mesh if big else smesh}
    return out


def run_reference(args):
    """The reference arm: the oracle (the paper ships no code), timed on the host cores. One step is one
    full oracle solve of the workload (2D+t and smaller): setup plus PCG to the workload's tolerance, no
    extrapolation. Warm-up steps are untimed solves of the half-size mesh. 3D+t workloads, whose full
    oracle solves take minutes, time the half-size mesh and say so."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    formulation = args.formulation
    if args.config == "c4":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single-problem workloads "
                          "(c1, c2, c3*, c5, tw); c4's 128 problems have no bounded oracle sample"}), flush=True)
        return
    cfg, _, _ = workload(args.config)
    tol = cfg.get("tol", 1e-8)
    big = cfg["d"] <= 2
    small = _small_mesh(cfg)
    _, disc_s, b_s = oracle_problem(args.config, formulation, n_el=small)
    oracle_solve_times(disc_s, b_s, tol, max(args.warmup, 1), args.prec_op)
    if big:
        _, disc, b = oracle_problem(args.config, formulation)
    else:
        disc, b = disc_s, b_s
    times, its = oracle_solve_times(disc, b, tol, args.steps, args.prec_op)
    v = statistics.mean(times)
    cores = _oracle_threads()
    smesh = "x".join(str(n) for n in small)
    sample = (f"{args.steps} full oracle solves (setup + PCG from x0 = 0 to {tol:g}, {its} iterations) of the "
              + ("workload" if big else f"workload on the half-size mesh {smesh}")
              + f" ({disc.N_dof} unknowns), mean; warm-up: {max(args.warmup, 1)} solves of the half-size mesh; "
              f"numpy/scipy FP64 on {cores} threads")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_name(args.config, cfg, tol)
                                  + (", ultraweak formulation (Sec. 4.4)" if formulation == "uw" else "")
                                  + ("" if big else f", half-size mesh {smesh}"),
                      "n_dof": disc.N_dof, "preconditioner": "fp64 (oracle) " + ("P_V (potential-aware)"
                                                                                if args.prec_op == "potential"
                                                                                else "P-hat"),
                      "solver": "pcg", "pcg_iterations": its, "step": "build_fd (setup) + pcg_solve from x0 = 0",
                      "parallelism": "oracle on the host cores, rank 0"},
           "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample,
                            "cpu": cpu_model()},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    TW["p"], TW["n_el"] = args.tw_p, args.tw_nel
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_2311_18461_gb300 import build
        build.build()
        import paper_2311_18461_gb300 as S
        S.stst_set_autotune(args.autotune)
        S.stst_set_time_solver(args.time_solver)
        S.stst_set_fused_transforms(args.fused_transforms)
        S.stst_set_pencil(args.pencil)
        S.stst_set_tensor_products(args.tensor_products)
        S.stst_set_fused_matvec(args.fused_matvec)
        if args.config == "c4":
            run_batch(args)
        elif args.config == "c5":
            run_warmstart(args)
        else:
            run_ours(args)


if __name__ == "__main__":
    main()
