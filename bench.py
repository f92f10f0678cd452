"""Benchmark of the CC linear-response hot path (arXiv 2307.14296) on one B300 per rank.

One step = the whole path on the diatomic-scale workload: ground-state CCSD (T1/T2) and its
Hbar intermediates, the Lambda equations (left sigma), the damped response solves of three
dipole operators at 16 frequencies (all shifts +-w +-i gamma in shared trial spaces) and the
symmetric CC-CC response function <<mu;mu>>(w + i gamma).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cclr|reference] [--precision bf16x3|fp64]

Prints one JSON line (rank 0).  `value` is the algorithmic sigma throughput of the whole step:
8 x (packed complex multiply-adds of one sigma product) x (sigma-type products in the step:
right and left sigma vectors, CCSD residual evaluations, Hessian products) / step time.
Under torchrun every rank solves its own replica of the workload (independent problems, no
data-path collective: weak scaling); rank 0 reports the sum over ranks and the max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # diatomic scale (the benchmark workload)
    "30x200": dict(n_occ=30, n_vir=200, n_freq=16, w_min=0.05, w_max=0.30, gamma=0.005, n_ops=3, tol=1e-8),
    # smaller replica of the same path (profiling captures that must stay small)
    "12x90": dict(n_occ=12, n_vir=90, n_freq=4, w_min=0.05, w_max=0.30, gamma=0.005, n_ops=3, tol=1e-8),
    # mixed precision at scale: 4 frequencies, gamma 0.01, refined to a residual of 1e-8
    "40x260": dict(n_occ=40, n_vir=260, n_freq=4, w_min=0.05, w_max=0.30, gamma=0.01, n_ops=3, tol=1e-8),
    # adjoint gradients of alpha(0.1 + 0.005i) (operator elements and a static field)
    "20x150": dict(n_occ=20, n_vir=150, n_freq=1, w_min=0.1, w_max=0.1, gamma=0.005, n_ops=3, tol=1e-10),
}
WORKLOAD = WORKLOADS["30x200"]
METRIC = "CC-LR sigma TFLOP/s and s per converged α(ω) at 1e-6; mixed/batched vs FP64"


def sigma_cmac(o: int, v: int) -> float:
    """Packed complex multiply-adds of one sigma product: ladder Po*Pv^2, ring o^3 v^3, and the
    o^2 v^3, o^3 v^2, o^4 v^2 terms (counts of the SI sigma equations on unique pairs)."""
    Po, Pv = o * (o - 1) / 2, v * (v - 1) / 2
    return Po * Pv * Pv + o**3 * v**3 + 5.5 * o**2 * v**3 + 6 * o**3 * v**2 + o**4 * v**2 / 4


# The per-vector contractions of the CC Hessian product (u F) as the library runs them (SI working
# equations for (t^X F), unpacked tensors); z is the batch index.
HESSIAN_TERMS = (
    "kica,zia->zkc ka,zia->zik ic,zik->zkc ic,zia->zca ka,zca->zkc eica,zia->zec ke,zec->zkc kima,zia->zkm "
    "mc,zkm->zkc ma,zia->zim ikmc,zim->zkc ie,zia->zea ekac,zea->zkc kjab,zijab->zki ic,zki->zkc "
    "ijcb,zijab->zca ka,zca->zkc ia,zijab->zjb jkbc,zjb->zkc mkae,zia->zmkei zmkei,iecm->zkc keam,zia->zekmi "
    "imec,zekmi->zkc kifa,zia->zkf fc,zkf->zkc nica,zia->znc kn,znc->zkc fa,zia->zif ikfc,zif->zkc "
    "in,zia->zna nkac,zna->zkc ijac,zijab->zcb kb,zcb->zkc ikab,zijab->zkj jc,zkj->zkc ikeb,zijab->zkeja "
    "zkeja,ejac->zkc ikmb,zijab->zkmja mjac,zkmja->zkc ekab,zijab->zekij ijec,zekij->zkc mkab,zijab->zmkij "
    "ijmc,zmkij->zkc ijae,zijab->zeb ekbc,zeb->zkc imab,zijab->zmj jkmc,zmj->zkc lida,zia->zld kc,zld->zklcd "
    "ka,zia->zki ikab,zijab->zkj zki,ilcd->zklcd ic,zia->zca ijac,zijab->zcb zca,klad->zklcd la,zia->zli "
    "lima,zia->zlm ljab,zijab->zli kicd,zli->zklcd id,zia->zda eida,zia->zde ijdb,zijab->zda "
    "klca,zda->zklcd klma,zia->zklmi klab,zijab->zklij micd,zklmi->zklcd kimd,zia->zkmda lida,zijab->zljdb "
    "ekdf,zif->zkide mlca,zkmda->zklcd klea,zia->zklei zklei,eicd->zklcd klab,zijab->zklij zklij,ijcd->zklcd"
).split()


def hessian_cmac(o: int, v: int) -> float:
    """Complex MACs of one Hessian product: per contraction, the product of the index ranges
    over both operands' indices (occupied i..n -> o, virtual a..f -> v)."""
    tot = 0.0
    for t in HESSIAN_TERMS:
        idx = set(t.split("->")[0].replace(",", "")) - {"z"}
        tot += float(np.prod([o if ch in "ijklmn" else v for ch in idx]))
    return tot


def prec_of(pk, name: str) -> int:
    return {"bf16x3": pk.TC_BF16X3, "bf16x6": pk.TC_BF16X6, "f64tc": pk.TC_F64, "fp64": pk.FP64}[name]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class Clocks:
    """nvidia-smi sampling (200 ms) during the timed region."""

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) > 8 for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce(x, world, op="max"):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------------------------------ CPU
def oracle_sample(budget_s: float = 20.0):
    """The FP64 oracle as it stands on this host: full path (CCSD, Lambda, one damped frequency
    for the three dipole operators) on the (8 occupied, 60 virtual) member of the benchmark's
    system family; returns (TFLOP/s by the same sigma-count rule, seconds, description)."""
    import synth
    from oracle.ints import Ints
    from oracle import response as R
    o, v = 8, 60
    inst = synth.make_instance(o, v)
    t0 = time.perf_counter()
    s = R.CCSystem(Ints.from_instance(inst), tol=1e-8)
    n_sig = s.ground_iters + s.lambda_iters
    z = [0.1 + 1j * WORKLOAD["gamma"]]
    calls = {"n": 0}
    orig = s.sigma_r

    def counted(vec):
        calls["n"] += 1
        return orig(vec)

    s.sigma_r = counted
    s.response(inst.ops, z, tol=1e-8)
    dt = time.perf_counter() - t0
    n_sig += calls["n"]
    flops = 8 * sigma_cmac(o, v) * n_sig
    return flops / dt / 1e12, dt, (f"oracle (NumPy FP64) full path at n_occ={o}, n_vir={v}: CCSD + Lambda + "
                                    f"one damped frequency x 3 operators ({n_sig} sigma-type products, {dt:.1f} s); "
                                    f"the oracle's v^4 tensors (25.6 GB at 200 virtuals) rule out a 30/200 sample")


def oracle_sigma_one_thread(o: int = 8, v: int = 60):
    """One right sigma product of the oracle with the BLAS limited to one thread (the paper's CPU
    timings use one OpenMP thread): seconds and TFLOP/s by the sigma-count rule."""
    # a fresh interpreter whose BLAS starts with one thread (the variables are read at load time)
    code = ("import sys, time; sys.path.insert(0, %r); import synth; from oracle.ints import Ints; "
            "from oracle import response as R; inst = synth.make_instance(%d, %d); "
            "s = R.CCSystem(Ints.from_instance(inst), tol=1e-8); x = synth.random_vector((s.D.size,), 5, 5, 1e-2); "
            "s.sigma_r(x); t0 = time.perf_counter(); s.sigma_r(x); print(time.perf_counter() - t0)") % (ROOT, o, v)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1200)
    dt = float(r.stdout.strip().splitlines()[-1])
    return dt, 8 * sigma_cmac(o, v) / dt / 1e12


def run_reference(args, world, rank):
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    times, vals = [], []
    for i in range(args.warmup + args.steps):
        tf, dt, desc = oracle_sample()
        if i >= args.warmup:
            times.append(dt)
            vals.append(tf)
    value = statistics.mean(vals)
    line = dict(metric=METRIC, value=value, unit="TFLOP/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * statistics.mean(times), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(config_dict(args), reference_sample="each step: the oracle's full path on the 8/60 "
                            "member of the same system family (the 30/200 system does not fit the oracle)"),
                cpu_baseline=dict(value=value, unit="TFLOP/s", cores=cores, kind="oracle", sample=desc),
                e2e=dict(value=value, unit="TFLOP/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def config_dict(args):
    w = WORKLOAD
    return {"workload": (f"diatomic-scale CC-LR: {w['n_occ']} occupied / {w['n_vir']} virtual spinors, "
                         f"{w['n_ops']} dipole operators, {w['n_freq']} frequencies on [{w['w_min']},{w['w_max']}] au, "
                         f"gamma {w['gamma']} au, synthetic complex antisymmetrized integrals"),
            "n_occ": w["n_occ"], "n_vir": w["n_vir"], "n_freq": w["n_freq"], "gamma": w["gamma"],
            "precision": args.precision,
            "l2": "inputs larger than L2 (packed vvvv block %.2f GB)" % (16 * (w["n_vir"] * (w["n_vir"] - 1) / 2) ** 2 / 1e9)}


# ------------------------------------------------------------------------------------------ GPU
def accuracy_vs_fp64(pk, synth):
    """The mixed-precision path against the GPU's plain FP64 path on the 12/90 replica (16
    frequencies, 3 operators, the full path from the Hamiltonian to alpha), both timed: alpha
    error per component (against its own size and against the largest component), of the mean
    alpha, and the end-to-end seconds of each run.  Runs: FP64 (DFMA) to 1e-11 / 1e-11 (residual
    of the response / ground-state equations), split BF16 with FP64 refinement to 1e-10 / 1e-10,
    and split BF16 without refinement (stopped at its floor) for contrast."""
    w = WORKLOADS["12x90"]
    o, v = w["n_occ"], w["n_vir"]
    inst = synth.make_instance(o, v)
    om = np.linspace(w["w_min"], w["w_max"], 16)
    runs = {"fp64": dict(precision=pk.FP64, tol=1e-11, ground_tol=1e-11),
            "bf16x3_refined": dict(precision=pk.TC_BF16X3, tol=1e-10, ground_tol=1e-10),
            "bf16x3_unrefined": dict(precision=pk.TC_BF16X3, tol=1e-10, ground_tol=1e-10, refine=0)}
    res, secs, refine = {}, {}, {}
    for name, opt in runs.items():
        ctx = pk.Context(0, max_subspace=64, batch=8, maxit=100, **opt)
        t0 = time.perf_counter()
        ctx.cclr_set_hamiltonian(o, v, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
        ctx.cc_ground()
        rv = ctx.cclr_get_stats()["refine_vectors"]
        ctx.cc_lambda()
        rv += ctx.cclr_get_stats()["refine_vectors"]
        ctx.cc_lr_solve(inst.ops, om, w["gamma"])
        st = ctx.cclr_get_stats()
        rv += st["refine_vectors"]
        res[name] = -ctx.cc_response_function()
        secs[name] = time.perf_counter() - t0
        refine[name] = dict(refine_sigma_products=rv, final_response_residual=st["max_residual"])
        if name == "bf16x3_refined":
            # the asymmetric form from the same solutions (first-order multipliers, left solves)
            t0 = time.perf_counter()
            res["asym_refined"] = -ctx.cc_response_function_asym()
            secs["asym_refined"] = time.perf_counter() - t0
        ctx.close()
    b = res["fp64"]
    out = dict(workload="12/90 replica, 16 frequencies on [0.05,0.30], gamma 0.005, 3 operators, "
                        "Hamiltonian to alpha", smallest_component=float(np.abs(b).min()),
               largest_component=float(np.abs(b).max()), fp64_seconds=secs["fp64"])
    for name in ("bf16x3_refined", "bf16x3_unrefined"):
        a = res[name]
        d = np.abs(a - b)
        mean_a, mean_b = np.trace(a, axis1=1, axis2=2) / 3, np.trace(b, axis1=1, axis2=2) / 3
        out[name] = dict(max_rel_per_component=float((d / np.abs(b)).max()),
                         max_rel_to_largest=float(d.max() / np.abs(b).max()),
                         max_rel_mean_alpha=float((np.abs(mean_a - mean_b) / np.abs(mean_b)).max()),
                         seconds=secs[name], speedup_vs_fp64=secs["fp64"] / secs[name], **refine[name])
    d = np.abs(res["asym_refined"] - b)
    out["asymmetric_form_refined"] = dict(
        note="split BF16 with refinement, multipliers refined to 1e-10; against the FP64 symmetric form",
        max_rel_per_component=float((d / np.abs(b)).max()), max_rel_to_largest=float(d.max() / np.abs(b).max()),
        seconds=secs["asym_refined"])
    return out


def eom_replica(pk, synth):
    """Four lowest EOM-EE roots on the 12/90 replica in split-BF16 and in FP64 (the FP64 solve at
    the full workload takes minutes): the difference of the roots."""
    w = WORKLOADS["12x90"]
    o, v = w["n_occ"], w["n_vir"]
    inst = synth.make_instance(o, v)
    out = {"workload": "12/90 replica, 4 lowest roots"}
    for name, prec in (("bf16x3", pk.TC_BF16X3), ("fp64", pk.FP64)):
        ctx = pk.Context(0, precision=prec, tol=1e-8, ground_tol=1e-10 if prec == pk.FP64 else 1e-8,
                         max_subspace=64, batch=8, maxit=80)
        ctx.cclr_set_hamiltonian(o, v, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
        ctx.cc_ground()
        t0 = time.perf_counter()
        roots, its = ctx.cc_eom_ee(4)
        dt = time.perf_counter() - t0
        st = ctx.cclr_get_stats()
        out[name] = dict(roots=[[float(r.real), float(r.imag)] for r in roots], iterations=its,
                         sigma_products=st["sigma_vectors"], seconds=dt)
        ctx.close()
    a = np.array([complex(*r) for r in out["bf16x3"]["roots"]])
    b = np.array([complex(*r) for r in out["fp64"]["roots"]])
    out["max_rel_diff_bf16x3_vs_fp64"] = float(np.abs(a - b).max() / np.abs(b).max())
    return out


def run_accuracy_at_scale(args):
    """The workload of --workload solved twice from the same Hamiltonian: split BF16 with FP64
    refinement (the requested tolerance) and the FP64-class tensor-core mode throughout (every
    contraction on the five-digit path, FP64 vector arithmetic, no mixed phase; the FP64 DFMA
    path would take ~45 min at 40/260), each timed end to end; prints the per-frequency,
    per-component relative error of alpha and both times as one JSON line."""
    import paper_2307_14296_b300 as pk
    import synth
    w = WORKLOAD
    o, v = w["n_occ"], w["n_vir"]
    inst = synth.make_instance(o, v)
    om = np.linspace(w["w_min"], w["w_max"], w["n_freq"])
    out, alpha = dict(mode="accuracy_at_scale", workload=config_dict(args)["workload"],
                      max_subspace=args.max_subspace, sigma_batch=args.sigma_batch), {}
    for name, prec in (("reference_f64tc", pk.TC_F64), ("bf16x3_refined", pk.TC_BF16X3)):
        ctx = pk.Context(0, precision=prec, tol=w["tol"], ground_tol=1e-9, max_subspace=args.max_subspace,
                         batch=args.sigma_batch, maxit=100)
        t0 = time.perf_counter()
        ctx.cclr_set_hamiltonian(o, v, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
        ctx.cc_ground()
        ctx.cc_lambda()
        ctx.cc_lr_solve(inst.ops, om, w["gamma"])
        st = ctx.cclr_get_stats()
        alpha[name] = -ctx.cc_response_function()
        out[name] = dict(seconds=time.perf_counter() - t0, final_response_residual=st["max_residual"],
                         refine_sigma_products=st["refine_vectors"])
        ctx.close()
    a, b = alpha["bf16x3_refined"], alpha["reference_f64tc"]
    out["per_frequency"] = [dict(omega=float(om[f]), max_rel_per_component=float((np.abs(a[f] - b[f]) / np.abs(b[f])).max()),
                                 max_rel_to_largest=float(np.abs(a[f] - b[f]).max() / np.abs(b[f]).max()),
                                 mean_alpha=[float(np.trace(b[f]).real / 3), float(np.trace(b[f]).imag / 3)])
                            for f in range(len(om))]
    print(json.dumps(out), flush=True)


def run_adjoint(args):
    """Gradients of alpha on the workload of --workload (20/150 at w = 0.1, gamma = 0.005 by
    default): forward solve, then d Re and d Im of all nine components with respect to every
    real parameter of the three Hermitian dipole operators through the autograd backward (one
    set of 4 n_ops left solves, reused for the 18 Jacobian rows), checked against a central
    difference (h = 1e-4) of two further solves along one random Hermitian direction; and the
    static-field derivative d alpha / d eps for a field along operator 2 analytically
    (cclr_field_derivative) and by finite field
    (h = 1e-4).  One JSON line."""
    import torch
    import paper_2307_14296_b300 as pk
    from paper_2307_14296_b300 import autograd as ag
    import synth
    w = WORKLOAD
    o, v = w["n_occ"], w["n_vir"]
    inst = synth.make_instance(o, v)
    n = inst.n
    om = list(np.linspace(w["w_min"], w["w_max"], w["n_freq"]))
    prec = prec_of(pk, args.precision)
    blocks = [inst.blocks[k] for k in synth.CLASSES]

    def new_context():
        return pk.Context(0, precision=prec, tol=w["tol"], ground_tol=1e-10, max_subspace=args.max_subspace,
                          batch=8, maxit=100)
    dev = torch.device("cuda", 0)
    out = dict(mode="adjoint", workload=config_dict(args)["workload"], precision=args.precision, omega=om,
               gamma=w["gamma"])
    # warm-up of the PyTorch side of the backward (its kernels load and compile for this GPU at
    # first use, ~10 s once per process) on a small system, so that the timed rows are steady state
    wi = synth.make_instance(3, 8)
    wctx = new_context()
    wctx.cclr_set_hamiltonian(3, 8, wi.fock, [wi.blocks[k] for k in synth.CLASSES])
    wctx.cc_ground()
    wctx.cc_lambda()
    wth = torch.tensor(np.stack([ag.hermitian_params(wi.ops[k]) for k in range(3)]), device=dev, requires_grad=True)
    wal = ag.polarizability(torch.stack([ag.hermitian_from_params(wth[k], wi.n) for k in range(3)]), wctx, om,
                            w["gamma"])
    wg = torch.zeros_like(wal)
    wg[0, 0, 0] = 1.0
    torch.autograd.grad(wal, wth, grad_outputs=wg)
    wctx.close()
    ctx = new_context()
    t0 = time.perf_counter()
    ctx.cclr_set_hamiltonian(o, v, inst.fock, blocks)
    ctx.cc_ground()
    ctx.cc_lambda()
    out["ground_lambda_seconds"] = time.perf_counter() - t0
    th0 = np.stack([ag.hermitian_params(inst.ops[k]) for k in range(3)])
    th = torch.tensor(th0, device=dev, requires_grad=True)
    ops = torch.stack([ag.hermitian_from_params(th[k], n) for k in range(3)])
    t0 = time.perf_counter()
    alpha = ag.polarizability(ops, ctx, om, w["gamma"])
    torch.cuda.synchronize()
    out["forward_seconds"] = time.perf_counter() - t0
    jac = np.zeros((2, 3, 3) + th0.shape)
    t0 = time.perf_counter()
    for x in range(3):
        for y in range(3):
            for part, gv in enumerate((1.0, 1j)):
                g = torch.zeros_like(alpha)
                g[0, x, y] = gv
                (gt,) = torch.autograd.grad(alpha, th, grad_outputs=g, retain_graph=True)
                jac[part, x, y] = gt.cpu().numpy()
    torch.cuda.synchronize()
    out["backward_seconds_18_rows"] = time.perf_counter() - t0
    out["left_solves"] = 4 * 3
    a0 = alpha.detach().cpu().numpy()[0]
    out["alpha"] = [[[float(a0[x, y].real), float(a0[x, y].imag)] for y in range(3)] for x in range(3)]
    out["grad_norm_re"] = float(np.linalg.norm(jac[0]))
    out["grad_norm_im"] = float(np.linalg.norm(jac[1]))
    # central difference along one random direction of all operator parameters
    rng = np.random.default_rng(23)
    d = rng.standard_normal(th0.shape)
    h = 1e-4

    def alpha_at(t):
        o3 = np.stack([ag.hermitian_from_params(torch.from_numpy(t[k]), n).numpy() for k in range(3)])
        ctx.cc_lr_solve(o3, om, w["gamma"])
        return -ctx.cc_response_function()[0]
    t0 = time.perf_counter()
    fd = (alpha_at(th0 + h * d) - alpha_at(th0 - h * d)) / (2 * h)
    out["fd_seconds"] = time.perf_counter() - t0
    got = np.einsum("rxyk,k->rxy", jac.reshape(2, 3, 3, -1), d.ravel())
    err = max(np.abs(got[0] - fd.real).max(), np.abs(got[1] - fd.imag).max())
    out["fd_check"] = dict(h=h, max_abs_diff=float(err), max_abs_fd=float(np.abs(fd).max()),
                           max_rel=float(err / np.abs(fd).max()))
    # the static-field derivative analytically (cclr_field_derivative on the converged state)
    ctx.cc_lr_solve(inst.ops, om, w["gamma"])
    t0 = time.perf_counter()
    danal = -ctx.cclr_field_derivative(inst.ops[2])
    t_anal = time.perf_counter() - t0
    ctx.close()
    t0 = time.perf_counter()
    dfield, _, _ = ag.alpha_field_derivative(new_context, o, v, inst.fock, blocks, inst.ops[2], inst.ops, om,
                                             w["gamma"], h=1e-4)
    out["field"] = dict(operator=2, h=1e-4, seconds=time.perf_counter() - t0,
                        d_alpha_d_eps=[[[float(dfield[0, x, y].real), float(dfield[0, x, y].imag)] for y in range(3)]
                                       for x in range(3)],
                        analytic_seconds=t_anal,
                        analytic_vs_finite_field_max_rel=float(np.abs(danal - dfield).max() / np.abs(dfield).max()))
    print(json.dumps(out), flush=True)


# The plain-FP64 step of the 30/200 workload, measured once: `python bench.py --precision fp64
# --warmup 0 --steps 1 --no-e2e --no-breakdown --no-extra --no-cpu-baseline --no-accuracy` on a
# B300 (2026-12-04) had not finished when stopped after 1500 s.
FP64_STEP_30x200 = dict(lower_bound_seconds=1500.0,
                        how="python bench.py --precision fp64 --warmup 0 --steps 1 (30/200, 16 frequencies, "
                            "residual 1e-8) on a B300, stopped unfinished after 1500 s")

C2_SYSTEMS = [(8, 60), (12, 90), (18, 120)]


def run_batch(args):
    """Three uneven systems, (8,60), (12,90) and (18,120), x 3 dipole operators x 16 frequencies on
    [0.05, 0.30] (gamma 0.005), each from Hamiltonian to alpha in the FP32-class tensor-core mode
    with FP64 refinement to 1e-8: once as one batch (cclr_response_batch: one host thread and
    stream per system, kernels overlapping on the GPU) and once one system after another.  Also
    the FP64-class mode throughout for the largest system as the accuracy reference.  One JSON
    line."""
    import paper_2307_14296_b300 as pk
    import synth
    om = np.linspace(0.05, 0.30, 16)
    gamma = 0.005
    insts = [synth.make_instance(o, v, seed=synth.DEFAULT_SEED + 7 + k) for k, (o, v) in enumerate(C2_SYSTEMS)]
    prec = prec_of(pk, args.precision) if args.precision != "bf16x3" else pk.TC_BF16X6

    def contexts(p):
        cs = []
        for inst in insts:
            c = pk.Context(0, precision=p, tol=1e-8, ground_tol=1e-9, max_subspace=args.max_subspace, batch=8,
                           maxit=100)
            c.cclr_set_hamiltonian(inst.n_occ, inst.n_vir, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
            cs.append(c)
        return cs
    out = dict(mode="batch", workload="three uneven systems " + ", ".join(f"{o}/{v}" for o, v in C2_SYSTEMS) +
               ": 3 operators x 16 frequencies on [0.05,0.30], gamma 0.005, residual 1e-8", precision=prec)
    cs = contexts(prec)
    pk.cclr_response_batch(cs, [i.ops for i in insts], om[:2], gamma)   # warm-up (autotuner, caches)
    for c in cs:
        c.close()
    cs = contexts(prec)
    t0 = time.perf_counter()
    batched = pk.cclr_response_batch(cs, [i.ops for i in insts], om, gamma)
    out["batched_seconds"] = time.perf_counter() - t0
    for c in cs:
        c.close()
    seq = []
    t0 = time.perf_counter()
    for inst, c in zip(insts, contexts(prec)):
        c.cc_ground()
        c.cc_lambda()
        c.cc_lr_solve(inst.ops, om, gamma)
        seq.append(-c.cc_response_function())
        c.close()
    out["sequential_seconds"] = time.perf_counter() - t0
    out["batch_speedup"] = out["sequential_seconds"] / out["batched_seconds"]
    out["batch_vs_sequential_max_rel"] = max(float(np.abs(-b - s).max() / np.abs(s).max()) for b, s in zip(batched, seq))
    ref = []
    t0 = time.perf_counter()
    for inst, c in zip(insts, contexts(pk.TC_F64)):
        c.cc_ground()
        c.cc_lambda()
        c.cc_lr_solve(inst.ops, om, gamma)
        ref.append(-c.cc_response_function())
        c.close()
    out["f64tc_seconds"] = time.perf_counter() - t0
    out["per_system"] = [dict(system=f"{o}/{v}",
                              max_rel_per_component_vs_f64tc=float((np.abs(-b - r) / np.abs(r)).max()),
                              max_rel_to_largest_vs_f64tc=float(np.abs(-b - r).max() / np.abs(r).max()))
                         for (o, v), b, r in zip(C2_SYSTEMS, batched, ref)]
    print(json.dumps(out), flush=True)


def run_gemm(args):
    """Tensor-core GEMM alone on one shape (A: M x K, B: N x K, complex), e.g. the packed ladder
    contraction of eight trial vectors (M = 8 Po, K = Pv): a small case for kernel captures."""
    import paper_2307_14296_b300 as pk
    import synth
    M, N, K = (int(x) for x in args.gemm.split(","))
    rng = np.random.default_rng(2307)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))
    prec = prec_of(pk, args.precision)
    ctx = pk.Context(0, precision=prec)
    tiny = synth.make_instance(2, 4)   # a Hamiltonian gives the context its device workspace
    ctx.cclr_set_hamiltonian(2, 4, tiny.fock, [tiny.blocks[k] for k in synth.CLASSES])
    ctx.cclr_kernel_profile(True)
    for _ in range(max(1, args.warmup)):
        ctx.cclr_zgemm_nt(A, B, prec)
    ctx.cclr_kernel_profile(True)
    for _ in range(max(1, args.steps)):
        C = ctx.cclr_zgemm_nt(A, B, prec)
    prof = ctx.cclr_kernel_profile(False)
    if prec == pk.TC_F64:
        prof = prof["f64"]
    part = A[:4] @ B[:4].T
    rel = float(np.abs(C[:4, :4] - part).max() / np.abs(part).max())
    per = prof["ms"] / max(1, args.steps)
    print(json.dumps({"mode": "gemm", "M": M, "N": N, "K": K, "precision": args.precision,
                      "kernel_ms": per, "launches_per_call": prof["launches"] / max(1, args.steps),
                      "exec_tflops": prof["flops_exec"] / max(1, args.steps) / (per * 1e-3) / 1e12 if per > 0 else None,
                      "useful_tflops": prof["flops_useful"] / max(1, args.steps) / (per * 1e-3) / 1e12 if per > 0 else None,
                      "sample_rel_err": rel}))


def run_sigma(args):
    """One batched sigma product (8 trial vectors) alone, on a system of O occupied / V virtual
    spinors (right sigma, or left with SIDE = 1): a small case for kernel captures.  Prints the
    number of tensor-core GEMM launches before the timed calls (the ncu launch-skip of the first
    timed launch) and the per-kernel times of the last call."""
    import paper_2307_14296_b300 as pk
    import synth
    parts = [int(x) for x in args.sigma.split(",")]
    o, v, side = parts[0], parts[1], (parts[2] if len(parts) > 2 else 0)
    inst = synth.make_instance(o, v)
    prec = prec_of(pk, args.precision)
    ctx = pk.Context(0, precision=prec, tol=1e-6, ground_tol=1e-8, max_subspace=32, batch=8, maxit=60)
    ctx.cclr_set_hamiltonian(o, v, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
    ctx.cclr_kernel_profile(True)
    ctx.cc_ground()
    if side:
        ctx.cc_lambda()
    x = synth.random_vector((8, ctx.N), 5, 5, 1e-3)
    for _ in range(max(1, args.warmup)):
        ctx.cclr_sigma(x, side=side, precision=prec)
    warm = ctx.cclr_kernel_breakdown()
    before = sum(n for k, (n, ms) in warm.items() if k.split(" | ")[-1] == "k_tc_zgemm")
    before_split = sum(n for k, (n, ms) in warm.items() if k.split(" | ")[-1].startswith("k_split_view"))
    t_ms = []
    for _ in range(max(1, args.steps)):
        ctx.cclr_sigma(x, side=side, precision=prec)
        bd = ctx.cclr_kernel_breakdown()
        t_ms.append(sum(ms for _, ms in bd.values()))
    ctx.cclr_kernel_profile(False)
    print(json.dumps({"mode": "sigma", "o": o, "v": v, "side": side, "vectors": 8, "precision": args.precision,
                      "tc_launches_before_timed": before,
                      "tc_and_split_launches_before_timed": before + before_split, "kernel_ms_per_call": t_ms,
                      "kernels": {k: [n, ms] for k, (n, ms) in sorted(bd.items(), key=lambda kv: -kv[1][1])}}))


def run_vector_kernels(args):
    """The Davidson solver's multi-vector kernels alone on synthetic device vectors of length N:
    a Gram block (NX x NY) and the NX-row, M-output vecmat passes (norms only; outputs stored).
    Reports milliseconds per call and the bandwidth of the bytes each pass must move."""
    import paper_2307_14296_b300 as pk
    import synth
    n, nx, ny, m = (int(x) for x in args.vector_kernels.split(","))
    prec = prec_of(pk, args.precision)
    ctx = pk.Context(0, precision=prec)
    tiny = synth.make_instance(2, 4)   # a Hamiltonian gives the context its device workspace
    ctx.cclr_set_hamiltonian(2, 4, tiny.fock, [tiny.blocks[k] for k in synth.CLASSES])
    r = ctx.cclr_bench_vector_kernels(n, nx, ny, m, reps=max(1, args.steps), precision=prec)
    gb = dict(gram=16.0 * n * (nx + ny) / 1e9, norms=16.0 * n * nx / 1e9, write=16.0 * n * (nx + m) / 1e9)
    print(json.dumps({"mode": "vector_kernels", "n": n, "nx": nx, "ny": ny, "m": m, "precision": args.precision,
                      **r, **{f"{k}_gbs": gb[k] / (r[f"{k}_ms"] * 1e-3) for k in gb}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cclr", choices=["cclr", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "bf16x6", "f64tc", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-breakdown", action="store_true", help="skip the per-kernel timing step")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the mixed-vs-FP64 accuracy check")
    ap.add_argument("--no-extra", action="store_true", help="skip the CC-CI and EOM-EE measurements")
    ap.add_argument("--workload", default="30x200", choices=sorted(WORKLOADS))
    ap.add_argument("--gemm", default=None, metavar="M,N,K",
                    help="time only the tensor-core complex GEMM C = A B^T on one shape (kernel profiling)")
    ap.add_argument("--vector-kernels", default=None, metavar="N,NX,NY,M",
                    help="time only the solver's Gram and vecmat kernels on synthetic vectors (kernel profiling)")
    ap.add_argument("--sigma", default=None, metavar="O,V[,SIDE]",
                    help="time only one batched sigma product of 8 vectors on an O/V system (kernel profiling)")
    ap.add_argument("--accuracy-at-scale", action="store_true",
                    help="solve the workload refined and in the FP64-class mode; per-frequency alpha errors")
    ap.add_argument("--max-subspace", type=int, default=64, help="Davidson trial-space limit")
    ap.add_argument("--sigma-batch", type=int, default=8, help="trial vectors per sigma call (--accuracy-at-scale)")
    ap.add_argument("--batch", action="store_true",
                    help="three uneven systems (8/60, 12/90, 18/120) solved as one batch and one by one")
    ap.add_argument("--adjoint", action="store_true",
                    help="gradients of alpha w.r.t. the operators and a static field (use --workload 20x150)")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = WORKLOADS[args.workload]
    if args.gemm:
        run_gemm(args)
        return
    if args.sigma:
        run_sigma(args)
        return
    if args.vector_kernels:
        run_vector_kernels(args)
        return
    if args.accuracy_at_scale:
        run_accuracy_at_scale(args)
        return
    if args.adjoint:
        run_adjoint(args)
        return
    if args.batch:
        run_batch(args)
        return
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import synth
    import paper_2307_14296_b300 as pk
    torch.cuda.set_device(local)
    w = WORKLOAD
    o, v = w["n_occ"], w["n_vir"]
    inst = synth.make_instance(o, v, seed=synth.DEFAULT_SEED + rank)
    omegas = np.linspace(w["w_min"], w["w_max"], w["n_freq"])
    prec = prec_of(pk, args.precision)
    ctx = pk.Context(local, precision=prec, tol=w["tol"], ground_tol=1e-8, max_subspace=args.max_subspace, batch=8,
                     maxit=80)
    blocks = [inst.blocks[k] for k in synth.CLASSES]
    # pinned host copies of the inputs (for the end-to-end measurement)
    pinned = [torch.from_numpy(np.ascontiguousarray(b)).pin_memory() for b in [inst.fock] + blocks + [inst.ops]]
    h2d = sum(p.numel() * p.element_size() for p in pinned)
    host = [p.numpy() for p in pinned]
    ctx.cclr_set_hamiltonian(o, v, host[0], host[1:7])

    def step():
        st = {}
        e, it = ctx.cc_ground()
        s = ctx.cclr_get_stats()
        st["ground_iters"] = it
        st["launches"] = s["kernel_launches"]
        st["phase"] = {"ground": s["total_seconds"], "ground_refine": s["refine_seconds"]}
        st["refine_products"] = s["refine_vectors"]
        ctx.cc_lambda()
        s = ctx.cclr_get_stats()
        st["launches"] += s["kernel_launches"]
        st["lambda_sigma"] = s["sigma_vectors"]
        st["refine_products"] += s["refine_vectors"]
        st["phase"]["lambda"] = s["total_seconds"]
        st["phase"]["lambda_refine"] = s["refine_seconds"]
        ctx.cc_lr_solve(host[7], omegas, w["gamma"])
        s = ctx.cclr_get_stats()
        st["lr_sigma"] = s["sigma_vectors"]
        st["refine_products"] += s["refine_vectors"]
        st["launches"] += s["kernel_launches"]
        st["phase"]["lr_solve"] = s["total_seconds"]
        st["phase"]["lr_sigma"] = s["sigma_seconds"]
        st["phase"]["lr_refine"] = s["refine_seconds"]
        st["final_residual"] = s["max_residual"]
        resp = ctx.cc_response_function()
        s = ctx.cclr_get_stats()
        st["launches"] += s["kernel_launches"]
        st["hessian"] = s["sigma_vectors"]
        st["phase"]["response_function"] = s["total_seconds"]
        st["resp"] = resp
        return st

    for _ in range(args.warmup):
        step()
    ctx.cclr_kernel_profile(True)
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    with Clocks(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            stats.append(step())
        ev1.record()
        torch.cuda.synchronize()
    prof = ctx.cclr_kernel_profile(False)
    barrier(world)
    t_local = ev0.elapsed_time(ev1) / 1e3 / args.steps
    t_step = allreduce(t_local, world, "max")
    n_prod = statistics.mean(s["ground_iters"] + s["lambda_sigma"] + s["lr_sigma"] + s["hessian"] for s in stats)

    def step_cmac(st):   # sigma-type products at the sigma count, Hessian products at their own
        return (sigma_cmac(o, v) * (st["ground_iters"] + st["lambda_sigma"] + st["lr_sigma"])
                + hessian_cmac(o, v) * st["hessian"])
    flops = 8 * statistics.mean(step_cmac(s) for s in stats)
    value = allreduce(flops / t_step / 1e12, world, "sum")

    # end to end through the C ABI: pinned host inputs copied in, response function copied out
    e2e = None
    if not args.no_e2e:
        barrier(world)
        t0 = time.perf_counter()
        ctx.cclr_set_hamiltonian(o, v, host[0], host[1:7])
        st = step()
        t_e2e = allreduce(time.perf_counter() - t0, world, "max")
        e2e = dict(value=allreduce(8 * step_cmac(st) / t_e2e / 1e12, world, "sum"), unit="TFLOP/s",
                   h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(st["resp"].nbytes), seconds=t_e2e)

    # plain-FP64 comparison at full size: one FP64 right sigma vector timed alone (outside the
    # timed region); the measured FP64-vs-mixed comparison of whole solves is the 12/90 replica
    # in accuracy_vs_fp64
    fp64 = None
    if rank == 0:
        x = synth.random_vector((1, ctx.N), 5, 5, 1e-3)
        ctx.cclr_sigma(x, side=0, precision=pk.FP64)
        t0 = time.perf_counter()
        ctx.cclr_sigma(x, side=0, precision=pk.FP64)
        fp64_sigma = time.perf_counter() - t0
        fp64 = dict(sigma_seconds=fp64_sigma,
                    step_seconds_extrapolated=fp64_sigma * statistics.mean(step_cmac(s) for s in stats) / sigma_cmac(o, v),
                    note="extrapolated, not measured: this step's work (Hessian products at their own cost) in "
                         "units of one FP64 sigma")
        if args.workload == "30x200":
            fp64["step_seconds_measured_lower_bound"] = FP64_STEP_30x200["lower_bound_seconds"]
            fp64["measured_how"] = FP64_STEP_30x200["how"]
            fp64["speedup_lower_bound"] = FP64_STEP_30x200["lower_bound_seconds"] / t_step
    # per-kernel shares: one extra untimed step with CUDA events around every launch
    breakdown = None
    if rank == 0 and not args.no_breakdown:
        ctx.cclr_kernel_profile(True)
        ctx.cclr_kernel_breakdown()
        step()
        ctx.cclr_kernel_profile(False)
        bd = ctx.cclr_kernel_breakdown()
        tot = sum(ms for _, ms in bd.values())
        top = sorted(bd.items(), key=lambda kv: -kv[1][1])[:12]
        breakdown = dict(note="one untimed step, CUDA events around every launch", total_ms=tot,
                         kernels=[dict(name=k, launches=n, ms=ms, share=ms / tot) for k, (n, ms) in top])
    # the next rows on the same converged state: CC-CI response function (no Hessian products)
    # and the four lowest EOM-EE roots (right sigma Davidson)
    extra = None
    if rank == 0 and not args.no_extra:
        t0 = time.perf_counter()
        ci = ctx.cc_response_function_ci()
        t_ci = time.perf_counter() - t0
        alpha_ci = -ci
        n0 = ctx.cclr_get_stats()["sigma_vectors"]
        t0 = time.perf_counter()
        roots, eom_its = ctx.cc_eom_ee(4)
        t_eom = time.perf_counter() - t0
        n_eom = ctx.cclr_get_stats()["sigma_vectors"] - n0
        extra = dict(cc_ci_seconds=t_ci,
                     cc_ci_alpha_mean_last_freq=[float(np.trace(alpha_ci[-1]).real / 3),
                                                 float(np.trace(alpha_ci[-1]).imag / 3)],
                     eom_ee=dict(workload="4 lowest roots of the benchmark system (split-BF16)",
                                 roots=[[float(r.real), float(r.imag)] for r in roots], iterations=eom_its,
                                 sigma_products=n_eom, seconds=t_eom),
                     eom_ee_accuracy=eom_replica(pk, synth))
    # accuracy of the mixed-precision step against the FP64 path, on the 12/90 replica (the FP64
    # step at the full workload takes ~13 min): 16 frequencies, every component of alpha
    accuracy = None
    if rank == 0 and not args.no_accuracy and prec != pk.FP64:
        accuracy = accuracy_vs_fp64(pk, synth)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        tf, dt, desc = oracle_sample()
        t1, tf1 = oracle_sigma_one_thread()
        cpu = dict(value=tf, unit="TFLOP/s", cores=len(os.sched_getaffinity(0)), kind="oracle", sample=desc,
                   one_thread_sigma=dict(seconds=t1, tflops=tf1, sample="one oracle right sigma at n_occ=8, n_vir=60, "
                                                                        "BLAS limited to 1 thread"))

    if rank != 0:
        return
    pk_, src = peaks()
    peak = pk_.get("bf16_tflops_sustained", pk_["bf16_tflops"])
    alpha = -stats[-1]["resp"]
    # Roofline of the tensor-core kernels on the BF16 flops of the slice or digit products the
    # method needs for the operands of each launch, counted by the library (8 per complex MAC and
    # product: 3 slice products in split BF16, 6 in the FP32-class split, 15 digit pairs for full
    # FP64-class operands and 9 for coarse corrections); beside it the rate of the complex
    # products themselves (8 flops per complex MAC: FP64-equivalent for the FP64-class kernel).
    per_kernel = {}
    for name, pr in (("k_tc_zgemm", prof), ("k_tc_zgemm_x", prof["f64"])):
        ms = pr["ms"] / args.steps
        per_kernel[name] = dict(
            kernel_ms_per_step=ms, launches_per_step=pr["launches"] / args.steps,
            achieved_tflops=(pr["flops_exec"] / args.steps / (ms * 1e-3) / 1e12 if ms > 0 else None),
            achieved_rule="8 BF16 flops x complex MACs x slice or digit products of each launch (library count)",
            complex_product_tflops=(pr["flops_useful"] / args.steps / (ms * 1e-3) / 1e12 if ms > 0 else None))
    dom = max(per_kernel, key=lambda k: per_kernel[k]["kernel_ms_per_step"])
    achieved = per_kernel[dom]["achieved_tflops"]
    line = dict(
        metric=METRIC, value=value, unit="TFLOP/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=1e3 * t_step, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="bf16x3+f64" if prec != pk.FP64 else "f64", data="synthetic", config=config_dict(args),
        s_per_alpha=statistics.mean(s["phase"]["lr_solve"] + s["phase"]["response_function"] for s in stats) / w["n_freq"],
        s_per_alpha_note="linear-response solves (with their FP64 refinement) + response function per frequency; "
                         "ground state and Lambda (once per Hamiltonian) in phase_seconds",
        s_per_step_per_freq=t_step / w["n_freq"],
        sigma_products_per_step=n_prod,
        final_response_residual=max(s["final_residual"] for s in stats),
        phase_seconds={k: statistics.mean(s["phase"][k] for s in stats) for k in stats[0]["phase"]},
        counts={k: statistics.mean(s[k] for s in stats)
                for k in ("ground_iters", "lambda_sigma", "lr_sigma", "hessian", "refine_products")},
        roofline=dict(bound="tensor", kernel=dom, achieved=achieved, peak=peak, unit="TFLOP/s",
                      frac=(achieved / peak if achieved else None), traffic=None,
                      traffic_note="DRAM bytes of this kernel are measured with ncu on a small case, outside this run",
                      peak_source=f"bf16_tflops_sustained of {src} MEASURED_PEAKS",
                      kernels=per_kernel),
        cpu_baseline=cpu, e2e=e2e, fp64=fp64, kernel_breakdown=breakdown, accuracy_vs_fp64=accuracy,
        next_rows=extra,
        gpu_launches=int(sum(s["launches"] for s in stats)),
        clocks=clk.summary(),
        alpha_mean_last_freq=[float(np.trace(alpha[-1]).real / 3), float(np.trace(alpha[-1]).imag / 3)],
    )
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
