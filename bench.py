#!/usr/bin/env python
"""Benchmark of the loop-estimate path: deflated loop estimates per second at a 1e-10 true residual.

Workload (plain FP64 on the GPU): 8^3 x 16 lattice, seeded near-identity SU(3) links with the
spread tuned to a mean plaquette of 0.6, kappa swept over {0.150, 0.155, 0.157}, 50 Z(4) noises,
GMRES-DR(60,30) on M and MINRES-DR(60,30) on M' = M gamma_5 for the special right-hand side,
GMRES-Proj(30) noise solves to a 1e-10 true residual, 30 deflation eigenvectors, 7-term
perturbative and degree-6 polynomial subtraction, all six subtraction modes and nine operators.

One step = one complete loop estimate (special solves, polynomial, hopping traces, 1/xi', 50 noise
solves, subtraction vectors and contractions) at one kappa; successive steps cycle through the
kappa sweep.  value = estimates (noises) of all ranks / wall time of the timed steps (max over
ranks), so the one-time setup is amortised over the 50 noises.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (8, 8, 8, 16)
KAPPAS = (0.150, 0.155, 0.157)
NNOISE, BLOCK = 50, 50
M_DR, K_DR = 60, 30
K_PS, NPOLY = 7, 6
TOL, TOL_SPECIAL = 1e-10, 1e-12
LINK_SEED, NOISE_SEED, PLAQ = 2024, 1, 0.6
WORKLOAD = "8^3x16 plain FP64, kappa {0.150,0.155,0.157}, 50 Z4 noises, GMRES-DR(60,30)+MINRES-DR(60,30), Q=30, PS K=7, POLY n=6, all 6 modes x 9 operators"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 2 DFMA / clock / SM at the 2070 MHz maximum clock
WILSON_FLOPS = 1368        # per site per right-hand side (1320 for P, 48 for 1 - kappa P)
L2_FLUSH_BYTES = 512 << 20
MULTIDOT_DRAM_RATIO = 1.011  # ncu: (318.4 + 397.0) MB DRAM over (314.6 + 393.2) MB compulsory, two launches
M_INNER_MIXED = 40         # GMRES cycle length of the reduced-precision inner solves


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-dslash", action="store_true")
    ap.add_argument("--batch", action="store_true", help="also measure the uneven multi-lattice batch")
    ap.add_argument("--no-defl", action="store_true")
    ap.add_argument("--case", default=None,
                    choices=["gmres-cycle", "gmres-cycle-f32", "dslash-packed", "dslash-half", "defl-tensor"],
                    help="run one small kernel case for profiling instead of the benchmark: one GMRES(30) "
                         "cycle on 50 noises of the 8^3x16 workload (FP64, or FP32 storage)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def make_links(rank):
    from paper_1903_06986_gb300 import synth
    eps = synth.eps_for_plaquette(DIMS, PLAQ, LINK_SEED)
    return synth.su3_links(DIMS, eps, LINK_SEED + rank), eps


# ---------------------------------------------------------------- clocks during the timed region
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append(dict(sm=float(p[1]), smax=float(p[2]), power=float(p[3]), hw=p[5], hwt=p[6], swt=p[7],
                                 swpc=p[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        load = [r for r in rows if r["power"] > 200.0] or rows
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("swpc", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r["sm"] for r in load])), "sm_max_mhz": rows[0]["smax"],
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(load)}


# ---------------------------------------------------------------- CPU oracle, bounded sample
def oracle_sample(U):
    """Time the oracle on a bounded sample of the same workload and extrapolate to estimates/s.

    Sample (kappa = 0.157): one GMRES-DR(60,30) cycle and one more (setup solve rate and residual
    reduction per cycle), one GMRES-Proj cycle for one noise over that deflation space (noise-solve
    rate and reduction per cycle), the subtraction vectors and 6 x 9 contractions of one noise,
    and 12 probes of the hopping traces.  Cycle counts to the tolerances are extrapolated from the
    observed per-cycle residual reductions; the result counts the oracle's own work only."""
    from oracle import krylov as Kr, lattice as L, operators as O, rng, subtract as S
    kappa = 0.157
    A = lambda v: L.flat(L.wilson(U, kappa, L.unflat(v, DIMS)))
    t0 = time.perf_counter()
    b0 = L.flat(rng.z4_noise(NOISE_SEED, rng.NOISE_SPECIAL, DIMS))
    _, info, defl = Kr.gmres_dr(A, b0, M_DR, K_DR, 1e-30, 2)
    t_dr = (time.perf_counter() - t0) / 2.0
    rho_dr = info["resid"][1] / info["resid"][0]
    cyc_special = int(np.ceil(np.log(TOL_SPECIAL / info["resid"][0]) / np.log(min(rho_dr, 0.999)))) + 1
    t1 = time.perf_counter()
    eta = rng.z4_noise(NOISE_SEED, 0, DIMS)
    x, pinfo = Kr.gmres_proj(A, L.flat(eta), defl, M_DR - K_DR, 1e-30, 2)
    t_proj = (time.perf_counter() - t1) / 2.0
    rho_p = pinfo["resid"][1] / pinfo["resid"][0]
    cyc_noise = int(np.ceil(np.log(TOL / pinfo["resid"][0]) / np.log(min(rho_p, 0.999)))) + 1
    t2 = time.perf_counter()
    xf = L.unflat(x, DIMS)
    Af = lambda f: L.wilson(U, kappa, f)
    xp = S.hop_series(U, kappa, eta, K_PS)
    xq = S.poly_apply(Af, np.ones(NPOLY + 1), eta)
    E = defl["V"][:, :K_DR]
    lam = np.ones(K_DR)
    for w in (xf, xf - xp, xf - xq, xf - S.defl_vector(E, lam, eta), xf - xp, xf - xq):
        O.per_t(O.densities(U, kappa, eta, w))
    t_sub = time.perf_counter() - t2
    t3 = time.perf_counter()
    z = np.zeros(L.field_shape(DIMS, (12,)), dtype=np.complex128)
    for a in range(12):
        z[a][0, 0, 0, 0, a // 3, a % 3] = 1.0
    w = z
    for k in range(1, K_PS):
        w = L.hop(U, w)
        O.densities(U, kappa, z, w)
    nprobe = 12 * int(np.prod(S.default_spacing(DIMS, K_PS)))
    t_probe = (time.perf_counter() - t3) / 12 * nprobe
    setup = 2 * cyc_special * t_dr + t_probe
    per_noise = cyc_noise * t_proj + t_sub
    rate = NNOISE / (setup + NNOISE * per_noise)
    sample = ("oracle on 8^3x16 kappa=0.157: 2 GMRES-DR(60,30) cycles (%.1fs/cycle, %d cycles to %.0e "
              "extrapolated, x2 for MINRES-DR), 2 GMRES-Proj cycles of 1 noise (%.1fs/cycle, %d cycles to %.0e "
              "extrapolated), subtraction+contractions of 1 noise (%.1fs), 12 of %d hopping-trace probes; "
              "rate = 50 / (setup + 50 x per-noise)" % (t_dr, cyc_special, TOL_SPECIAL, t_proj, cyc_noise, TOL,
                                                        t_sub, nprobe))
    return rate, sample, time.perf_counter() - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


# ---------------------------------------------------------------- reference arm (the oracle)
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    U, _ = make_links(0)
    times, rates = [], []
    for i in range(args.warmup + args.steps):
        rate, sample, dt = oracle_sample(U)
        if i >= args.warmup:
            times.append(dt)
            rates.append(rate)
    value = float(np.mean(rates))
    line = {"metric": "deflated loop estimates/s at 1e-10 true residual", "value": value,
            "unit": "estimates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "lattice": "8x8x8x16", "noises": NNOISE},
            "cpu_baseline": {"value": value, "unit": "estimates/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "estimates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- GPU arm
DSLASH_DIMS = (24, 24, 24, 32)   # the paper's large lattice (Sec. 7); fields exceed L2 at nrhs >= 2
def _measured_hbm_gbs(default=6789.6):
    """Copy bandwidth measured on this GPU pool (MEASURED_PEAKS.json beside this file), else the
    last measured value."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return default


HBM_PEAK_GBS = _measured_hbm_gbs()


def dslash_rates(torch):
    """Wilson operator throughput on the 24^3x32 lattice: the FP64 operator of the plain path
    (canonical layout) and the packed operators of the mixed-precision inner solver (FP32, FP16 and
    BF16 fields; FP32 links, recon 12 and 18).  Algorithmic bytes per launch: each spinor read once
    and written once (nrhs x V x 24 reals each way) plus the links once (4 x V x 18 or 12 reals);
    flops 1368 per site and right-hand side.
    CUDA events on the library stream, 2 warm-up and 5 timed launches; fields exceed L2 for nrhs > 1."""
    from paper_1903_06986_gb300 import lqcd, synth
    ctx = lqcd.Context(DSLASH_DIMS, recon=12)
    V = int(np.prod(DSLASH_DIMS))
    U = torch.from_numpy(synth.su3_links(DSLASH_DIMS, 0.4323, 7)).cuda()
    packed_links = {12: ctx.pack_links_f32(U, 12), 18: ctx.pack_links_f32(U, 18)}
    out = {}
    cases = [("f64", 18, 1), ("f64", 18, 8), ("f32packed", 12, 1), ("f32packed", 12, 8), ("f32packed", 12, 16),
             ("f32packed", 18, 8), ("f16packed", 12, 1), ("f16packed", 12, 8), ("f16packed", 12, 16),
             ("bf16packed", 12, 8)]
    for prec, recon, nrhs in cases:
        x = ctx.noise_z4(3, 0, nrhs)
        lw = 4
        if prec == "f64":
            y = torch.empty_like(x)
            fn = lambda: ctx.wilson_apply(U, 0.157, x, y)
            w, lreals, lw = 8, 18, 8
        elif prec in ("f16packed", "bf16packed"):
            hp = lqcd.PREC_F16 if prec == "f16packed" else lqcd.PREC_BF16
            x = ctx.pack_half(x, hp)
            y = torch.empty_like(x)
            Up = packed_links[recon]
            fn = lambda: ctx.wilson_apply_half(Up, recon, 0.157, x, y, prec=hp)
            w, lreals = 2, recon
        else:
            x = ctx.pack_f32(x)
            y = torch.empty_like(x)
            Up = packed_links[recon]
            fn = lambda: ctx.wilson_apply_packed(Up, recon, 0.157, x, y)
            w, lreals = 4, recon
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            fn()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 5 / 1000.0
        nbytes = nrhs * V * 48 * w + V * 4 * lreals * lw
        gbs = nbytes / t / 1e9
        tf = 1368.0 * V * nrhs / t / 1e12
        out["%s_recon%d_rhs%d" % (prec, recon, nrhs)] = {
            "ms": round(t * 1e3, 4), "GB/s": round(gbs, 1), "TFLOP/s": round(tf, 4),
            "frac_hbm": round(gbs / HBM_PEAK_GBS, 4),
            "frac_fp64": round(tf / FP64_PEAK_TFLOPS, 4) if prec == "f64" else None}
        del x, y
    ctx.close()
    return {"lattice": "24x24x24x32", "bytes": "nrhs*V*24 reals read+written + links once",
            "hbm_peak_gbs": HBM_PEAK_GBS, "results": out}


DEFL_DIMS = (24, 24, 24, 32)
DEFL_K, DEFL_NRHS = 200, 16


def deflation_rates(torch):
    """HFES projection gamma_5 V' diag(d) V'^dag eta (Sec. 5.4) on the 24^3x32 lattice with 200
    deflation vectors and 16 Z(4) noises: FP64 CUDA-core kernels against the split-precision
    tcgen05 kernels (bf16 slices, FP64 accuracy).  The vectors are seeded Gaussian (the projection's
    cost does not depend on their values).  CUDA events on the library stream, 1 warm-up and 3 timed
    projections per engine; the operands (17 GB of vectors, 71 GB of slices) exceed L2 by far.
    Algorithmic bytes of the tensor-core launches per projection: the two slice copies of V' read
    once (7 bf16 slices per real entry, in row tiles of 128 vectors for V'^dag eta and in K chunks
    of 32 vectors for V' C), the noise slice read once, the output fields written once."""
    from paper_1903_06986_gb300 import lqcd
    ctx = lqcd.Context(DEFL_DIMS)
    V = int(np.prod(DEFL_DIMS))
    n = 12 * V
    k, nrhs = DEFL_K, DEFL_NRHS
    gen = torch.Generator(device="cuda").manual_seed(5)
    E = torch.randn((k, n), dtype=torch.complex128, device="cuda", generator=gen)
    E /= torch.linalg.vector_norm(E, dim=1, keepdim=True)
    lam = (0.05 + 0.01 * np.arange(k)) * np.where(np.arange(k) % 2 == 0, 1.0, -1.0)
    defl = ctx.defl_import(E.reshape((k,) + tuple(ctx.field(1).shape[1:])), lam.astype(np.complex128))
    del E
    eta = ctx.noise_z4(9, 0, nrhs)
    d = 1.0 / lam
    out = {}

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1000.0, r

    ctx.set_defl_engine(lqcd.DEFL_FP64)
    t64, y64 = timed(lambda: ctx.deflate_project(defl, eta, d))
    ctx.set_defl_engine(lqcd.DEFL_TENSOR)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.deflate_project(defl, eta, d)                 # makes the slices of V' (once per space)
    torch.cuda.synchronize()
    t_slice = time.perf_counter() - t0
    ctx.timing(True)
    ctx.timing_reset()
    ttc, ytc = timed(lambda: ctx.deflate_project(defl, eta, d))
    tm = ctx.timing_read()
    ctx.timing(False)
    ctx.set_defl_engine(lqcd.DEFL_FP64)
    err = float((ytc - y64).abs().max().item() / y64.abs().max().item())
    L_re = 2 * n
    np16 = max(16, ((2 * nrhs + 15) // 16) * 16)
    bytes_alg = 14.0 * k * L_re + 2.0 * np16 * L_re + 14.0 * L_re * (((k + 31) // 32) * 32) + 8.0 * nrhs * L_re
    ms_t, nl_t, _ = tm["tensor"]
    per_proj = ms_t / 1000.0 / 4                      # 4 projections ran with timing on (1 warm + 3 timed)
    gbs = bytes_alg / per_proj / 1e9
    emu_flops = 8.0 * k * nrhs * n * 2                # the FP64 complex products emulated (two contractions)
    out = {"lattice": "24x24x24x32", "k": k, "nrhs": nrhs, "fp64_ms": round(t64 * 1e3, 3),
           "tensor_ms": round(ttc * 1e3, 3), "speedup": round(t64 / ttc, 2), "slice_setup_s": round(t_slice, 3),
           "max_rel_diff_vs_fp64": err,
           "tensor_kernel": {"launches_per_projection": nl_t / 4, "ms_per_projection": round(per_proj * 1e3, 3),
                             "algorithmic_bytes": bytes_alg, "GB/s": round(gbs, 1),
                             "frac_hbm": round(gbs / HBM_PEAK_GBS, 4),
                             "fp64_equivalent_tflops": round(emu_flops / per_proj / 1e12, 3)},
           "breakdown_ms": {kk: round(v[0] / 4, 3) for kk, v in tm.items() if v[0] > 0}}
    defl.close()
    ctx.close()
    return out


BATCH_SHAPES = ((8, 8, 8, 8), (12, 12, 12, 12), (12, 12, 12, 24), (16, 16, 16, 16))
BATCH_NOISE = 40
BATCH_KAPPA = 0.150


def batching_rates(torch):
    """Uneven multi-lattice batch: loop estimates of 40 noises each (kappa 0.150, the method
    parameters of the main workload, 1e-10 true residual, block width picked by the autotuner) on
    8^4, 12^4, 12^3x24 and 16^4 lattices (links of the same generator and plaquette): first one
    after another with direct launches (this pass also makes each context's workspace), then all
    four concurrently (lqcd_batch_loop_estimate, Krylov cycles replayed from CUDA graphs, captured
    during the pass).  Wall time per variant; estimates/s = 160 / time.  About two minutes, so it
    runs only with --batch."""
    from paper_1903_06986_gb300 import lqcd, synth
    probs = []
    for i, dims in enumerate(BATCH_SHAPES):
        eps = synth.eps_for_plaquette(dims, PLAQ, LINK_SEED + 10 + i)
        U = torch.from_numpy(synth.su3_links(dims, eps, LINK_SEED + 10 + i)).cuda()
        probs.append(dict(ctx=lqcd.Context(dims, recon=12), links=U, kappa=BATCH_KAPPA, seed=NOISE_SEED,
                          nnoise=BATCH_NOISE, block=0, m=M_DR, k=K_DR, K=K_PS, npoly=NPOLY, tol=TOL,
                          tol_special=TOL_SPECIAL, max_cycles=400))
    keys = ("seed", "nnoise", "block", "m", "k", "K", "npoly", "tol", "tol_special", "max_cycles")

    def sequential(graphs):
        for p in probs:
            p["ctx"].set_graphs(graphs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = [p["ctx"].loop_estimate(p["links"], p["kappa"], **{k: p[k] for k in keys}) for p in probs]
        torch.cuda.synchronize()
        return time.perf_counter() - t0, res

    def concurrent():
        for p in probs:
            p["ctx"].set_graphs(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = lqcd.batch_loop_estimate(probs)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, res

    t_dir, r_dir = sequential(False)
    t_cc, r_cc = concurrent()
    for a, b in zip(r_dir, r_cc):
        if not (a["converged"] and b["converged"]) or max(a["max_true_resid"], b["max_true_resid"]) > TOL:
            raise RuntimeError("batched loop estimate did not reach the tolerance")
    n = BATCH_NOISE * len(probs)
    out = {"lattices": ["x".join(map(str, d)) for d in BATCH_SHAPES], "noises_each": BATCH_NOISE,
           "kappa": BATCH_KAPPA, "method": "as the main workload, FP64",
           "autotuned_block": [r["block"] for r in r_cc],
           "per_lattice_s_direct": [round(r["seconds_setup"] + r["seconds_noise"], 3) for r in r_dir],
           "sequential_direct": {"s": round(t_dir, 3), "estimates_per_s": n / t_dir},
           "concurrent_graphs": {"s": round(t_cc, 3), "estimates_per_s": n / t_cc},
           "speedup_concurrent_vs_direct": t_dir / t_cc,
           "max_abs_diff_concurrent_vs_direct": float(max(np.abs(a["mean"] - b["mean"]).max()
                                                          for a, b in zip(r_dir, r_cc)))}
    for p in probs:
        p["ctx"].close()
    return out


def run_case(args):
    """Small fixed workloads for ncu captures (no timing output): one GMRES(30) cycle on the 50 noises
    of the 8^3x16 workload (FP64, or the mixed solver's FP32 cycle), or four applications of the
    packed FP32 or FP16 operator (recon 12, 8 right-hand sides) on the 24^3x32 lattice."""
    import torch
    from paper_1903_06986_gb300 import build, lqcd, synth
    build.build()
    if args.case == "defl-tensor":
        # 12^3x24, 128 vectors, 16 Z(4) noises: slices of V' 3.6 GB, two projections
        dims = (12, 12, 12, 24)
        ctx = lqcd.Context(dims)
        n = 12 * int(np.prod(dims))
        gen = torch.Generator(device="cuda").manual_seed(5)
        E = torch.randn((128, n), dtype=torch.complex128, device="cuda", generator=gen)
        lam = np.linspace(0.05, 0.5, 128).astype(np.complex128)
        defl = ctx.defl_import(E.reshape((128,) + tuple(ctx.field(1).shape[1:])), lam)
        eta = ctx.noise_z4(9, 0, 16)
        ctx.set_defl_engine(lqcd.DEFL_TENSOR)
        for _ in range(2):
            ctx.deflate_project(defl, eta, 1.0 / lam)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "launches": ctx.launches}))
        return
    if args.case in ("dslash-packed", "dslash-half"):
        ctx = lqcd.Context(DSLASH_DIMS, recon=12)
        U = torch.from_numpy(synth.su3_links(DSLASH_DIMS, 0.4323, 7)).cuda()
        Up = ctx.pack_links_f32(U, 12)
        half = args.case == "dslash-half"
        x = ctx.pack_half(ctx.noise_z4(3, 0, 8)) if half else ctx.pack_f32(ctx.noise_z4(3, 0, 8))
        y = torch.empty_like(x)
        for _ in range(4):
            if half:
                ctx.wilson_apply_half(Up, 12, 0.157, x, y)
            else:
                ctx.wilson_apply_packed(Up, 12, 0.157, x, y)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "launches": ctx.launches}))
        return
    U = torch.from_numpy(synth.su3_links(DIMS, 0.4323, LINK_SEED)).cuda()
    ctx = lqcd.Context(DIMS)
    etas = ctx.noise_z4(NOISE_SEED, 0, NNOISE)
    if args.case == "gmres-cycle":
        x, info, _ = ctx.gmresdr_solve(U, KAPPAS[-1], etas, M_DR - K_DR, 0, 1e-30, 1)
    else:
        _, _, defl = ctx.gmresdr_solve(U, KAPPAS[-1], etas[:1].contiguous(), M_DR - K_DR, 4, 1e-3, 5,
                                       want_defl=True)
        x, info = ctx.proj_solve(U, KAPPAS[-1], defl, etas, M_DR - K_DR, 1e-6, 1, prec=1)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "matvecs": info["matvecs"], "launches": ctx.launches}))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args)
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1903_06986_gb300 import build, lqcd
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    U, eps = make_links(rank)
    ctx = lqcd.Context(DIMS, recon=12)     # the synthetic links are SU(3)
    Ud = torch.from_numpy(U).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stats = []

    def step(i, links, prec=0):
        kappa = KAPPAS[i % len(KAPPAS)]
        r = ctx.loop_estimate(links, kappa, NOISE_SEED, NNOISE, BLOCK, M_DR, K_DR, K_PS, NPOLY, TOL, TOL_SPECIAL,
                              max_cycles=1000, prec=prec, m_inner=M_INNER_MIXED if prec else 0)
        if not r["converged"] or r["max_true_resid"] > TOL:
            raise RuntimeError("loop estimate did not reach the tolerance: %g" % r["max_true_resid"])
        stats.append(dict(kappa=kappa, setup_s=r["seconds_setup"], noise_s=r["seconds_noise"],
                          mv_setup=r["matvecs_setup"], mv_noise=r["matvecs_noise"], resid=r["max_true_resid"],
                          mean=r["mean"], stderr=r["stderr"]))
        return r

    for i in range(args.warmup):
        step(i, Ud)
    stats.clear()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- timed region (device-resident inputs)
    clocks = Clocks(local)
    barrier()
    clocks.start()
    launches0 = ctx.launches
    ctx.timing(True)
    ctx.timing_reset()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for i in range(args.steps):
        flush.zero_()                                   # flush L2 between steps
        step(args.warmup + i, Ud)
    ev1.record()
    barrier()
    t_dev = ev0.elapsed_time(ev1) / 1000.0
    tm = ctx.timing_read()
    tbytes = ctx.timing_bytes()
    ctx.timing(False)
    launches = ctx.launches - launches0
    clk = clocks.stop()
    stats_fp64 = list(stats[:args.steps])
    t_max = t_dev
    if world > 1:
        t = torch.tensor([t_dev], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    value = NNOISE * args.steps * world / t_max

    # ---- end to end through the public API: links from pinned host memory every step, results to host
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else args.steps
    Uh = torch.from_numpy(U).pin_memory()
    h2d = Uh.numel() * 16
    d2h = 0
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        flush.zero_()
        links = Uh.to("cuda", non_blocking=True)
        r = step(args.warmup + i, links)
        d2h = sum(r[k].nbytes for k in ("per_noise", "per_t", "addback", "mean", "stderr", "lam", "poly_a"))
    barrier()
    t_e2e = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([t_e2e], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_e2e = float(t.item())
    e2e_value = NNOISE * e2e_steps * world / t_e2e

    # ---- the same steps with mixed-precision noise solves (GMRES-Proj with FP32 arithmetic and FP32,
    # FP16 or BF16 storage inside FP64 defect correction, stopped on the FP64 true residual); setup,
    # series, projections and contractions FP64.  Every estimate is compared with the FP64 run's.
    mixed = None
    if not args.no_mixed:
        mixed = {}
        for name, prec in (("fp32", 1), ("fp16", 2), ("bf16", 3)):
            step(0, Ud, prec=prec)
            stats.clear()
            barrier()
            ctx.timing(True)
            ctx.timing_reset()
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            m0.record()
            for i in range(args.steps):
                flush.zero_()
                step(args.warmup + i, Ud, prec=prec)
            m1.record()
            barrier()
            tm_mixed = m0.elapsed_time(m1) / 1000.0
            tmm = ctx.timing_read()
            ctx.timing(False)
            ms_ = stats[:args.steps]
            diff = [np.abs(a["mean"] - b["mean"]) for a, b in zip(ms_, stats_fp64)]
            mixed[name] = {
                "value": NNOISE * args.steps * world / tm_mixed, "unit": "estimates/s",
                "speedup_vs_fp64": t_max / tm_mixed,
                "noise_phase_estimates_per_s": NNOISE * len(ms_) / sum(x["noise_s"] for x in ms_),
                "noise_phase_speedup_vs_fp64": (sum(x["noise_s"] for x in stats_fp64) /
                                                sum(x["noise_s"] for x in ms_)),
                "max_true_resid": max(x["resid"] for x in ms_),
                "estimate_vs_fp64": {
                    "max_abs_diff": float(max(d.max() for d in diff)),
                    "max_rel_diff": float(max((d / np.maximum(np.abs(b["mean"]), 1e-300)).max()
                                              for d, b in zip(diff, stats_fp64))),
                    "max_diff_over_stderr": float(max((d / np.maximum(b["stderr"], 1e-300)).max()
                                                      for d, b in zip(diff, stats_fp64)))},
                "matvecs_per_noise": float(np.mean([x["mv_noise"] / NNOISE for x in ms_])),
                "breakdown_ms": {k: round(v[0], 1) for k, v in tmm.items()},
                "launches": int(sum(v[1] for v in tmm.values())),
                "precision": "%s storage of the inner Krylov basis and deflation space, FP32 arithmetic, inside "
                             "FP64 defect correction (true residual FP64), GMRES-Proj(%d)" % (name.upper(), M_INNER_MIXED)}
        stats.clear()

    # ---- roofline of the dominant kernel class (device time over the timed region)
    dom = max(tm, key=lambda k: tm[k][0])
    ms, nl, units = tm[dom]
    flops_per_unit = {"wilson": WILSON_FLOPS, "dot": 8.0, "axpy": 8.0, "combine": 8.0, "norm": 4.0, "contract": None}
    fpu = flops_per_unit.get(dom)
    achieved = (units * fpu / (ms / 1000.0) / 1e12) if (fpu and ms > 0) else None
    roofline = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None, "traffic": None,
                "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived; probe measured 1.155 at 1.94 GHz)",
                "avg_launch_ms": ms / max(nl, 1), "launches": nl,
                "breakdown_ms": {k: round(v[0], 1) for k, v in tm.items()},
                "class_tflops": {k: round(v[2] * flops_per_unit[k] / (v[0] / 1000.0) / 1e12, 4)
                                 for k, v in tm.items() if flops_per_unit.get(k) and v[0] > 0}}
    if dom == "dot" and tbytes.get("dot", 0) > 0:
        # DRAM bytes per launch: the class's compulsory bytes per launch (recorded by the library
        # for every timed launch) times the DRAM / compulsory ratio that ncu measured on launches of
        # the same kernel (GMRES cycle of this workload, profiles/multidot_fp64_8x8x8x16_50rhs.md)
        roofline["traffic"] = MULTIDOT_DRAM_RATIO * tbytes["dot"] / max(nl, 1)
        roofline["traffic_source"] = ("compulsory bytes per launch x %.3f (ncu dram__bytes_read+write over "
                                      "compulsory bytes, multidot on 8^3x16, 50 rhs)" % MULTIDOT_DRAM_RATIO)
        roofline["compulsory_gbs"] = tbytes["dot"] / (ms / 1000.0) / 1e9
    w = tm["wilson"]
    if w[0] > 0:
        roofline["wilson_fp64_tflops"] = w[2] * WILSON_FLOPS / (w[0] / 1000.0) / 1e12

    dslash = None if args.no_dslash else dslash_rates(torch)
    deflation = None
    if not args.no_defl:
        try:
            deflation = deflation_rates(torch)
        except Exception as e:  # reported, not fatal
            deflation = {"error": str(e)[:300]}
    batching = None
    if args.batch:
        try:
            batching = batching_rates(torch)
        except Exception as e:  # reported, not fatal: the headline numbers above stand on their own
            batching = {"error": str(e)[:300]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, sample, _ = oracle_sample(U)
        cpu = {"value": rate, "unit": "estimates/s", "cores": cpu_cores(), "kind": "oracle", "sample": sample}

    if rank == 0:
        st = stats_fp64
        line = {"metric": "deflated loop estimates/s at 1e-10 true residual", "value": value, "unit": "estimates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "lattice": "8x8x8x16", "noises_per_step": NNOISE,
                           "kappas": list(KAPPAS), "link_eps": eps, "l2": "flushed between steps (512 MiB write)",
                           "parallelism": "independent gauge configuration per rank" if world > 1 else "single GPU"},
                "gpu_launches": launches,
                "noise_phase_estimates_per_s": NNOISE * len(st) / sum(s["noise_s"] for s in st),
                "setup_s_per_step": float(np.mean([s["setup_s"] for s in st])),
                "matvecs_per_noise": float(np.mean([s["mv_noise"] / NNOISE for s in st])),
                "max_true_resid": max(s["resid"] for s in st),
                "roofline": roofline,
                "e2e": {"value": e2e_value, "unit": "estimates/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h), "steps": e2e_steps},
                "clocks": clk, "cpu_baseline": cpu, "mixed_precision": mixed, "dslash": dslash,
                "deflation_tensor_cores": deflation,
                "batching": batching}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
